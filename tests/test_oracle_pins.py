"""Pins for the CPU oracle against facts that do not come from the oracle itself.

Each test checks the oracle against the paper or plain mathematics:
closed-form cell counts (Eq. 1 and the stacking identity of Sec. 2), the
inverse of the hash, a hand-worked automaton example, textbook Life patterns,
and an array-shift brute force of the automaton on tiny domains.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_2208_11617_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
GOLDEN_RATIO_32 = 0x9E3779B9
M32 = 0xFFFFFFFF


# ---------------------------------------------------------------- hash pins
def _inv_xorshift(y, s):
    x = y
    for _ in range(32 // s + 1):
        x = y ^ (x >> s)
    return x & M32


def _inv_fmix32(h):
    """Inverse of the MurmurHash3 finaliser, from modular inverses of its multipliers."""
    h = _inv_xorshift(h, 16)
    h = (h * pow(0xC2B2AE35, -1, 1 << 32)) & M32
    h = _inv_xorshift(h, 13)
    h = (h * pow(0x85EBCA6B, -1, 1 << 32)) & M32
    h = _inv_xorshift(h, 16)
    return h


def test_golden_ratio_increment_is_floor_2_32_over_phi():
    # 2^32 / phi = 2^31 (sqrt 5 - 1) ; floor via integer square root
    val = (math.isqrt(5 << 62) - (1 << 31))
    assert val == GOLDEN_RATIO_32


@pytest.mark.parametrize("x", [0, 1, 2, 0xFFFFFFFF, 0x12345678, 0x22081161, 1 << 31, 1023 * 1024 + 5])
def test_splitmix32_inverts_to_counter(x):
    h = oracle.splitmix32(x)
    assert _inv_fmix32(h) == (x + GOLDEN_RATIO_32) & M32


def test_splitmix32_is_a_bijection_on_a_block():
    xs = np.arange(1 << 16, dtype=np.uint64)
    hs = {oracle.splitmix32(int(x)) for x in xs}
    assert len(hs) == len(xs)


# ---------------------------------------------------------------- cell counts
@pytest.mark.parametrize("m", [1, 2, 3, 4])
def test_cell_count_closed_form(m):
    for n in list(range(0, 25)) + [63, 100]:
        assert oracle.count_cells(m, n) == math.comb(n + m, m), (m, n)


def test_cell_count_stacking_identity():
    # V(Delta^{m+1}) is the sum of the volumes of its stacked m-simplices (Sec. 2)
    for m in (1, 2, 3):
        for n in range(0, 20):
            assert oracle.count_cells(m + 1, n) == sum(oracle.count_cells(m, i) for i in range(n + 1))


@pytest.mark.parametrize("m,n,expected", [(2, 1023, 524_800), (3, 1023, 179_481_600),
                                          (4, 127, 11_716_640), (2, 4095, 8_390_656),
                                          (2, 32767, 536_887_296)])
def test_cell_count_workload_sizes(m, n, expected):
    assert oracle.count_cells(m, n) == expected == math.comb(n + m, m)


def test_cell_count_degenerate():
    assert oracle.count_cells(2, 0) == 1
    assert oracle.count_cells(3, -1) == 0


# ---------------------------------------------------------------- write test
def _box_cells(m, n):
    """All cells of the bounding box filtered by the simplex predicate (brute force)."""
    return [x for x in itertools.product(range(n + 1), repeat=m) if sum(x) <= n]


@pytest.mark.parametrize("m,n", [(2, 0), (2, 1), (2, 9), (3, 6), (4, 4)])
def test_accum_adds_once_to_every_domain_cell(m, n):
    # brute force over the bounding box: domain cells (sum <= n) gain `add`
    # exactly once per call, wrapping mod 2^32; every other cell is unchanged
    rng = np.random.default_rng(m * 100 + n)
    data = rng.integers(0, 1 << 32, size=(n + 1,) * m, dtype=np.uint64).astype(np.uint32)
    data.reshape(-1)[0] = 0xFFFFFFFF                    # wraps to add - 1
    once = oracle.accum(m, n, data, 7)
    twice = oracle.accum(m, n, once, 7)
    inside = np.zeros(data.shape, dtype=bool)
    for x in _box_cells(m, n):
        inside[x] = True
    assert inside.sum() == math.comb(n + m, m)
    d64 = data.astype(np.uint64)
    assert (once[inside] == ((d64[inside] + 7) % (1 << 32)).astype(np.uint32)).all()
    assert (twice[inside] == ((d64[inside] + 14) % (1 << 32)).astype(np.uint32)).all()
    assert (once[~inside] == data[~inside]).all() and (twice[~inside] == data[~inside]).all()
    assert once.reshape(-1)[0] == 6
    # the total grows by add x C(n + m, m) per call (mod 2^64 here: no overflow)
    assert int(twice.astype(np.uint64).sum()) - int(once.astype(np.uint64).sum()) == \
        7 * math.comb(n + m, m) - (1 << 32) * int(((once[inside].astype(np.uint64) + 7) >> 32).sum())


@pytest.mark.parametrize("m,n", [(2, 0), (2, 1), (2, 7), (3, 5), (4, 4), (2, 30), (3, 11)])
def test_write_support_and_values(m, n):
    seed = 0xDEADBEEF
    out = oracle.write(m, n, seed)
    D = n + 1
    inside = np.zeros(out.shape, dtype=bool)
    for x in _box_cells(m, n):
        inside[x] = True
    flat = out.reshape(-1)
    ins = inside.reshape(-1)
    # outside cells untouched
    assert not flat[~ins].any()
    # every written value decodes to seed ^ (row-major index on side n + 1)
    for lin in np.flatnonzero(ins):
        x = np.unravel_index(lin, out.shape)
        expect_lin = 0
        for xi in x:
            expect_lin = expect_lin * D + int(xi)
        assert (_inv_fmix32(int(flat[lin])) - GOLDEN_RATIO_32) & M32 == seed ^ expect_lin


# ---------------------------------------------------------------- initial state
def test_init_matches_threshold_rule_and_rate():
    m, n, seed = 2, 1023, inputs.DEFAULT_SEED
    thr = inputs.bernoulli_threshold(0.5)
    assert thr == 1 << 31
    g = oracle.ca_init(m, n, seed, thr)
    cells = math.comb(n + 2, 2)
    live = int(g.sum())
    assert abs(live - cells / 2) < 6 * math.sqrt(cells / 4)
    # spot-check the rule cell by cell on a strip, outside cells zero
    for x1 in range(0, n + 1, 97):
        for x2 in range(0, n + 1):
            if x1 + x2 <= n:
                h = oracle.splitmix32(seed ^ (x1 * (n + 1) + x2))
                assert g[x1, x2] == (1 if h < thr else 0)
            else:
                assert g[x1, x2] == 0


def test_init_threshold_is_strict():
    """A cell is alive iff its hash is strictly below the threshold: with the
    threshold equal to one cell's hash that cell is dead, one above it alive."""
    seed, n = 77, 20
    for m, (x1, x2, x3) in ((2, (3, 5, 0)), (3, (2, 4, 6))):
        D = n + 1
        lin = x1 * D + x2 if m == 2 else (x1 * D + x2) * D + x3
        cell = (x1, x2) if m == 2 else (x1, x2, x3)
        h = oracle.splitmix32(seed ^ lin)
        assert oracle.ca_init(m, n, seed, h)[cell] == 0
        assert oracle.ca_init(m, n, seed, h + 1)[cell] == 1


def test_bernoulli_thresholds():
    assert inputs.bernoulli_threshold(0.4) == 1717986918
    assert inputs.bernoulli_threshold(0.3) == 1288490188
    assert inputs.bernoulli_threshold(0) == 0


# ---------------------------------------------------------------- automaton
def _read_golden_life(path):
    steps = {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, _, cells = line.partition(":")
        steps[int(k)] = {tuple(int(v) for v in c.split(",")) for c in cells.split()}
    return steps


def test_life_hand_worked_delta2():
    steps = _read_golden_life(os.path.join(GOLDEN, "life_delta2_n2_all_alive.txt"))
    n = 2
    g = np.zeros((3, 3), dtype=np.uint8)
    for c in steps[0]:
        g[c] = 1
    birth, survive = inputs.B3S23
    for s in range(1, max(steps) + 1):
        g, live = oracle.ca_step(2, n, birth, survive, g)
        got = {tuple(int(v) for v in c) for c in np.argwhere(g)}
        assert got == steps[s], s
        assert live == len(steps[s])


def _place(n, cells, m=2):
    g = np.zeros((n + 1,) * m, dtype=np.uint8)
    for c in cells:
        g[c] = 1
    return g


def _cells(g):
    return {tuple(int(v) for v in c) for c in np.argwhere(g)}


def test_life_block_and_beehive_are_still():
    n = 40
    block = [(5, 5), (5, 6), (6, 5), (6, 6)]
    hive = [(12, 11), (12, 12), (13, 10), (13, 13), (14, 11), (14, 12)]
    g = _place(n, block + hive)
    birth, survive = inputs.B3S23
    for _ in range(3):
        g, live = oracle.ca_step(2, n, birth, survive, g)
        assert _cells(g) == set(block + hive)
        assert live == 10


def test_life_blinker_period_two():
    n = 40
    horiz = {(10, 9), (10, 10), (10, 11)}
    vert = {(9, 10), (10, 10), (11, 10)}
    g = _place(n, horiz)
    birth, survive = inputs.B3S23
    g, _ = oracle.ca_step(2, n, birth, survive, g)
    assert _cells(g) == vert
    g, _ = oracle.ca_step(2, n, birth, survive, g)
    assert _cells(g) == horiz


def test_life_glider_moves_one_diagonal_per_four_steps():
    n = 60
    glider = {(0, 1), (1, 2), (2, 0), (2, 1), (2, 2)}
    start = {(r + 5, c + 5) for r, c in glider}
    g = _place(n, start)
    birth, survive = inputs.B3S23
    final, live = oracle.ca_run(2, n, 8, birth, survive, g)
    assert _cells(final) == {(r + 2, c + 2) for r, c in start}
    assert list(live) == [5] * 9


def test_all_dead_stays_dead_and_outside_never_lives():
    for m, rule in ((2, inputs.B3S23), (3, inputs.B5S45)):
        n = 9
        g = np.zeros((n + 1,) * m, dtype=np.uint8)
        final, live = oracle.ca_run(m, n, 5, rule[0], rule[1], g)
        assert not final.any() and not live.any()
    # birth on zero neighbours: every dead domain cell is born, nothing outside
    n = 6
    g = np.zeros((n + 1, n + 1), dtype=np.uint8)
    out, live = oracle.ca_step(2, n, 1, 0, g)
    assert live == math.comb(n + 2, 2)
    idx = np.indices(out.shape).sum(0)
    assert (out == (idx <= n)).all()


def _shift_sum_step(grid, n, birth, survive):
    """Array-shift restatement: pad with dead cells, add the 3^m - 1 shifted copies."""
    m = grid.ndim
    D = n + 1
    inside = np.indices(grid.shape).sum(0) <= n
    g = np.where(inside, grid, 0).astype(np.int64)
    pad = np.pad(g, 1)
    cnt = np.zeros_like(g)
    for off in itertools.product((-1, 0, 1), repeat=m):
        if any(off):
            cnt += pad[tuple(slice(1 + o, 1 + o + D) for o in off)]
    btab = np.array([(birth >> k) & 1 for k in range(3 ** m)], dtype=np.uint8)
    stab = np.array([(survive >> k) & 1 for k in range(3 ** m)], dtype=np.uint8)
    new = np.where(g == 1, stab[cnt], btab[cnt])
    return np.where(inside, new, 0).astype(np.uint8)


RULES_2D = [inputs.B3S23, (1 << 3 | 1 << 6, 1 << 2 | 1 << 3), (1 << 2, 0), (0b111111111, 0b101010101)]
RULES_3D = [inputs.B5S45, (1 << 4, 1 << 2 | 1 << 3 | 1 << 4), ((1 << 27) - 1, 1 << 26 | 1)]


@pytest.mark.parametrize("rule", RULES_2D)
@pytest.mark.parametrize("n", [0, 1, 2, 5, 17, 40])
def test_ca_step_2d_matches_shift_sum(rule, n):
    rng = np.random.default_rng(1000 + n)
    g = rng.integers(0, 2, size=(n + 1, n + 1), dtype=np.uint8)
    g = np.where(np.indices(g.shape).sum(0) <= n, g, 0).astype(np.uint8)
    for _ in range(3):
        ref = _shift_sum_step(g, n, *rule)
        got, live = oracle.ca_step(2, n, rule[0], rule[1], g)
        np.testing.assert_array_equal(got, ref)
        assert live == int(ref.sum())
        g = got


@pytest.mark.parametrize("rule", RULES_3D)
@pytest.mark.parametrize("n", [0, 1, 3, 8, 15])
def test_ca_step_3d_matches_shift_sum(rule, n):
    rng = np.random.default_rng(2000 + n)
    g = rng.integers(0, 2, size=(n + 1,) * 3, dtype=np.uint8)
    g = np.where(np.indices(g.shape).sum(0) <= n, g, 0).astype(np.uint8)
    for _ in range(3):
        ref = _shift_sum_step(g, n, *rule)
        got, live = oracle.ca_step(3, n, rule[0], rule[1], g)
        np.testing.assert_array_equal(got, ref)
        assert live == int(ref.sum())
        g = got


def test_ca_step_ignores_outside_content():
    # a neighbour outside the domain is dead whatever the array holds there
    n = 12
    rng = np.random.default_rng(7)
    g = rng.integers(0, 2, size=(n + 1, n + 1), dtype=np.uint8)
    inside = np.indices(g.shape).sum(0) <= n
    clean = np.where(inside, g, 0).astype(np.uint8)
    a, la = oracle.ca_step(2, n, *inputs.B3S23, g)
    b, lb = oracle.ca_step(2, n, *inputs.B3S23, clean)
    np.testing.assert_array_equal(np.where(inside, a, 0), b)
    assert la == lb


def test_ca_run_live_counts_are_popcounts():
    n = 50
    g = oracle.ca_init(2, n, 5, inputs.bernoulli_threshold(0.5))
    final, live = oracle.ca_run(2, n, 7, *inputs.B3S23, g)
    cur = g
    for s in range(1, 8):
        cur, _ = oracle.ca_step(2, n, *inputs.B3S23, cur)
        assert live[s] == int(cur.sum())
    np.testing.assert_array_equal(final, cur)
    assert live[0] == int(g.sum())


# ---------------------------------------------------------------- block indicator
@pytest.mark.parametrize("m,n,rho", [(2, 63, 16), (2, 100, 16), (2, 1023, 16), (3, 63, 8),
                                     (3, 40, 8), (4, 31, 4), (4, 30, 8), (2, 5, 4),
                                     (2, 64, 16), (3, 48, 8), (4, 32, 8)])  # tiles holding one cell
def test_block_indicator_closed_form(m, n, rho):
    ind = oracle.block_indicator(m, n, rho)
    X = np.indices(ind.shape).sum(0)
    np.testing.assert_array_equal(ind, (rho * X <= n).astype(np.uint32))
    assert int(ind.sum()) == math.comb(n // rho + m, m)


def test_ca_cells_agrees_with_whole_step():
    for m, n, rule in ((2, 30, inputs.B3S23), (3, 12, inputs.B5S45)):
        rng = np.random.default_rng(m)
        g = rng.integers(0, 2, size=(n + 1,) * m, dtype=np.uint8)
        g = np.where(np.indices(g.shape).sum(0) <= n, g, 0).astype(np.uint8)
        ref = _shift_sum_step(g, n, *rule)
        coords = np.argwhere(np.indices(g.shape).sum(0) <= n)
        got = oracle.ca_cells(m, n, rule[0], rule[1], g, coords)
        np.testing.assert_array_equal(got, ref[tuple(coords.T)])


# ---------------------------------------------------------------- EDM (Table 1 test 3)
def test_edm_pythagorean_points():
    """Hand-worked example: points with integer distances (3-4-5, 5-12-13 and
    the 1-2-2 triple); cell (x1, x2) holds d(p[x1], p[n - x2])."""
    pts = np.array([[0, 0, 0], [3, 4, 0], [0, 0, 12], [1, 2, 2]], dtype=np.float32)
    d = oracle.edm(3, pts)
    want = {(0, 0): 3.0, (0, 1): 12.0, (0, 2): 5.0, (0, 3): 0.0,
            (1, 0): math.sqrt(12.0), (1, 1): 13.0, (1, 2): 0.0,
            (2, 0): math.sqrt(1 + 4 + 100), (2, 1): 0.0,
            (3, 0): 0.0}
    for (x1, x2), v in want.items():
        assert d[x1, x2] == pytest.approx(v, rel=1e-15)
    # outside the simplex nothing is written
    assert d[1, 3] == 0 and d[3, 3] == 0 and d[2, 2] == 0


@pytest.mark.parametrize("n,dim", [(0, 1), (1, 3), (30, 3), (57, 16), (40, 1)])
def test_edm_matches_scipy_cdist(n, dim):
    """The oracle's triangle is the upper triangle (diagonal included) of
    scipy's distance matrix, read with j = n - x2."""
    spatial = pytest.importorskip("scipy.spatial")
    pts = np.random.default_rng(n * 31 + dim).random((n + 1, dim), dtype=np.float32)
    ref = spatial.distance.cdist(pts.astype(np.float64), pts.astype(np.float64))
    d = oracle.edm(n, pts)
    x1, x2 = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    inside = x1 + x2 <= n
    np.testing.assert_allclose(d[inside], ref[x1[inside], n - x2[inside]], rtol=1e-14, atol=0)
    assert not d[~inside].any()
    # the anti-diagonal x1 + x2 = n is the matrix diagonal i = j: exactly zero
    assert not d[x1 + x2 == n].any()


def test_edm_cells_agree_with_whole_matrix():
    pts = inputs.edm_points(50, 5, seed=3)
    full = oracle.edm(50, pts)
    rng = np.random.default_rng(4)
    x1 = rng.integers(0, 51, 200)
    x2 = (rng.random(200) * (51 - x1)).astype(np.int64)
    c = np.stack([x1, x2], 1)
    np.testing.assert_array_equal(oracle.edm_cells(50, pts, c), full[x1, x2])
