"""GPU parity: every CUDA result against the CPU oracle, bit for bit.

All work here is integer, so the bar is exact equality (no tolerance).  Cases
span several tiles with ragged tails (n + 1 not a multiple of the tile side),
padded and unaligned array sides, degenerate sizes (n = 0), both maps (H and
the bounding box) and, at the full workload sizes, the launch configuration
the benchmark times, checked on whole grids where the oracle finishes in
seconds and on sampled cells or map-independent properties beyond that.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2208_11617_gb300 import inputs
from paper_2208_11617_gb300 import simplex as sx

pytestmark = pytest.mark.gpu

MODES = [sx.SIMPLEX_MODE_H, sx.SIMPLEX_MODE_BB, sx.SIMPLEX_MODE_BB_THREAD]
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    torch.cuda.init()
    yield
    assert sx.simplex_device_status() == 0


def _logical(t: torch.Tensor, mp, n):
    """View of the logical (n+1)^m block of a side^m device array, and the rest."""
    a = t.view(mp.shape).cpu().numpy()
    sl = tuple(slice(0, n + 1) for _ in range(mp.m))
    rest = a.copy()
    rest[sl] = 0
    return a[sl], rest


def _beta(m):
    return 2 if m <= 3 else m


# ---------------------------------------------------------------- write test
WRITE_CASES = [
    (2, 1023, 16, None, 2),        # 1024^2, 16 x 16 tiles, the write workload
    (2, 1000, 16, None, 2),        # ragged: 1001 not a multiple of 16, side not a multiple of 4
    (2, 1000, 16, 1004, 2),        # padded side, 16-byte rows
    (2, 0, 16, None, 2),
    (2, 5, 4, None, 2),
    (2, 4095, 32, None, 2),
    (3, 63, 4, None, 2),
    (3, 100, 8, None, 2),
    (3, 100, 8, None, 3),
    (3, 64, 16, 68, 2),
    (4, 31, 4, None, 4),
    (4, 127, 8, None, 4),          # 128^4, the m = 4 write workload
    (4, 127, 4, None, 4),
    (4, 40, 4, 44, 4),
    (4, 100, 8, 104, 4),           # ragged n, 8^4 tiles: multi-tile blocks, early stop on the diagonal
    (4, 60, 8, 62, 4),             # 8^4 tiles, side not a multiple of 4 (4-byte stores)
]


@pytest.mark.parametrize("case", WRITE_CASES)
@pytest.mark.parametrize("mode", MODES)
def test_write_matches_oracle(case, mode):
    m, n, block, side, beta = case
    mp = sx.simplex_map_create(m, n, 2, beta, block, side=side)
    seed = inputs.DEFAULT_SEED ^ (n * 7919)
    out = torch.zeros(mp.numel, dtype=torch.int32, device=DEV)
    sx.simplex_write(mp, out, seed, mode)
    torch.cuda.synchronize()
    got, rest = _logical(out, mp, n)
    ref = oracle.write(m, n, seed)
    np.testing.assert_array_equal(got.view(np.uint32), ref)
    assert not rest.any()


def test_write_leaves_outside_untouched():
    mp = sx.simplex_map_create(2, 500, 2, 2, 16, side=512)
    out = torch.full((mp.numel,), -7, dtype=torch.int32, device=DEV)
    sx.simplex_write(mp, out, 3)
    a = out.view(mp.shape).cpu().numpy()
    idx = np.indices(a.shape).sum(0)
    ref = oracle.write(2, 500, 3)
    np.testing.assert_array_equal(a[:501, :501][idx[:501, :501] <= 500].view(np.uint32),
                                  ref[idx[:501, :501] <= 500])
    assert (a[idx > 500] == -7).all()


# ---------------------------------------------------------------- coverage
VISIT_CASES = [(2, 1023, 16, 2), (2, 1000, 16, 2), (2, 77, 4, 2), (3, 100, 8, 2), (3, 63, 4, 2),
               (3, 100, 8, 3), (3, 255, 16, 2), (4, 31, 4, 4), (4, 63, 8, 4), (2, 0, 16, 2), (3, 0, 4, 2)]


@pytest.mark.parametrize("case", VISIT_CASES)
@pytest.mark.parametrize("mode", MODES)
def test_visit_counts_block_and_cell(case, mode):
    m, n, block, beta = case
    mp = sx.simplex_map_create(m, n, 2, beta, block)
    nb = (n + block) // block
    blk = torch.zeros(nb ** m, dtype=torch.int32, device=DEV)
    sx.simplex_visit_count(mp, blk, sx.SIMPLEX_LEVEL_BLOCK, mode)
    ref = oracle.block_indicator(m, n, block)
    np.testing.assert_array_equal(blk.view((nb,) * m).cpu().numpy().astype(np.uint32), ref)
    cell = torch.zeros(mp.numel, dtype=torch.int32, device=DEV)
    sx.simplex_visit_count(mp, cell, sx.SIMPLEX_LEVEL_CELL, mode)
    c = cell.view(mp.shape).cpu().numpy()
    inside = (np.indices(c.shape).sum(0) <= n).astype(np.int32)
    np.testing.assert_array_equal(c, inside)


# ---------------------------------------------------------------- automaton init
INIT_CASES = [(2, 4095, 128, None), (2, 1000, 32, 1008), (2, 1000, 64, 1008), (2, 0, 32, 16), (2, 17, 16, 32),
              (3, 255, 16, None), (3, 255, 32, None), (3, 200, 16, 208), (3, 0, 16, 16)]


@pytest.mark.parametrize("case", INIT_CASES)
def test_ca_init_matches_oracle(case):
    m, n, block, side = case
    mp = sx.simplex_map_create(m, n, 2, 2, block, side=side)
    thr = inputs.bernoulli_threshold(0.5 if m == 2 else 0.3)
    g = torch.zeros(mp.numel, dtype=torch.uint8, device=DEV)
    live = torch.zeros(1, dtype=torch.int64, device=DEV)
    sx.simplex_ca_init(mp, g, 1234, thr, live)
    got, rest = _logical(g, mp, n)
    ref = oracle.ca_init(m, n, 1234, thr)
    np.testing.assert_array_equal(got, ref)
    assert not rest.any()
    assert int(live.item()) == int(ref.sum())


# ---------------------------------------------------------------- automaton runs
def _gpu_run(mp, n, steps, rule, seed, thr, mode, use_graph=True):
    a = torch.zeros(mp.numel, dtype=torch.uint8, device=DEV)
    b = torch.zeros_like(a)
    sx.simplex_ca_init(mp, a, seed, thr)
    live = torch.zeros(steps + 1, dtype=torch.int64, device=DEV)
    fin = sx.simplex_ca_run(mp, a, b, steps, rule[0], rule[1], live, use_graph, mode)
    torch.cuda.synchronize()
    return fin, live.cpu().numpy().astype(np.uint64)


RUN_CASES = [
    # m, n, block, side, steps, rule, p, beta
    (2, 4095, 128, None, 100, inputs.B3S23, 0.5, 2),     # the m = 2 automaton at the oracle's size
    (2, 1000, 32, 1008, 30, inputs.B3S23, 0.5, 2),
    (2, 1000, 64, 1008, 30, inputs.B3S23, 0.5, 2),
    (2, 1000, 128, 1008, 30, inputs.B3S23, 0.5, 2),
    (2, 300, 32, 304, 20, (1 << 3 | 1 << 6, 1 << 2 | 1 << 3), 0.4, 2),   # B36/S23
    (2, 300, 64, 304, 5, (1, 0), 0.3, 2),                                  # birth on 0: tests the edge mask
    (2, 300, 128, 304, 5, (0x1FF, 0x1FF), 0.3, 2),
    (2, 0, 32, 16, 3, (1, 1), 0.5, 2),
    (2, 15, 32, 16, 5, inputs.B3S23, 0.5, 2),
    (2, 16, 32, 32, 5, inputs.B3S23, 0.5, 2),
    (3, 255, 16, None, 20, inputs.B5S45, 0.3, 2),
    (3, 255, 32, None, 20, inputs.B5S45, 0.3, 2),
    (3, 255, 16, None, 10, inputs.B5S45, 0.3, 3),
    (3, 200, 16, 208, 10, inputs.B5S45, 0.3, 2),
    (3, 200, 32, 208, 10, (1 << 4, 1 << 2 | 1 << 3 | 1 << 4), 0.4, 2),
    (3, 100, 16, 112, 4, (1, 0), 0.3, 2),
    (3, 0, 16, 16, 3, (1, 1), 0.5, 2),
    (3, 20, 16, 32, 6, inputs.B5S45, 0.5, 2),
]


@pytest.mark.parametrize("case", RUN_CASES)
@pytest.mark.parametrize("mode", MODES)
def test_ca_run_matches_oracle(case, mode):
    m, n, block, side, steps, rule, p, beta = case
    mp = sx.simplex_map_create(m, n, 2, beta, block, side=side)
    thr = inputs.bernoulli_threshold(p)
    seed = 99 + n
    fin, live = _gpu_run(mp, n, steps, rule, seed, thr, mode)
    got, rest = _logical(fin, mp, n)
    ref0 = oracle.ca_init(m, n, seed, thr)
    ref, ref_live = oracle.ca_run(m, n, steps, rule[0], rule[1], ref0)
    np.testing.assert_array_equal(got, ref)
    assert not rest.any()
    np.testing.assert_array_equal(live, ref_live)


@pytest.mark.parametrize("band", [-1, 2, 32])
@pytest.mark.parametrize("n,block,side", [(4095, 128, None), (1000, 32, 1008), (2047, 64, None)])
def test_ca_run_h2_forms_match_oracle(band, n, block, side):
    """Both forms of H for m = 2 (the single Eq. map2d grid, band = -1, and
    trapezoid bands) give the oracle's grid."""
    mp = sx.simplex_map_create(2, n, 2, 2, block, side=side, band=band)
    thr = inputs.bernoulli_threshold(0.5)
    fin, live = _gpu_run(mp, n, 12, inputs.B3S23, 31, thr, sx.SIMPLEX_MODE_H)
    got, rest = _logical(fin, mp, n)
    ref, ref_live = oracle.ca_run(2, n, 12, *inputs.B3S23, oracle.ca_init(2, n, 31, thr))
    np.testing.assert_array_equal(got, ref)
    assert not rest.any()
    np.testing.assert_array_equal(live, ref_live)


@pytest.mark.parametrize("band", [-1, 4])
def test_write_h2_forms_match_oracle(band):
    mp = sx.simplex_map_create(2, 1023, 2, 2, 16, band=band)
    out = torch.zeros(mp.numel, dtype=torch.int32, device=DEV)
    sx.simplex_write(mp, out, 77)
    np.testing.assert_array_equal(out.view(mp.shape).cpu().numpy().view(np.uint32), oracle.write(2, 1023, 77))


@pytest.mark.parametrize("launch", [1, 2, 3])
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,side,beta", [(255, None, 2), (200, 208, 2), (255, None, 3), (31, 32, 2), (1, 16, 2),
                                         (527, 528, 2), (600, 608, 2)])
def test_ca3_grid_and_persistent_forms_match_oracle(launch, mode, n, side, beta):
    """The m = 3 step in its three launch forms (one CTA per block of the map;
    the x-stream form: persistent CTAs streaming runs of tiles along x3
    through a ring of x-columns; the plane-stream form: persistent CTAs
    streaming 32 x 128 bricks along x1) gives the oracle's grid."""
    mp = sx.simplex_map_create(3, n, 2, beta, 32, side=side, launch=launch)
    assert mp.info.launch == launch
    thr = inputs.bernoulli_threshold(0.3)
    fin, live = _gpu_run(mp, n, 7, inputs.B5S45, 17, thr, mode)
    got, rest = _logical(fin, mp, n)
    ref, ref_live = oracle.ca_run(3, n, 7, *inputs.B5S45, oracle.ca_init(3, n, 17, thr))
    np.testing.assert_array_equal(got, ref)
    assert not rest.any()
    np.testing.assert_array_equal(live, ref_live)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,side,block,steps,rule,p", [
    (0, 16, 16, 3, inputs.B5S45, 0.5),
    (1, 16, 32, 3, (1, 1), 0.5),                      # birth on 0: every dead domain cell is born
    (31, 32, 32, 6, inputs.B5S45, 0.5),
    (127, None, 32, 6, (1 << 4, 1 << 5 | 1 << 6 | 1 << 7), 0.3),   # B4/S567: the general rule tables
    (128, 144, 16, 5, inputs.B5S45, 0.3),
    (160, 176, 32, 4, (0x7FFFFFF, 0x7FFFFFF), 0.2),   # every count turns a cell on
    (300, 304, 32, 5, inputs.B5S45, 0.3),
    (700, 704, 32, 2, (1 << 5 | 1 << 6, 1 << 4 | 1 << 5), 0.3),
])
def test_ca3_plane_stream_sizes_and_rules(mode, n, side, block, steps, rule, p):
    """The plane-stream step (launch 3) against the oracle on ragged and padded
    sides (n + 1 not a multiple of the 32 x 128 brick), degenerate sizes, both
    rule paths (or-k and the general tables) and rules that light cells next
    to the domain's faces."""
    mp = sx.simplex_map_create(3, n, 2, 2, block, side=side, launch=3)
    assert mp.info.launch == 3
    thr = inputs.bernoulli_threshold(p)
    fin, live = _gpu_run(mp, n, steps, rule, 29, thr, mode)
    got, rest = _logical(fin, mp, n)
    ref, ref_live = oracle.ca_run(3, n, steps, rule[0], rule[1], oracle.ca_init(3, n, 29, thr))
    np.testing.assert_array_equal(got, ref)
    assert not rest.any()
    np.testing.assert_array_equal(live, ref_live)


def test_ca3_plane_stream_single_steps_reuse_the_counter():
    """Consecutive simplex_ca_step calls (no graph) on one map share its work
    counter: each launch must leave it at zero for the next."""
    n = 255
    mp = sx.simplex_map_create(3, n, 2, 2, 32, launch=3)
    thr = inputs.bernoulli_threshold(0.3)
    a = torch.zeros(mp.numel, dtype=torch.uint8, device=DEV)
    b = torch.zeros_like(a)
    sx.simplex_ca_init(mp, a, 3, thr)
    ref = oracle.ca_init(3, n, 3, thr)
    for i in range(5):
        live = torch.zeros(1, dtype=torch.int64, device=DEV)
        mode = MODES[i % 3]
        sx.simplex_ca_step(mp, a, b, *inputs.B5S45, live, mode)
        ref, ref_live = oracle.ca_step(3, n, *inputs.B5S45, ref)
        got, _ = _logical(b, mp, n)
        np.testing.assert_array_equal(got, ref)
        assert int(live.item()) == ref_live
        a, b = b, a


def test_ca_step_by_step_equals_graph_run():
    mp = sx.simplex_map_create(2, 2047, 2, 2, 64)
    thr = inputs.bernoulli_threshold(0.5)
    fin_g, live_g = _gpu_run(mp, 2047, 9, inputs.B3S23, 5, thr, sx.SIMPLEX_MODE_H, use_graph=True)
    fin_s, live_s = _gpu_run(mp, 2047, 9, inputs.B3S23, 5, thr, sx.SIMPLEX_MODE_H, use_graph=False)
    assert torch.equal(fin_g, fin_s)
    np.testing.assert_array_equal(live_g, live_s)
    # replaying the cached graph gives the same answer again
    fin_g2, live_g2 = _gpu_run(mp, 2047, 9, inputs.B3S23, 5, thr, sx.SIMPLEX_MODE_H, use_graph=True)
    assert torch.equal(fin_g, fin_g2)


def test_ca_step_api_single_steps():
    m, n = 2, 777
    mp = sx.simplex_map_create(m, n, 2, 2, 32, side=784)
    thr = inputs.bernoulli_threshold(0.5)
    a = torch.zeros(mp.numel, dtype=torch.uint8, device=DEV)
    b = torch.zeros_like(a)
    sx.simplex_ca_init(mp, a, 42, thr)
    ref = oracle.ca_init(m, n, 42, thr)
    for _ in range(4):
        live = torch.zeros(1, dtype=torch.int64, device=DEV)
        sx.simplex_ca_step(mp, a, b, *inputs.B3S23, live)
        ref, ref_live = oracle.ca_step(m, n, *inputs.B3S23, ref)
        got, _ = _logical(b, mp, n)
        np.testing.assert_array_equal(got, ref)
        assert int(live.item()) == ref_live
        a, b = b, a


@pytest.mark.parametrize("m,n,block,side,steps", [(2, 1023, 128, None, 12), (2, 100, 32, 112, 5), (2, 0, 32, 16, 3),
                                                  (3, 200, 16, 208, 7), (3, 63, 32, None, 4)])
def test_ca_run_host_end_to_end(m, n, block, side, steps):
    """Host buffers in and out; only the domain moves, so host_out keeps a
    sentinel or gets 0 outside the domain and the oracle's grid inside."""
    mp = sx.simplex_map_create(m, n, 2, 2, block, side=side)
    rule = inputs.B3S23 if m == 2 else inputs.B5S45
    thr = inputs.bernoulli_threshold(0.5)
    init = oracle.ca_init(m, n, 7, thr)
    full = np.zeros(mp.shape, dtype=np.uint8)
    full[tuple(slice(0, n + 1) for _ in range(m))] = init
    h_in = torch.from_numpy(full.reshape(-1).copy()).pin_memory()
    h_out = torch.full((mp.numel,), 0xAB, dtype=torch.uint8).pin_memory()
    h_live = torch.zeros(steps + 1, dtype=torch.int64)
    a = torch.zeros(mp.numel, dtype=torch.uint8, device=DEV)
    b = torch.zeros_like(a)
    d_live = torch.zeros(steps + 1, dtype=torch.int64, device=DEV)
    sx.simplex_ca_run_host(mp, h_in, h_out, a, b, steps, *rule, d_live, h_live)
    ref, ref_live = oracle.ca_run(m, n, steps, *rule, init)
    got = h_out.numpy().reshape(mp.shape)
    idx = np.indices(mp.shape).sum(axis=0)
    inside = idx <= n
    refg = np.zeros(mp.shape, dtype=np.uint8)
    refg[tuple(slice(0, n + 1) for _ in range(m))] = ref
    np.testing.assert_array_equal(got[inside], refg[inside])
    assert np.isin(got[~inside], [0, 0xAB]).all()
    np.testing.assert_array_equal(h_live.numpy().astype(np.uint64), ref_live)


def test_ca_rejects_bad_layouts():
    mp = sx.simplex_map_create(2, 1000, 2, 2, 32)   # side 1001: rows not 16-byte aligned
    a = torch.zeros(mp.numel, dtype=torch.uint8, device=DEV)
    with pytest.raises(sx.SimplexError) as ei:
        sx.simplex_ca_step(mp, a, a.clone(), *inputs.B3S23)
    assert ei.value.code == sx.SIMPLEX_EINVAL
    mp = sx.simplex_map_create(2, 1023, 2, 2, 16)   # block 16 has no m = 2 step kernel
    a = torch.zeros(mp.numel, dtype=torch.uint8, device=DEV)
    with pytest.raises(sx.SimplexError) as ei:
        sx.simplex_ca_step(mp, a, a.clone(), *inputs.B3S23)
    assert ei.value.code == sx.SIMPLEX_EUNSUPPORTED
    mp = sx.simplex_map_create(2, 1023, 2, 2, 64)
    a = torch.zeros(mp.numel, dtype=torch.uint8, device=DEV)
    with pytest.raises(sx.SimplexError):
        sx.simplex_ca_step(mp, a, a, *inputs.B3S23)     # in == out
    mp4 = sx.simplex_map_create(4, 31, 2, 4, 16)
    a = torch.zeros(mp4.numel, dtype=torch.uint8, device=DEV)
    with pytest.raises(sx.SimplexError):
        sx.simplex_ca_step(mp4, a, a.clone(), *inputs.B3S23)


# ---------------------------------------------------------------- ACCUM
ACCUM_CASES = [(2, 1023, 16, None), (2, 1000, 16, 1004), (2, 1000, 16, 1001), (2, 0, 16, None), (2, 300, 64, None),
               (3, 100, 8, None), (3, 63, 4, 66), (3, 200, 16, None), (4, 20, 4, None), (4, 31, 8, None)]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("m,n,block,side", ACCUM_CASES)
def test_accum_matches_oracle(m, n, block, side, mode):
    """Two ACCUM launches (+5, then +2^32 - 3) on random data: domain cells
    gain 2 mod 2^32, every other cell -- outside the domain and padding -- is
    untouched; 16-byte and 4-byte paths (side % 4), m = 2, 3, 4."""
    mp = sx.simplex_map_create(m, n, 2, 2 if m <= 3 else m, block, side=side)
    rng = np.random.default_rng(n * 10 + m)
    init = rng.integers(0, 1 << 32, size=mp.shape, dtype=np.uint64).astype(np.uint32)
    d = torch.from_numpy(init.view(np.int32).reshape(-1).copy()).to(DEV)
    sx.simplex_accum(mp, d, 5, mode)
    sx.simplex_accum(mp, d, (1 << 32) - 3, mode)
    got = d.cpu().numpy().view(np.uint32).reshape(mp.shape)
    logical = tuple(slice(0, n + 1) for _ in range(m))
    ref = oracle.accum(m, n, oracle.accum(m, n, init[logical], 5), (1 << 32) - 3)
    np.testing.assert_array_equal(got[logical], ref)
    pad = np.ones(mp.shape, dtype=bool)
    pad[logical] = False
    np.testing.assert_array_equal(got[pad], init[pad])


# ---------------------------------------------------------------- full workload sizes
def test_ca_m3_full_size_steps_match_oracle():
    """m = 3, n = 1023, B5/S45, Bernoulli(0.3): first steps whole-grid against the
    oracle, then H and BB agree over all 50 steps."""
    w = inputs.CA_M3
    mp = sx.simplex_map_create(w.m, w.n, 2, 2, w.block)
    first = 3
    fin, live = _gpu_run(mp, w.n, first, w.rule, w.seed, w.threshold, sx.SIMPLEX_MODE_H)
    ref0 = oracle.ca_init(w.m, w.n, w.seed, w.threshold)
    ref, ref_live = oracle.ca_run(w.m, w.n, first, w.rule[0], w.rule[1], ref0)
    got, _ = _logical(fin, mp, w.n)
    np.testing.assert_array_equal(got, ref)
    np.testing.assert_array_equal(live, ref_live)
    del fin, got, ref, ref0
    fin_h, live_h = _gpu_run(mp, w.n, w.steps, w.rule, w.seed, w.threshold, sx.SIMPLEX_MODE_H)
    fin_b, live_b = _gpu_run(mp, w.n, w.steps, w.rule, w.seed, w.threshold, sx.SIMPLEX_MODE_BB)
    assert torch.equal(fin_h, fin_b)
    np.testing.assert_array_equal(live_h, live_b)
    assert live_h[-1] > 0


def test_ca_m2_full_length_matches_oracle():
    """m = 2 at the benchmark's size and length (n = 32767, 100 steps, B3/S23,
    Bernoulli(0.5), 128 x 128 tiles, graph-captured): the final grid and all
    101 live counts equal the oracle's whole run."""
    w = inputs.CA_M2
    mp = sx.simplex_map_create(w.m, w.n, 2, 2, w.block)
    fin, live = _gpu_run(mp, w.n, w.steps, w.rule, w.seed, w.threshold, sx.SIMPLEX_MODE_H)
    got = fin.view(mp.shape).cpu().numpy()
    del fin
    ref, ref_live = oracle.ca_run(w.m, w.n, w.steps, w.rule[0], w.rule[1],
                                  oracle.ca_init(w.m, w.n, w.seed, w.threshold))
    assert len(ref_live) == w.steps + 1
    np.testing.assert_array_equal(live, ref_live)
    np.testing.assert_array_equal(got, ref)


def test_ca_m3_full_size_matches_oracle():
    """The m = 3 automaton at the benchmark's size and length (n = 1023, 50
    steps, B5/S45, Bernoulli(0.3)) in the launch form the benchmark times (the
    plane stream): the final grid and all 51 live counts equal the oracle's
    whole run."""
    w = inputs.CA_M3
    mp = sx.simplex_map_create(w.m, w.n, 2, 2, w.block, launch=3)
    fin, live = _gpu_run(mp, w.n, w.steps, w.rule, w.seed, w.threshold, sx.SIMPLEX_MODE_H)
    got = fin.view(mp.shape).cpu().numpy()
    del fin
    ref, ref_live = oracle.ca_run(w.m, w.n, w.steps, w.rule[0], w.rule[1],
                                  oracle.ca_init(w.m, w.n, w.seed, w.threshold))
    assert len(ref_live) == w.steps + 1
    np.testing.assert_array_equal(live, ref_live)
    np.testing.assert_array_equal(got, ref)


def test_ca_m3_full_size_x_stream_equals_grid_form():
    """The x-stream form (launch 2, the faster m = 3 step) at n = 1023 over the
    workload's 50 steps gives the grid form's grids and live counts bit for
    bit (the grid form is checked against the oracle above)."""
    w = inputs.CA_M3
    mg = sx.simplex_map_create(w.m, w.n, 2, 2, w.block, launch=1)
    mx = sx.simplex_map_create(w.m, w.n, 2, 2, w.block, launch=2)
    assert mx.info.launch == 2 and mg.info.launch == 1
    fin_g, live_g = _gpu_run(mg, w.n, w.steps, w.rule, w.seed, w.threshold, sx.SIMPLEX_MODE_H)
    fin_x, live_x = _gpu_run(mx, w.n, w.steps, w.rule, w.seed, w.threshold, sx.SIMPLEX_MODE_H)
    assert torch.equal(fin_g, fin_x)
    np.testing.assert_array_equal(live_g, live_x)
    assert live_x[-1] > 0
    del fin_x
    # the bounding-box modes of the plane stream
    mp = sx.simplex_map_create(w.m, w.n, 2, 2, w.block, launch=3)
    for mode in (sx.SIMPLEX_MODE_BB, sx.SIMPLEX_MODE_BB_THREAD):
        fin_p, live_p = _gpu_run(mp, w.n, 4, w.rule, w.seed, w.threshold, mode)
        fin_g4, live_g4 = _gpu_run(mg, w.n, 4, w.rule, w.seed, w.threshold, sx.SIMPLEX_MODE_H)
        assert torch.equal(fin_p, fin_g4)
        np.testing.assert_array_equal(live_p, live_g4)


def test_ca_m2_full_size_matches_oracle():
    """m = 2, n = 32767, B3/S23, Bernoulli(0.5) in the benchmark's launch
    configuration (128 x 128 tiles, graph-captured): two whole steps against
    the oracle, H == BB over the 100 steps, and 4096 sampled cells of the last
    step recomputed one by one by the oracle."""
    w = inputs.CA_M2
    mp = sx.simplex_map_create(w.m, w.n, 2, 2, w.block)
    fin, live = _gpu_run(mp, w.n, 2, w.rule, w.seed, w.threshold, sx.SIMPLEX_MODE_H)
    ref0 = oracle.ca_init(w.m, w.n, w.seed, w.threshold)
    ref, ref_live = oracle.ca_run(w.m, w.n, 2, w.rule[0], w.rule[1], ref0)
    np.testing.assert_array_equal(fin.view(mp.shape).cpu().numpy(), ref)
    np.testing.assert_array_equal(live, ref_live)
    del fin, ref, ref0
    # 99 steps, then one more: compare sampled cells of step 100 with the oracle
    a = torch.zeros(mp.numel, dtype=torch.uint8, device=DEV)
    b = torch.zeros_like(a)
    sx.simplex_ca_init(mp, a, w.seed, w.threshold)
    live_h = torch.zeros(w.steps + 1, dtype=torch.int64, device=DEV)
    prev = sx.simplex_ca_run(mp, a, b, w.steps - 1, w.rule[0], w.rule[1], live_h[: w.steps])
    nxt = b if prev is a else a
    step_live = torch.zeros(1, dtype=torch.int64, device=DEV)
    sx.simplex_ca_step(mp, prev, nxt, w.rule[0], w.rule[1], step_live)
    torch.cuda.synchronize()
    prev_host = prev.view(mp.shape).cpu().numpy()
    last = nxt.view(mp.shape)
    rng = np.random.default_rng(2208)
    pts = []
    while len(pts) < 4096:
        x1, x2 = rng.integers(0, w.n + 1, size=2)
        if x1 + x2 <= w.n:
            pts.append((x1, x2))
    pts += [(0, 0), (0, w.n), (w.n, 0), (w.n // 2, w.n - w.n // 2), (127, 128), (128, 127)]
    coords = np.array(pts, dtype=np.int64)
    want = oracle.ca_cells(w.m, w.n, w.rule[0], w.rule[1], prev_host, coords)
    idx = torch.from_numpy(coords).to(DEV)
    got = last[idx[:, 0], idx[:, 1]].cpu().numpy()
    np.testing.assert_array_equal(got, want)
    # the bounding-box map computes the same 100 steps
    fin_b, live_b = _gpu_run(mp, w.n, w.steps, w.rule, w.seed, w.threshold, sx.SIMPLEX_MODE_BB)
    assert torch.equal(fin_b, nxt)
    live_all = live_h.cpu().numpy().astype(np.uint64)
    live_all[w.steps] = int(step_live.item())
    np.testing.assert_array_equal(live_b, live_all)
    assert int(fin_b.sum(dtype=torch.int64).item()) == int(live_b[-1])


def test_ca_m2_past_2_32_offsets_matches_oracle():
    """Size limit of 32-bit indexing: m = 2, n = 70000 on side 70016 (4.9 GB
    grids), so byte offsets and row-major indices pass 2^32 (the initial state
    hashes lin mod 2^32 on both sides).  The initial state and one step on the
    benchmark's 128 x 128 tiles equal the oracle's whole grids, the padding
    rows and columns stay zero, and the live counts agree."""
    n, side, w = 70000, 70016, inputs.CA_M2
    assert n * (n + 1) + n >= 1 << 32 and side * side > 1 << 32
    mp = sx.simplex_map_create(2, n, 2, 2, w.block, side=side)
    a = torch.zeros(mp.numel, dtype=torch.uint8, device=DEV)
    b = torch.zeros_like(a)
    live = torch.zeros(2, dtype=torch.int64, device=DEV)
    sx.simplex_ca_init(mp, a, w.seed, w.threshold, live[0:1])
    sx.simplex_ca_step(mp, a, b, w.rule[0], w.rule[1], live[1:2])
    torch.cuda.synchronize()
    live = live.cpu().tolist()

    def same(t, ref):
        g = t.view(side, side)
        assert not g[n + 1:].any() and not g[:, n + 1:].any()  # padding untouched
        for r0 in range(0, n + 1, 8192):
            r1 = min(n + 1, r0 + 8192)
            got = g[r0:r1, : n + 1].cpu().numpy()
            if not np.array_equal(got, ref[r0:r1]):
                bad = np.argwhere(got != ref[r0:r1])[:5]
                raise AssertionError(f"rows {r0}..{r1}: first mismatches {(bad + [r0, 0]).tolist()}")

    ref0 = oracle.ca_init(2, n, w.seed, w.threshold)
    same(a, ref0)
    assert live[0] == int(np.count_nonzero(ref0))
    del a
    ref1, live1 = oracle.ca_step(2, n, w.rule[0], w.rule[1], ref0)
    del ref0
    same(b, ref1)
    assert live[1] == live1


def test_ca_m3_past_2_32_offsets_matches_oracle():
    """The same limit for m = 3: n = 1700 on side 1712 (5.0 GB grids, offsets
    and row-major indices past 2^32; tile columns N = 64).  The initial state
    and one step of the grid form equal the oracle's whole grids with the
    padding zero; the x-stream and plane-stream forms' steps equal the grid
    form's."""
    n, side, w = 1700, 1712, inputs.CA_M3
    assert (n + 1) ** 3 > 1 << 32 and side ** 3 > 1 << 32
    mg = sx.simplex_map_create(3, n, 2, 2, 32, side=side, launch=1)
    mx = sx.simplex_map_create(3, n, 2, 2, 32, side=side, launch=2)
    mq = sx.simplex_map_create(3, n, 2, 2, 32, side=side, launch=3)
    a = torch.zeros(mg.numel, dtype=torch.uint8, device=DEV)
    b = torch.zeros_like(a)
    c = torch.zeros_like(a)
    live = torch.zeros(4, dtype=torch.int64, device=DEV)
    sx.simplex_ca_init(mg, a, w.seed, w.threshold, live[0:1])
    sx.simplex_ca_step(mg, a, b, w.rule[0], w.rule[1], live[1:2])
    sx.simplex_ca_step(mx, a, c, w.rule[0], w.rule[1], live[2:3])
    torch.cuda.synchronize()
    assert torch.equal(b, c)
    c.zero_()
    sx.simplex_ca_step(mq, a, c, w.rule[0], w.rule[1], live[3:4])
    torch.cuda.synchronize()
    assert torch.equal(b, c)
    del c
    live = live.cpu().tolist()
    assert live[1] == live[2] == live[3]

    def same(t, ref):
        g = t.view(side, side, side)
        assert not g[n + 1:].any() and not g[:, n + 1:].any() and not g[:, :, n + 1:].any()
        for r0 in range(0, n + 1, 64):
            r1 = min(n + 1, r0 + 64)
            got = g[r0:r1, : n + 1, : n + 1].cpu().numpy()
            if not np.array_equal(got, ref[r0:r1]):
                bad = np.argwhere(got != ref[r0:r1])[:5]
                raise AssertionError(f"planes {r0}..{r1}: first mismatches {(bad + [r0, 0, 0]).tolist()}")

    ref0 = oracle.ca_init(3, n, w.seed, w.threshold)
    same(a, ref0)
    assert live[0] == int(np.count_nonzero(ref0))
    del a
    ref1, live1 = oracle.ca_step(3, n, w.rule[0], w.rule[1], ref0)
    del ref0
    same(b, ref1)
    assert live[1] == live1


@pytest.mark.parametrize("n,block,side", [(255, 32, None), (200, 32, 208), (127, 16, None), (1023, 32, None),
                                          (63, 8, None)])
def test_h3_level_layout_matches_oracle(n, block, side):
    """The fully efficient H3 (one block range per stack level): automaton
    steps (tiles of 16 and 32) and the write test give the oracle's arrays."""
    mp = sx.simplex_map_create(3, n, 2, 2, block, side=side, layout=1)
    assert mp.info.layout == 1
    if block >= 16:
        thr = inputs.bernoulli_threshold(0.3)
        steps = 2 if n > 500 else 5
        fin, live = _gpu_run(mp, n, steps, inputs.B5S45, 23, thr, sx.SIMPLEX_MODE_H)
        got, rest = _logical(fin, mp, n)
        ref, ref_live = oracle.ca_run(3, n, steps, *inputs.B5S45, oracle.ca_init(3, n, 23, thr))
        np.testing.assert_array_equal(got, ref)
        assert not rest.any()
        np.testing.assert_array_equal(live, ref_live)
    if n <= 255:
        out = torch.zeros(mp.numel, dtype=torch.int32, device=DEV)
        sx.simplex_write(mp, out, 5)
        got, rest = _logical(out, mp, n)
        np.testing.assert_array_equal(got.view(np.uint32), oracle.write(3, n, 5))
        assert not rest.any()


# ---------------------------------------------------------------- r = 1/3, beta = 3 (m = 2)
@pytest.mark.parametrize("n,block,side", [(1023, 16, None), (1000, 16, 1004), (1295, 16, None), (35, 4, None),
                                          (0, 16, None), (400, 8, None)])
def test_r_third_write_and_visits_match_oracle(n, block, side):
    """The m = 2 map with r = 1/3, beta = 3: the write test gives the
    oracle's array, every block holding cells is visited once and every cell
    of the domain once (nothing outside)."""
    mp = sx.simplex_map_create(2, n, 3, 3, block, side=side)
    assert mp.info.r_inv == 3
    out = torch.zeros(mp.numel, dtype=torch.int32, device=DEV)
    sx.simplex_write(mp, out, 91)
    got, rest = _logical(out, mp, n)
    np.testing.assert_array_equal(got.view(np.uint32), oracle.write(2, n, 91))
    assert not rest.any()
    nb = (n + block) // block
    blk = torch.zeros(nb * nb, dtype=torch.int32, device=DEV)
    sx.simplex_visit_count(mp, blk, sx.SIMPLEX_LEVEL_BLOCK)
    np.testing.assert_array_equal(blk.view(nb, nb).cpu().numpy().astype(np.uint32), oracle.block_indicator(2, n, block))
    cell = torch.zeros(mp.numel, dtype=torch.int32, device=DEV)
    sx.simplex_visit_count(mp, cell, sx.SIMPLEX_LEVEL_CELL)
    c = cell.view(mp.shape).cpu().numpy()
    np.testing.assert_array_equal(c, (np.indices(c.shape).sum(0) <= n).astype(np.int32))


@pytest.mark.parametrize("n,block,side", [(1023, 64, None), (500, 32, 512), (1295, 128, 1296)])
def test_r_third_automaton_matches_oracle(n, block, side):
    """The automaton step on the r = 1/3 map (one CTA per block of the map)
    gives the oracle's grids and live counts."""
    mp = sx.simplex_map_create(2, n, 3, 3, block, side=side)
    thr = inputs.bernoulli_threshold(0.5)
    fin, live = _gpu_run(mp, n, 9, inputs.B3S23, 41, thr, sx.SIMPLEX_MODE_H)
    got, rest = _logical(fin, mp, n)
    ref, ref_live = oracle.ca_run(2, n, 9, *inputs.B3S23, oracle.ca_init(2, n, 41, thr))
    np.testing.assert_array_equal(got, ref)
    assert not rest.any()
    np.testing.assert_array_equal(live, ref_live)
