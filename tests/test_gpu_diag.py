"""GPU parity of the paper's diagnostic tests (Table 1): MAP and EDM.

MAP has no output besides the count of cells its threads map, which must be
the closed-form C(n + m, m) for both maps.  EDM is float32 on the GPU against
the oracle's double-precision distances of the same float32 points; the bound
is derived from the arithmetic: with u = 2^-24, each difference, square and
partial sum of d^2 = sum_k (a_k - b_k)^2 (non-negative terms, no cancellation)
adds at most u of relative error, so d^2 is within (dim + 2) u and its
correctly rounded square root within (dim / 2 + 2) u of the exact distance;
the test allows (dim + 4) u.  Zero distances (i = j) are exact.
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
U = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    torch.cuda.init()
    yield
    assert sx.simplex_device_status() == 0


# ---------------------------------------------------------------- MAP
MAP_CASES = [
    (2, 0, 16), (2, 1, 4), (2, 17, 4), (2, 1023, 16), (2, 1000, 16), (2, 4095, 32), (2, 32767, 16),
    (3, 0, 8), (3, 5, 4), (3, 63, 4), (3, 200, 8), (3, 1023, 8),
    (4, 0, 4), (4, 7, 4), (4, 31, 4), (4, 127, 4),
]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("m,n,block", MAP_CASES)
def test_map_test_maps_every_cell_once(m, n, block, mode):
    mp = sx.simplex_map_create(m, n, 2, 2 if m <= 3 else m, block)
    cells = torch.zeros(1, dtype=torch.int64, device=DEV)
    sx.simplex_map_test(mp, cells, mode)
    assert int(cells.item()) == math.comb(n + m, m) == oracle.count_cells(m, n)
    sx.simplex_map_test(mp, None, mode)  # the timed form: no output, must run
    torch.cuda.synchronize()


@pytest.mark.parametrize("n,block", [(1023, 16), (1295, 16), (32767, 16), (17, 4)])
def test_map_test_r_third_maps_every_cell_once(n, block):
    """MAP on the r = 1/3 map of m = 2: C(n + 2, 2) cells, each once."""
    mp = sx.simplex_map_create(2, n, 3, 3, block)
    cells = torch.zeros(1, dtype=torch.int64, device=DEV)
    sx.simplex_map_test(mp, cells)
    assert int(cells.item()) == math.comb(n + 2, 2)


def test_map_test_rejects_blocks_over_1024_threads():
    mp = sx.simplex_map_create(3, 100, 2, 2, 16)
    with pytest.raises(sx.SimplexError):
        sx.simplex_map_test(mp, None)


# ---------------------------------------------------------------- EDM
def _edm_gpu(mp, pts, mode, fill=-1.0):
    out = torch.full((mp.numel,), fill, dtype=torch.float32, device=DEV)
    sx.simplex_edm(mp, torch.from_numpy(pts).to(DEV), out, mode)
    torch.cuda.synchronize()
    return out.view(mp.shape).cpu().numpy().astype(np.float64)


EDM_CASES = [
    (0, 3, 16, None), (1, 3, 16, None), (15, 1, 16, None), (16, 3, 16, None), (100, 3, 32, 104),
    (1023, 3, 32, None), (1000, 16, 64, 1004), (1000, 2, 16, 1004), (2047, 3, 64, None), (300, 7, 32, 304),
]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,dim,block,side", EDM_CASES)
def test_edm_matches_oracle(n, dim, block, side, mode):
    pts = inputs.edm_points(n, dim, seed=n + dim)
    mp = sx.simplex_map_create(2, n, 2, 2, block, side=side)
    got = _edm_gpu(mp, pts, mode)
    ref = oracle.edm(n, pts)
    x1, x2 = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    inside = x1 + x2 <= n
    g, r = got[: n + 1, : n + 1], ref
    np.testing.assert_allclose(g[inside], r[inside], rtol=(dim + 4) * U, atol=0)
    assert (g[x1 + x2 == n] == 0).all()             # i = j: exactly zero
    assert (g[~inside] == -1).all()                 # outside the simplex: untouched
    full = got.copy()
    full[: n + 1, : n + 1] = -1
    assert (full == -1).all()                       # padding untouched


def test_edm_h_equals_bb_bitwise():
    n = 2047
    pts = inputs.edm_points(n, 3, seed=9)
    mp = sx.simplex_map_create(2, n, 2, 2, 32)
    a = _edm_gpu(mp, pts, sx.SIMPLEX_MODE_H)
    b = _edm_gpu(mp, pts, sx.SIMPLEX_MODE_BB)
    np.testing.assert_array_equal(a, b)


def test_edm_full_size_sampled():
    """The benchmark's workload (n = 32767, 3-D points, 32 x 32 tiles): sampled
    cells against the oracle computed one by one, plus the diagonal and the
    first row/column exactly where they are zero."""
    n, dim = inputs.EDM_N, inputs.EDM_DIM
    pts = inputs.edm_points(n, dim)
    mp = sx.simplex_map_create(2, n, 2, 2, inputs.EDM_BLOCK)
    out = torch.full((mp.numel,), -1.0, dtype=torch.float32, device=DEV)
    sx.simplex_edm(mp, torch.from_numpy(pts).to(DEV), out)
    rng = np.random.default_rng(5)
    x1 = rng.integers(0, n + 1, 20000)
    x2 = (rng.random(20000) * (n + 1 - x1)).astype(np.int64)
    x1 = np.concatenate([x1, [0, n, 0, n // 2, 1]])
    x2 = np.concatenate([x2, [n, 0, 0, n - n // 2, n - 1]])
    lin = torch.from_numpy(x1 * mp.side + x2).to(DEV)
    got = out[lin].cpu().numpy().astype(np.float64)
    ref = oracle.edm_cells(n, pts, np.stack([x1, x2], 1))
    np.testing.assert_allclose(got, ref, rtol=(dim + 4) * U, atol=0)
    # cells just past the diagonal stay untouched
    past = torch.from_numpy(np.array([1 * mp.side + n, n * mp.side + 1, (n // 2 + 1) * mp.side + n // 2 + 1])).to(DEV)
    assert (out[past] == -1).all()
