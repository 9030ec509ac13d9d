"""Host-side tests of libsimplex: exported symbols, the launch plan and the maps.

These run without a GPU: simplex_map_create / simplex_map_info /
simplex_map_block only touch host memory, and simplex_map_block evaluates the
same integer decode the kernels run, so the coverage of H is checked
exhaustively here (Def. 1: every block of the simplex gets exactly one CUDA
block).
"""
import collections
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_2208_11617_gb300 import simplex as sx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "simplex.h")).read()
    declared = set(re.findall(r"^(?:int|const char \*)\s*(simplex_\w+)\s*\(", hdr, flags=re.M))
    assert declared, "no declarations parsed"
    assert declared == set(sx.EXPORTED)
    for name in declared:
        assert hasattr(sx._lib, name), name
    assert "sm_103a" in sx.simplex_version()


def test_binding_fails_loudly_without_the_library(tmp_path):
    """A copy of the binding next to no libsimplex.so refuses to import: the
    product path has no CPU fallback."""
    import shutil
    import subprocess
    import sys
    pkg = tmp_path / "pkg_copy"
    pkg.mkdir()
    shutil.copy(os.path.join(ROOT, "paper_2208_11617_gb300", "simplex.py"), pkg / "simplex.py")
    (pkg / "__init__.py").write_text("")
    r = subprocess.run([sys.executable, "-c", "import pkg_copy.simplex"], cwd=tmp_path, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "no CPU fallback" in r.stderr


def test_product_package_never_touches_the_oracle():
    """Only tests, the smoke check and the bench's CPU legs may use oracle/:
    no file of the package imports it, loads its library or calls its C entry
    points (comments may mention it)."""
    pkg = os.path.join(ROOT, "paper_2208_11617_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath or "__pycache__" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                use = re.search(r"^\s*(import|from)\s+oracle\b|\boracle\.\w|liboracle|simplex_oracle|\boracle_\w+\s*\(",
                                text, flags=re.M)
                assert not use, (os.path.join(dirpath, f), use.group(0) if use else None)


# ------------------------------------------------------------------ plan sizes
@pytest.mark.parametrize("m,n,block", [(2, 1023, 16), (2, 32767, 128), (2, 4095, 128), (3, 1023, 32),
                                       (3, 1023, 16), (4, 127, 4), (4, 127, 8), (2, 1000, 16), (3, 200, 16),
                                       (2, 0, 16), (3, 5, 4)])
def test_info_counts(m, n, block):
    beta = 2 if m <= 3 else 4
    mp = sx.simplex_map_create(m, n, 2, beta, block)
    info = sx.simplex_map_info(mp)
    nb = (n + block) // block
    N = 1 << max(0, (nb - 1).bit_length())
    assert info["N"] == N
    assert info["cells"] == math.comb(n + m, m)
    assert info["useful_blocks"] == math.comb(n // block + m, m)
    assert info["bb_blocks"] == N ** m
    logN = N.bit_length() - 1
    # Eq. generic-m with r = 1/2 (reduces to Eq. m2 / Eq. m3 for beta = 2)
    assert info["h_set_blocks"] == (N ** m - beta ** logN) // (2 ** m - beta)
    if m == 2:
        assert info["h_set_blocks"] == N * (N - 1) // 2          # Eq. m2 (Lemma 1)
        band = info["band"]
        Ne = -(-nb // band) * band
        assert info["Ne"] == Ne
        assert info["h_blocks"] == Ne * (Ne + 1) // 2            # trapezoid bands
        single = sx.simplex_map_info(sx.simplex_map_create(m, n, 2, beta, block, band=-1))
        assert single["band"] == 0 and single["h_blocks"] == N * (N - 1) // 2 + N
    if m == 3:
        assert info["h_set_blocks"] == (N ** 3 - N) // 6          # Eq. m3 (Lemma 3)


def test_h3_packing_waste_tends_to_one_eighth():
    # Sec. 4.3: the single-grid packing adds 1/8 of V(Delta) in the limit
    mp = sx.simplex_map_create(3, 32767, 2, 2, 4)   # N = 8192
    info = sx.simplex_map_info(mp)
    N = info["N"]
    plane = (N // 2) * (N - 1) + N
    packed = info["h_blocks"] - plane
    tet = (N ** 3 - N) // 6
    assert abs(packed / tet - 1 - 0.125) < 0.002


def test_m4_overhang_fraction_matches_lemma_5_scaling():
    # beta = m = 4 cubes: V = (N^4 - N^2)/12 against V(Delta) ~ N^4/24
    mp = sx.simplex_map_create(4, 2 ** 12 - 1, 2, 4, 4)
    info = sx.simplex_map_info(mp)
    N = info["N"]
    assert info["h_set_blocks"] == (N ** 4 - N ** 2) // 12


# ------------------------------------------------------------------ errors
@pytest.mark.parametrize("args,code", [((1, 10, 2, 2, 16), sx.SIMPLEX_EINVAL), ((5, 10, 2, 2, 16), sx.SIMPLEX_EINVAL),
                                       ((2, -1, 2, 2, 16), sx.SIMPLEX_EINVAL), ((2, 10, 3, 2, 16), sx.SIMPLEX_EUNSUPPORTED),
                                       ((2, 10, 2, 3, 16), sx.SIMPLEX_EUNSUPPORTED), ((4, 10, 2, 2, 4), sx.SIMPLEX_EUNSUPPORTED),
                                       ((2, 10, 2, 2, 12), sx.SIMPLEX_EINVAL), ((2, 10, 2, 2, 2), sx.SIMPLEX_EINVAL),
                                       ((2, 10, 2, 2, 512), sx.SIMPLEX_EINVAL), ((2, 2 ** 40, 2, 2, 16), sx.SIMPLEX_EINVAL)])
def test_create_rejects_bad_arguments(args, code):
    with pytest.raises(sx.SimplexError) as ei:
        sx.simplex_map_create(*args)
    assert ei.value.code == code
    assert sx.simplex_last_error()


def test_padded_side_must_hold_the_domain():
    with pytest.raises(sx.SimplexError) as ei:
        sx.simplex_map_create(2, 100, 2, 2, 16, side=100)
    assert ei.value.code == sx.SIMPLEX_EINVAL
    mp = sx.simplex_map_create(2, 100, 2, 2, 16, side=112)
    assert mp.side == 112


def test_map_block_rejects_out_of_range():
    mp = sx.simplex_map_create(2, 63, 2, 2, 16)
    with pytest.raises(sx.SimplexError):
        sx.simplex_map_block(mp, sx.SIMPLEX_MODE_H, mp.info.h_blocks)
    with pytest.raises(sx.SimplexError):
        sx.simplex_map_block(mp, 7, 0)


# ------------------------------------------------------------------ Eq. map2d as printed
@pytest.mark.parametrize("N", [2, 4, 8, 16, 32, 64, 128, 256])
def test_h2_grid_is_eq_map2d(N):
    rho = 4
    mp = sx.simplex_map_create(2, N * rho - 1, 2, 2, rho, band=-1)
    assert mp.info.N == N
    seen = set()
    for v in range((N // 2) * (N - 1)):
        wx, wy = v % (N // 2), v // (N // 2)
        b = 1 << (wy + 1).bit_length() - 1
        q = wx // b
        hx, hy = wx + q * b, wy + 2 * q * b + 1          # Thm. 1
        (X1, X2), valid = sx.simplex_map_block(mp, sx.SIMPLEX_MODE_H, v)
        assert valid
        assert (X2, N - 1 - X1) == (hx, hy)
        assert hx < hy <= N - 1
        seen.add((hx, hy))
    # a bijection onto the blocks strictly below the diagonal (Lemma 1, Lemma 2)
    assert len(seen) == N * (N - 1) // 2


# ------------------------------------------------------------------ exhaustive coverage
def _covered(mp, mode):
    nblocks = mp.info.h_blocks if mode == sx.SIMPLEX_MODE_H else mp.info.bb_blocks
    cnt = collections.Counter()
    for v in range(nblocks):
        X, valid = sx.simplex_map_block(mp, mode, v)
        if valid:
            cnt[X] += 1
    return cnt


COVER_CASES = [(2, n, 4) for n in (0, 1, 3, 4, 7, 8, 15, 16, 17, 31, 63, 100, 127, 255, 1000, 1023)] + \
    [(3, n, 4, 2) for n in (0, 3, 4, 7, 8, 15, 31, 63, 100, 127, 255)] + \
    [(3, n, 4, 3) for n in (0, 7, 15, 31, 63, 100, 127)] + \
    [(4, n, 4, 4) for n in (0, 3, 7, 15, 31, 50, 63)]


@pytest.mark.parametrize("band", [-1, 1, 2, 4, 8, 16, 64])
@pytest.mark.parametrize("n,rho", [(0, 4), (3, 4), (4, 4), (31, 4), (63, 4), (100, 4), (101, 8), (255, 4),
                                   (1000, 16), (1023, 4), (77, 4)])
def test_h2_forms_cover_each_simplex_block_exactly_once(band, n, rho):
    mp = sx.simplex_map_create(2, n, 2, 2, rho, band=band)
    got = _covered(mp, sx.SIMPLEX_MODE_H)
    ind = oracle.block_indicator(2, n, rho)
    want = {tuple(int(i) for i in x) for x in np.argwhere(ind)}
    assert set(got) == want
    assert all(c == 1 for c in got.values())


def test_h2_trapezoid_bands_walk_rows_in_order():
    # consecutive blocks of a band's rectangle are consecutive tiles of a row
    mp = sx.simplex_map_create(2, 64 * 16 - 1, 2, 2, 16, band=8)
    Ne = mp.info.Ne
    first = [sx.simplex_map_block(mp, sx.SIMPLEX_MODE_H, v)[0] for v in range(Ne - 8)]
    assert first == [(0, j) for j in range(Ne - 8)]


def test_band_rejected_for_m3_and_bad_values():
    with pytest.raises(sx.SimplexError):
        sx.simplex_map_create(3, 63, 2, 2, 4, band=8)
    with pytest.raises(sx.SimplexError):
        sx.simplex_map_create(2, 63, 2, 2, 4, band=6)
    prm = sx.SimplexMapParams(2, 2, 2, 4, 63, 0, 0, 7)
    h = sx._vp()
    assert sx._lib.simplex_map_create_ex(sx.ctypes.byref(prm), sx.ctypes.byref(h)) == sx.SIMPLEX_EINVAL


@pytest.mark.parametrize("case", COVER_CASES)
def test_h_covers_each_simplex_block_exactly_once(case):
    m, n, rho = case[:3]
    beta = case[3] if len(case) > 3 else 2
    mp = sx.simplex_map_create(m, n, 2, beta, rho)
    got = _covered(mp, sx.SIMPLEX_MODE_H)
    ind = oracle.block_indicator(m, n, rho)
    want = {tuple(int(i) for i in x) for x in np.argwhere(ind)}
    assert set(got) == want
    assert all(c == 1 for c in got.values())


@pytest.mark.parametrize("case", [(2, 63, 4), (2, 100, 8), (3, 63, 4), (3, 50, 8), (4, 31, 4)])
def test_bb_covers_each_simplex_block_exactly_once(case):
    m, n, rho = case
    mp = sx.simplex_map_create(m, n, 2, 2 if m <= 3 else 4, rho)
    got = _covered(mp, sx.SIMPLEX_MODE_BB)
    ind = oracle.block_indicator(m, n, rho)
    want = {tuple(int(i) for i in x) for x in np.argwhere(ind)}
    assert set(got) == want and all(c == 1 for c in got.values())


@pytest.mark.parametrize("N", [4, 8, 16, 32, 64])
def test_h3_hinge_valid_blocks_equal_eq_m3(N):
    # blocks mapped by the cube + layer regions (before the diagonal plane):
    # exactly the (N^3 - N)/6 blocks of Delta_{N-1} below the plane (Lemma 3)
    rho = 4
    mp = sx.simplex_map_create(3, N * rho - 1, 2, 2, rho)
    plane = (N // 2) * (N - 1) + N
    main = mp.info.h_blocks - plane
    valid = sum(1 for v in range(main) if sx.simplex_map_block(mp, sx.SIMPLEX_MODE_H, v)[1])
    assert valid == (N ** 3 - N) // 6


def test_launch_form_choice():
    assert sx.simplex_map_info(sx.simplex_map_create(3, 1023, 2, 2, 32))["launch"] == 1
    assert sx.simplex_map_info(sx.simplex_map_create(3, 1023, 2, 2, 32, launch=2))["launch"] == 2
    assert sx.simplex_map_info(sx.simplex_map_create(3, 1023, 2, 2, 32, launch=1))["launch"] == 1
    assert sx.simplex_map_info(sx.simplex_map_create(3, 1023, 2, 2, 16))["launch"] == 1
    assert sx.simplex_map_info(sx.simplex_map_create(2, 1023, 2, 2, 128))["launch"] == 1
    with pytest.raises(sx.SimplexError) as ei:
        sx.simplex_map_create(2, 1023, 2, 2, 128, launch=2)
    assert ei.value.code == sx.SIMPLEX_EUNSUPPORTED
    assert sx.simplex_map_info(sx.simplex_map_create(3, 1023, 2, 2, 32, launch=3))["launch"] == 3
    assert sx.simplex_map_info(sx.simplex_map_create(3, 200, 2, 2, 16, side=208, launch=3))["launch"] == 3
    with pytest.raises(sx.SimplexError) as ei:
        sx.simplex_map_create(2, 1023, 2, 2, 128, launch=3)
    assert ei.value.code == sx.SIMPLEX_EUNSUPPORTED
    with pytest.raises(sx.SimplexError) as ei:
        sx.simplex_map_unit(sx.simplex_map_create(3, 63, 2, 2, 32), sx.SIMPLEX_MODE_H, 0)
    assert ei.value.code == sx.SIMPLEX_EINVAL


# ---------------------------------------------------------------- plane-stream work units (launch 3)
def _plane_units(mp, mode):
    info = mp.info
    total = info.plane_units if mode == sx.SIMPLEX_MODE_H else info.plane_units_bb
    out = []
    for w in range(total):
        u, ok = sx.simplex_map_unit(mp, mode, w)
        out.append((u, ok))
    with pytest.raises(sx.SimplexError):
        sx.simplex_map_unit(mp, mode, total)
    return out


@pytest.mark.parametrize("n", [0, 1, 31, 32, 127, 128, 200, 255, 300, 527, 1023])
def test_plane_units_cover_each_brick_plane_exactly_once(n):
    """Every plane x1 of every 32 x 128 brick that holds a domain cell on that
    plane (32 Y + 128 X <= n - x1) is written by exactly one unit of a step in
    mode H, and by exactly one valid unit in mode BB; mode BB_THREAD runs every
    brick of the square on every plane once.  Units are numbered slab by slab
    and slabs shrink towards the apex."""
    mp = sx.simplex_map_create(3, n, 2, 2, 32, side=((n + 16) // 16) * 16, launch=3)
    ty, tx = 32, 128
    nY, nX = (n + ty) // ty, (n + tx) // tx
    want = np.zeros((n + 1, nY, nX), dtype=np.int64)
    for x1 in range(n + 1):
        for Y in range(nY):
            for X in range(nX):
                want[x1, Y, X] = 1 if ty * Y + tx * X <= n - x1 else 0
    for mode in (sx.SIMPLEX_MODE_H, sx.SIMPLEX_MODE_BB, sx.SIMPLEX_MODE_BB_THREAD):
        got = np.zeros_like(want)
        last_b = -1
        for (y0, x0, b, e), ok in _plane_units(mp, mode):
            assert y0 % ty == 0 and x0 % tx == 0 and 0 <= b
            assert b >= last_b  # slab by slab
            last_b = b
            if mode == sx.SIMPLEX_MODE_H:
                assert ok
            if not ok:
                assert y0 + x0 > n - b
                continue
            assert b <= e <= n
            assert e - b + 1 <= 64
            got[b:e + 1, y0 // ty, x0 // tx] += 1
        if mode == sx.SIMPLEX_MODE_BB_THREAD:
            np.testing.assert_array_equal(got, np.ones_like(want))
        else:
            np.testing.assert_array_equal(got, want)
    if n == 1023:
        # slab lengths: 2^floor(log2((n + 1 - b) / 64)) clamped to [4, 64]
        starts = sorted({u[2] for u, _ in _plane_units(mp, sx.SIMPLEX_MODE_H)})
        lens = np.diff(starts + [n + 1])
        assert lens[0] == 16 and lens[-1] == 4 and all(np.diff(lens) <= 0)
        for b, ln in zip(starts, lens[:-1]):
            q = (n + 1 - b) // 64
            assert ln == min(64, max(4, 1 << (q.bit_length() - 1) if q else 4))


# ---------------------------------------------------------------- fully efficient H3 (layout 1)
@pytest.mark.parametrize("n,rho", [(0, 4), (3, 4), (4, 4), (7, 4), (15, 4), (31, 4), (63, 4), (100, 4),
                                   (127, 4), (255, 4), (200, 8)])
def test_h3_levels_cover_each_simplex_block_exactly_once(n, rho):
    mp = sx.simplex_map_create(3, n, 2, 2, rho, layout=1)
    assert mp.info.layout == 1
    got = _covered(mp, sx.SIMPLEX_MODE_H)
    ind = oracle.block_indicator(3, n, rho)
    want = {tuple(int(i) for i in x) for x in np.argwhere(ind)}
    assert set(got) == want
    assert all(c == 1 for c in got.values())


@pytest.mark.parametrize("N", [1, 2, 4, 8, 16, 32, 64, 1024])
def test_h3_levels_launch_exactly_the_block_simplex(N):
    # no packing waste: (N^3 - N)/6 blocks below the plane (Eq. m3) plus the
    # plane's H2 cover; every one of them maps to a block of Delta_{N-1}
    rho = 4
    mp = sx.simplex_map_create(3, N * rho - 1, 2, 2, rho, layout=1)
    plane = (N // 2) * (N - 1) + N
    assert mp.info.h_blocks == (N ** 3 - N) // 6 + plane
    if N <= 64:
        main = mp.info.h_blocks - plane
        assert all(sx.simplex_map_block(mp, sx.SIMPLEX_MODE_H, v)[1] for v in range(main))


def test_layout_rejected_outside_m3_beta2():
    with pytest.raises(sx.SimplexError):
        sx.simplex_map_create(2, 63, 2, 2, 4, layout=1)
    with pytest.raises(sx.SimplexError):
        sx.simplex_map_create(3, 63, 2, 3, 4, layout=1)
    with pytest.raises(sx.SimplexError):
        sx.simplex_map_create(3, 63, 2, 2, 4, layout=2)


# ---------------------------------------------------------------- Thm. 3 / Lemma 5 (host analysis)
def test_extra_volume_limits_match_lemma_5():
    from paper_2208_11617_gb300 import autotune
    # the paper's values for r = 1/2, beta = 2: 5/7 (m = 4), 3x (m = 5), 39x (m = 7)
    assert autotune.extra_volume_limit(4, 2, 2) == pytest.approx(5 / 7)
    assert autotune.extra_volume_limit(5, 2, 2) == pytest.approx(3.0)
    assert autotune.extra_volume_limit(7, 2, 2) == pytest.approx(39.0)
    # m = 2, 3: the efficient cases (alpha -> 0)
    assert autotune.extra_volume_limit(2, 2, 2) == pytest.approx(0.0)
    assert autotune.extra_volume_limit(3, 2, 2) == pytest.approx(0.0)


def test_generic_m_volume_reduces_to_eq_m2_m3():
    from paper_2208_11617_gb300 import autotune
    for n in (2, 4, 64, 1024):
        assert autotune.set_volume(2, n, 2, 2) == pytest.approx((n * n - n) / 2)      # Eq. m2
        assert autotune.set_volume(3, n, 2, 2) == pytest.approx((n ** 3 - n) / 6)     # Eq. m3
        # the maps' block counts agree: H2 grid N/2 x (N-1) and H3 (N^3 - N)/6 cells of S
    mp = sx.simplex_map_create(4, 2 ** 10 - 1, 2, 4, 4)
    N = mp.info.N
    # beta = m = 4: (N^4 - 4^log2 N) / (16 - 4) blocks in the cube set (Eq. generic-m)
    assert mp.info.h_set_blocks == (N ** 4 - 4 ** int(math.log2(N))) // 12


def test_search_r_beta_orders_by_volume_gap():
    from paper_2208_11617_gb300 import autotune
    c = autotune.search_r_beta(4, 1024, k_max=4)
    gaps = [abs(x["volume"] - autotune.simplex_volume(4, 1024)) for x in c]
    assert gaps == sorted(gaps)
    # the volume optimum makes k^4 - beta close to 4! = 24 (k = 3, beta near 57
    # in the limit; the finite-n term beta^(log_k n) moves it at n = 1024)
    best = c[0]
    assert best["k"] == 3 and abs(best["extra"]) < 0.01
    # under the paper's stated bound 1/r > beta no set even reaches the volume
    # of the 4-simplex: k = 2 leaves no beta >= 2, and k >= 3 with beta < k
    # has k^4 - beta >= 79 > 24
    assert not any(x["paper_bound"] and x["covers_volume"] for x in c)


@pytest.mark.parametrize("m,n,block", [(2, 0, 32), (2, 1, 32), (2, 100, 32), (2, 1023, 128), (2, 32767, 128),
                                       (3, 0, 16), (3, 5, 16), (3, 200, 16), (3, 1023, 32)])
def test_host_copy_covers_the_domain_and_less_than_the_array(m, n, block):
    # simplex_ca_run_host moves every domain row prefix: at least the domain's
    # C(n + m, m) cells, at most the (n + 1)^m box; for the large cases close
    # to the domain (a few percent of staircase for m = 2, under 30 % for m = 3)
    mp = sx.simplex_map_create(m, n, 2, 2, block)
    info = sx.simplex_map_info(mp)
    cells = math.comb(n + m, m)
    assert cells <= info["host_copy_bytes"] <= (n + 1) ** m
    if n >= 1023:
        assert info["host_copy_bytes"] <= cells * (1.05 if m == 2 else 1.30)


@pytest.mark.parametrize("case", [(2, 63, 4), (3, 50, 8), (4, 31, 4)])
def test_bb_thread_mode_decodes_like_bb(case):
    # the per-thread-filter bounding box enumerates the same N^m lattice
    m, n, rho = case
    mp = sx.simplex_map_create(m, n, 2, 2 if m <= 3 else 4, rho)
    for v in range(0, mp.info.bb_blocks, 7):
        assert sx.simplex_map_block(mp, sx.SIMPLEX_MODE_BB_THREAD, v) == sx.simplex_map_block(mp, sx.SIMPLEX_MODE_BB, v)


_NULL_PROBE = r'''
import json, sys
sys.path.insert(0, sys.argv[1])
from paper_2208_11617_gb300 import simplex as sx
L, N = sx._lib, None
calls = {
    "simplex_map_info": (N, N), "simplex_map_block": (N, 0, 0, N, N), "simplex_map_unit": (N, 0, 0, N, N),
    "simplex_write": (N, N, 0, 0, N),
    "simplex_accum": (N, N, 0, 0, N), "simplex_ca_init": (N, N, 0, 0, N, N),
    "simplex_ca_step": (N, N, N, 0, 0, N, 0, N), "simplex_ca_run": (N, N, N, 1, 0, 0, N, 1, 0, N),
    "simplex_ca_run_host": (N, N, N, N, N, 1, 0, 0, N, N, 1, 0, N), "simplex_visit_count": (N, N, 0, 0, N),
    "simplex_map_test": (N, N, 0, N), "simplex_edm": (N, N, 3, N, 0, N), "simplex_ca_digest": (N, N, N, N, N),
    "simplex_batch_info": (N, N), "simplex_batch_bind": (N, N, 0, N), "simplex_batch_init": (N, N),
    "simplex_batch_run": (N, 1, N, 1, N), "simplex_batch_grid": (N, 0, N, N),
    "simplex_batch_run_static": (N, N, 0, 0, 1, N, N), "simplex_server_run": (N, N, N, 0, 0, N),
    "simplex_server_begin": (N, N), "simplex_server_submit": (N, N, N), "simplex_server_poll": (N, N),
    "simplex_server_wait": (N, -1), "simplex_server_result": (N, 0, N, N), "simplex_server_stats": (N, N),
    "simplex_server_arena_bytes": (N, N), "simplex_server_create": (N, N, 0, N), "simplex_map_create_ex": (N, N),
    "simplex_map_create": (2, 10, 2, 2, 16, N), "simplex_batch_create": (N, 0, N),
    "simplex_map_destroy": (N,), "simplex_batch_destroy": (N,), "simplex_server_destroy": (N,),
}
print(json.dumps({name: getattr(L, name)(*args) for name, args in calls.items()}))
'''


def test_null_handles_and_outputs_are_rejected():
    """Every entry point given a NULL handle (or NULL output) returns
    SIMPLEX_EINVAL before touching the GPU; destroying NULL is a no-op.  Run in
    a child process so that a crash would fail this test, not the suite."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, "-c", _NULL_PROBE, ROOT], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    got = json.loads(r.stdout.strip().splitlines()[-1])
    assert set(got) >= set(sx.EXPORTED) - {"simplex_device_status", "simplex_last_error", "simplex_version",
                                             "simplex_selftest_wait_timeout", "simplex_map_create_padded"}
    for name, rc in got.items():
        want = sx.SIMPLEX_OK if name.endswith("_destroy") else sx.SIMPLEX_EINVAL
        assert rc == want, (name, rc)



# ---------------------------------------------------------------- r = 1/3, beta = 3 (m = 2)
def _n3(n, rho):
    nb, N3 = (n + rho) // rho, 1
    while N3 < nb:
        N3 *= 3
    return N3


@pytest.mark.parametrize("n,rho", [(0, 4), (3, 4), (11, 4), (35, 4), (100, 4), (107, 4), (323, 4), (400, 8),
                                   (1295, 16)])
def test_r_third_map_covers_each_block_exactly_once(n, rho):
    """The m = 2 map with r = 1/3, beta = 3 (three squares and three triangles
    per split) sends its N3 (N3 + 1) / 2 CUDA blocks one-to-one onto the block
    triangle X1 + X2 <= N3 - 1 of the power-of-three lattice, the diagonal
    blocks last; a block holds cells iff rho (X1 + X2) <= n."""
    mp = sx.simplex_map_create(2, n, 3, 3, rho)
    info = mp.info
    N3 = _n3(n, rho)
    assert info.r_inv == 3 and info.h_blocks == N3 * (N3 + 1) // 2
    assert info.h_set_blocks == (N3 * N3 - N3) // 2
    seen = collections.Counter()
    valid = 0
    for v in range(info.h_blocks):
        X, ok = sx.simplex_map_block(mp, sx.SIMPLEX_MODE_H, v)
        assert X[0] >= 0 and X[1] >= 0 and X[0] + X[1] <= N3 - 1
        assert ok == (rho * (X[0] + X[1]) <= n)
        if v >= info.h_blocks - N3:
            assert X[0] + X[1] == N3 - 1  # the diagonal comes last
        seen[X] += 1
        valid += ok
    assert len(seen) == info.h_blocks and max(seen.values()) == 1
    assert valid == info.useful_blocks == math.comb(n // rho + 2, 2)


def test_r_third_map_first_level_layout():
    """N3 = 9: the first 27 blocks are the three 3 x 3 squares at (0, 0),
    (3, 0), (0, 3) -- the split of Sec. 6 with 1/r = 3 -- row by row."""
    mp = sx.simplex_map_create(2, 35, 3, 3, 4)  # 9 tiles per axis
    got = [sx.simplex_map_block(mp, sx.SIMPLEX_MODE_H, v)[0] for v in range(27)]
    want = [(o1 + i, o2 + j) for (o1, o2) in ((0, 0), (3, 0), (0, 3)) for i in range(3) for j in range(3)]
    assert got == want


def test_r_third_refusals_and_padding():
    with pytest.raises(sx.SimplexError) as ei:
        sx.simplex_map_create(3, 100, 3, 3, 16)
    assert ei.value.code == sx.SIMPLEX_EUNSUPPORTED
    with pytest.raises(sx.SimplexError) as ei:
        sx.simplex_map_create(2, 100, 3, 2, 16)
    assert ei.value.code == sx.SIMPLEX_EUNSUPPORTED
    with pytest.raises(sx.SimplexError):
        sx.simplex_map_create(2, 100, 3, 3, 16, band=4)
    # n + 1 = 81 tiles: r = 1/3 needs no padding, r = 1/2 pads to 128 tiles
    third, half = sx.simplex_map_create(2, 1295, 3, 3, 16), sx.simplex_map_create(2, 1295, 2, 2, 16, band=-1)
    assert third.info.h_blocks == third.info.useful_blocks == 3321
    assert half.info.h_blocks == 64 * 127 + 128
