"""CPU oracle for the simplex workloads of arXiv 2208.11617 (test infrastructure).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may load this module; the product package never
imports it.  The arithmetic lives in ``simplex_oracle.c`` (plain nested loops
over x_1 + ... + x_m <= n, Eq. 1); this file only compiles it with gcc and
marshals numpy arrays through ctypes.

Arrays are dense with side D = n + 1 and x_m fastest (row-major).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "simplex_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def compile_source(src: str, out: str) -> str:
    """gcc a C source file into the shared library `out` (OpenMP if gcc supports it)."""
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", src, "-o", out, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    return out


def build(force: bool = False) -> str:
    """Compile simplex_oracle.c into liboracle.so."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    compile_source(_SRC, tmp)
    os.replace(tmp, _LIB)
    return _LIB


def configure(lib):
    """Declares the C signatures of the oracle's entry points on a loaded library."""
    u8p = ctypes.POINTER(ctypes.c_uint8)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    i64, u32, i32, u64 = ctypes.c_int64, ctypes.c_uint32, ctypes.c_int, ctypes.c_uint64
    lib.oracle_splitmix32.argtypes = [u32]
    lib.oracle_splitmix32.restype = u32
    lib.oracle_num_threads.argtypes = []
    lib.oracle_num_threads.restype = i32
    lib.oracle_count_cells.argtypes = [i32, i64]
    lib.oracle_count_cells.restype = u64
    lib.oracle_write.argtypes = [i32, i64, u32, u32p]
    lib.oracle_write.restype = u64
    lib.oracle_accum.argtypes = [i32, i64, u32, u32p]
    lib.oracle_accum.restype = u64
    lib.oracle_ca_init.argtypes = [i32, i64, u32, u32, u8p]
    lib.oracle_ca_init.restype = u64
    lib.oracle_ca_step.argtypes = [i32, i64, u32, u32, u8p, u8p]
    lib.oracle_ca_step.restype = u64
    lib.oracle_ca_run.argtypes = [i32, i64, i32, u32, u32, u8p, u8p, u64p]
    lib.oracle_ca_run.restype = None
    lib.oracle_ca_cells.argtypes = [i32, i64, u32, u32, u8p, ctypes.POINTER(ctypes.c_int64), i64, u8p]
    lib.oracle_ca_cells.restype = None
    lib.oracle_block_indicator.argtypes = [i32, i64, i32, u32p]
    lib.oracle_block_indicator.restype = None
    lib.oracle_edm.argtypes = [i64, i32, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double)]
    lib.oracle_edm.restype = None
    lib.oracle_edm_cells.argtypes = [i64, i32, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int64), i64,
                                     ctypes.POINTER(ctypes.c_double)]
    lib.oracle_edm_cells.restype = None
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = configure(ctypes.CDLL(_LIB))
        return _lib


def _ptr(a: np.ndarray, ctype):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def splitmix32(z: int) -> int:
    return int(_load().oracle_splitmix32(z & 0xFFFFFFFF))


def count_cells(m: int, n: int) -> int:
    """|Delta_n^m| by enumeration (Eq. 1)."""
    return int(_load().oracle_count_cells(m, n))


def dense_shape(m: int, n: int) -> tuple:
    return (n + 1,) * m


def write(m: int, n: int, seed: int) -> np.ndarray:
    """Coordinate-write test: dense uint32 array, simplex cells hashed, rest 0."""
    out = np.zeros(dense_shape(m, n), dtype=np.uint32)
    c = _load().oracle_write(m, n, seed & 0xFFFFFFFF, _ptr(out, ctypes.c_uint32))
    assert c == count_cells(m, n) or m not in (2, 3, 4)
    return out


def accum(m: int, n: int, data: np.ndarray, add: int) -> np.ndarray:
    """ACCUM test (Table 1): a copy of the dense uint32 array `data` (side n + 1)
    with `add` added (mod 2^32) to every cell of the domain."""
    out = np.ascontiguousarray(data, dtype=np.uint32).copy()
    assert out.shape == dense_shape(m, n)
    c = _load().oracle_accum(m, n, add & 0xFFFFFFFF, _ptr(out, ctypes.c_uint32))
    assert c == count_cells(m, n) or m not in (2, 3, 4)
    return out


def ca_init(m: int, n: int, seed: int, threshold: int) -> np.ndarray:
    """Seeded Bernoulli state: simplex cells alive iff splitmix32(seed ^ lin) < threshold."""
    g = np.zeros(dense_shape(m, n), dtype=np.uint8)
    _load().oracle_ca_init(m, n, seed & 0xFFFFFFFF, threshold & 0xFFFFFFFF, _ptr(g, ctypes.c_uint8))
    return g


def ca_step(m: int, n: int, birth: int, survive: int, grid: np.ndarray):
    """One synchronous step; returns (new grid, live count)."""
    src = np.ascontiguousarray(grid, dtype=np.uint8)
    dst = np.zeros_like(src)
    live = _load().oracle_ca_step(m, n, birth, survive, _ptr(src, ctypes.c_uint8),
                                  _ptr(dst, ctypes.c_uint8))
    return dst, int(live)


def ca_run(m: int, n: int, steps: int, birth: int, survive: int, grid: np.ndarray):
    """`steps` synchronous steps; returns (final grid, live counts [steps + 1])."""
    a = np.array(grid, dtype=np.uint8, order="C", copy=True)
    b = np.zeros_like(a)
    live = np.zeros(steps + 1, dtype=np.uint64)
    _load().oracle_ca_run(m, n, steps, birth, survive, _ptr(a, ctypes.c_uint8),
                          _ptr(b, ctypes.c_uint8), _ptr(live, ctypes.c_uint64))
    return (a if steps % 2 == 0 else b), live


def ca_cells(m: int, n: int, birth: int, survive: int, grid: np.ndarray, coords: np.ndarray) -> np.ndarray:
    """Next state of the listed cells (coords: [k, m] int64), computed one by one."""
    src = np.ascontiguousarray(grid, dtype=np.uint8)
    assert src.shape == dense_shape(m, n)
    c = np.ascontiguousarray(coords, dtype=np.int64)
    assert c.ndim == 2 and c.shape[1] == m and (c.sum(1) <= n).all() and (c >= 0).all()
    out = np.zeros(len(c), dtype=np.uint8)
    _load().oracle_ca_cells(m, n, birth, survive, _ptr(src, ctypes.c_uint8),
                            c.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(c), _ptr(out, ctypes.c_uint8))
    return out


def block_indicator(m: int, n: int, rho: int) -> np.ndarray:
    """1 for every tile of side rho that holds a simplex cell, found cell by cell."""
    nb = (n + rho) // rho
    ind = np.zeros((nb,) * m, dtype=np.uint32)
    _load().oracle_block_indicator(m, n, rho, _ptr(ind, ctypes.c_uint32))
    return ind


def edm(n: int, points: np.ndarray) -> np.ndarray:
    """Distance matrix on the 2-simplex: dense (n+1) x (n+1) float64, entry
    (x1, x2) with x1 + x2 <= n = |p[x1] - p[n - x2]|, others 0."""
    pts = np.ascontiguousarray(points, dtype=np.float32)
    assert pts.ndim == 2 and pts.shape[0] == n + 1
    out = np.zeros((n + 1, n + 1), dtype=np.float64)
    _load().oracle_edm(n, pts.shape[1], _ptr(pts, ctypes.c_float), _ptr(out, ctypes.c_double))
    return out


def edm_cells(n: int, points: np.ndarray, coords: np.ndarray) -> np.ndarray:
    """Distances of the listed cells (coords: [k, 2] int64, x1 + x2 <= n), one by one."""
    pts = np.ascontiguousarray(points, dtype=np.float32)
    c = np.ascontiguousarray(coords, dtype=np.int64)
    assert c.ndim == 2 and c.shape[1] == 2 and (c >= 0).all() and (c.sum(1) <= n).all()
    out = np.zeros(len(c), dtype=np.float64)
    _load().oracle_edm_cells(n, pts.shape[1], _ptr(pts, ctypes.c_float), c.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                             len(c), _ptr(out, ctypes.c_double))
    return out
