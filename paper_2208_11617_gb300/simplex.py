"""Python binding of libsimplex (include/simplex.h): argument marshalling only.

Every function has the name of the C entry point it calls and takes torch
tensors (or host numpy arrays where the C call takes host memory); the work
itself runs in the CUDA kernels of ``libsimplex.so``.  Importing this module
fails loudly when the library has not been built -- there is no fallback.

The stream of every call is torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsimplex.so")

SIMPLEX_OK = 0
SIMPLEX_EINVAL = 1
SIMPLEX_ENOMEM = 2
SIMPLEX_ECUDA = 3
SIMPLEX_ETIMEOUT = 4
SIMPLEX_EUNSUPPORTED = 5

SIMPLEX_MODE_H = 0
SIMPLEX_MODE_BB = 1
SIMPLEX_MODE_BB_THREAD = 2
SIMPLEX_LEVEL_BLOCK = 0
SIMPLEX_LEVEL_CELL = 1

EXPORTED = (
    "simplex_map_create", "simplex_map_create_padded", "simplex_map_create_ex", "simplex_map_destroy", "simplex_map_info",
    "simplex_map_block", "simplex_map_unit", "simplex_accum", "simplex_write", "simplex_ca_init", "simplex_ca_step", "simplex_ca_run",
    "simplex_ca_run_host", "simplex_visit_count", "simplex_device_status", "simplex_last_error",
    "simplex_version", "simplex_selftest_wait_timeout", "simplex_batch_create", "simplex_batch_destroy",
    "simplex_batch_info", "simplex_batch_bind", "simplex_batch_init", "simplex_batch_run", "simplex_batch_grid",
    "simplex_batch_run_static", "simplex_server_arena_bytes", "simplex_server_create", "simplex_server_destroy",
    "simplex_server_run", "simplex_server_begin", "simplex_server_submit", "simplex_server_poll",
    "simplex_server_wait", "simplex_server_result", "simplex_server_stats", "simplex_ca_digest",
    "simplex_map_test", "simplex_edm",
)

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built: run `python -m paper_2208_11617_gb300.build` "
                      "(the CUDA library is required; there is no CPU fallback)")

_lib = ctypes.CDLL(LIB_PATH)

_vp = ctypes.c_void_p
_i32, _i64, _u32, _u64 = ctypes.c_int, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64


class SimplexMapInfo(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("r_inv", ctypes.c_int32), ("beta", ctypes.c_int32),
                ("block", ctypes.c_int32), ("n", ctypes.c_int64), ("side", ctypes.c_int64),
                ("N", ctypes.c_int32), ("log2N", ctypes.c_int32), ("band", ctypes.c_int32),
                ("Ne", ctypes.c_int32), ("launch", ctypes.c_int32), ("layout", ctypes.c_int32),
                ("cells", ctypes.c_uint64),
                ("useful_blocks", ctypes.c_uint64), ("h_blocks", ctypes.c_uint64),
                ("bb_blocks", ctypes.c_uint64), ("h_set_blocks", ctypes.c_uint64),
                ("host_copy_bytes", ctypes.c_uint64), ("plane_units", ctypes.c_uint64),
                ("plane_units_bb", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class SimplexMapParams(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("r_inv", ctypes.c_int32), ("beta", ctypes.c_int32),
                ("block", ctypes.c_int32), ("n", ctypes.c_int64), ("side", ctypes.c_int64),
                ("band", ctypes.c_int32), ("launch", ctypes.c_int32), ("layout", ctypes.c_int32)]


class SimplexInstance(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("block", ctypes.c_int32), ("beta", ctypes.c_int32),
                ("band", ctypes.c_int32), ("n", ctypes.c_int64), ("birth", ctypes.c_uint32),
                ("survive", ctypes.c_uint32), ("seed", ctypes.c_uint32), ("threshold", ctypes.c_uint32)]


class SimplexBatchInfo(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int32), ("parity", ctypes.c_int32), ("items", ctypes.c_uint64),
                ("blocks", ctypes.c_uint64), ("cells", ctypes.c_uint64), ("arena_bytes", ctypes.c_uint64),
                ("grids_offset", ctypes.c_uint64), ("grids_bytes", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class SimplexServerParams(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_uint64), ("max_jobs", ctypes.c_int32), ("max_steps", ctypes.c_int32),
                ("max_items", ctypes.c_int32), ("max_inflight", ctypes.c_int32), ("round_steps", ctypes.c_int32),
                ("direct_jobs", ctypes.c_int32)]


class SimplexJob(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("steps", ctypes.c_int32), ("n", ctypes.c_int64),
                ("birth", ctypes.c_uint32), ("survive", ctypes.c_uint32), ("seed", ctypes.c_uint32),
                ("threshold", ctypes.c_uint32)]


class SimplexJobResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("steps", ctypes.c_int32), ("arrival_ms", ctypes.c_double),
                ("admit_ms", ctypes.c_double), ("done_ms", ctypes.c_double), ("digest", ctypes.c_uint64),
                ("live_final", ctypes.c_uint64), ("seen_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class SimplexServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("rounds", ctypes.c_uint64), ("cell_updates", ctypes.c_uint64), ("peak_pool_bytes", ctypes.c_uint64),
                ("wall_ms", ctypes.c_double), ("mean_active", ctypes.c_double), ("p50_ms", ctypes.c_double),
                ("p90_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("host_issue_ms", ctypes.c_double), ("gpu_round_ms", ctypes.c_double),
                ("launches", ctypes.c_uint64), ("host_p50_ms", ctypes.c_double), ("host_p99_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


def _sig(name, args):
    f = getattr(_lib, name)
    f.argtypes = args
    f.restype = _i32
    return f


_sig("simplex_map_create", [_i32, _i64, _i32, _i32, _i32, ctypes.POINTER(_vp)])
_sig("simplex_map_create_padded", [_i32, _i64, _i32, _i32, _i32, _i64, ctypes.POINTER(_vp)])
_sig("simplex_map_create_ex", [ctypes.POINTER(SimplexMapParams), ctypes.POINTER(_vp)])
_sig("simplex_map_destroy", [_vp])
_sig("simplex_map_info", [_vp, ctypes.POINTER(SimplexMapInfo)])
_sig("simplex_map_block", [_vp, _i32, _u64, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(_i32)])
_sig("simplex_map_unit", [_vp, _i32, _u64, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(_i32)])
_sig("simplex_write", [_vp, _vp, _u32, _i32, _vp])
_sig("simplex_accum", [_vp, _vp, _u32, _i32, _vp])
_sig("simplex_ca_init", [_vp, _vp, _u32, _u32, _vp, _vp])
_sig("simplex_ca_step", [_vp, _vp, _vp, _u32, _u32, _vp, _i32, _vp])
_sig("simplex_ca_run", [_vp, _vp, _vp, _i32, _u32, _u32, _vp, _i32, _i32, _vp])
_sig("simplex_ca_run_host", [_vp, _vp, _vp, _vp, _vp, _i32, _u32, _u32, _vp, _vp, _i32, _i32, _vp])
_sig("simplex_visit_count", [_vp, _vp, _i32, _i32, _vp])
_sig("simplex_map_test", [_vp, _vp, _i32, _vp])
_sig("simplex_edm", [_vp, _vp, _i32, _vp, _i32, _vp])
_sig("simplex_device_status", [ctypes.POINTER(_u32)])
_sig("simplex_selftest_wait_timeout", [_u64, _vp])
_sig("simplex_batch_create", [ctypes.POINTER(SimplexInstance), _i32, ctypes.POINTER(_vp)])
_sig("simplex_batch_destroy", [_vp])
_sig("simplex_batch_info", [_vp, ctypes.POINTER(SimplexBatchInfo)])
_sig("simplex_batch_bind", [_vp, _vp, _u64, _vp])
_sig("simplex_batch_init", [_vp, _vp])
_sig("simplex_batch_run", [_vp, _i32, _vp, _i32, _vp])
_sig("simplex_batch_grid", [_vp, _i32, ctypes.POINTER(_vp), ctypes.POINTER(_i64)])
_sig("simplex_batch_run_static", [_vp, _vp, _u64, _i32, _i32, _vp, _vp])
_sig("simplex_server_arena_bytes", [ctypes.POINTER(SimplexServerParams), ctypes.POINTER(_u64)])
_sig("simplex_server_create", [ctypes.POINTER(SimplexServerParams), _vp, _u64, ctypes.POINTER(_vp)])
_sig("simplex_server_destroy", [_vp])
_sig("simplex_server_run", [_vp, ctypes.POINTER(SimplexJob), ctypes.POINTER(ctypes.c_double), _i32, _i32, _vp])
_sig("simplex_server_begin", [_vp, _vp])
_sig("simplex_server_submit", [_vp, ctypes.POINTER(SimplexJob), ctypes.POINTER(_i64)])
_sig("simplex_server_poll", [_vp, ctypes.POINTER(_i32)])
_sig("simplex_server_wait", [_vp, _i64])
_sig("simplex_server_result", [_vp, _i64, ctypes.POINTER(SimplexJobResult), _vp])
_sig("simplex_server_stats", [_vp, ctypes.POINTER(SimplexServerStats)])
_sig("simplex_ca_digest", [_vp, _vp, _vp, _vp, _vp])
_lib.simplex_last_error.argtypes = []
_lib.simplex_last_error.restype = ctypes.c_char_p
_lib.simplex_version.argtypes = []
_lib.simplex_version.restype = ctypes.c_char_p


class SimplexError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _lib.simplex_last_error().decode()
        super().__init__(f"{where} failed with status {code}: {msg}")
        self.code = code


def _check(rc: int, where: str):
    if rc != SIMPLEX_OK:
        raise SimplexError(rc, where)


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _dptr(t: torch.Tensor | None, dtype, name: str, numel: int | None = None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} needs at least {numel} elements, has {t.numel()}")
    return t.data_ptr()


@dataclass
class SimplexMap:
    """A planned map (owns the C handle)."""
    handle: int
    info: SimplexMapInfo

    @property
    def m(self) -> int:
        return self.info.m

    @property
    def n(self) -> int:
        return self.info.n

    @property
    def side(self) -> int:
        return self.info.side

    @property
    def numel(self) -> int:
        return self.info.side ** self.info.m

    @property
    def shape(self) -> tuple:
        return (self.info.side,) * self.info.m

    def close(self):
        if self.handle:
            _lib.simplex_map_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def simplex_map_create(m: int, n: int, r_inv: int = 2, beta: int | None = None, block: int = 16,
                       side: int | None = None, band: int | None = None, launch: int = 0,
                       layout: int = 0) -> SimplexMap:
    """Plan H for Delta_n^m (beta defaults to the paper's 2 for m <= 3, m for m = 4, and to 3 for the
    r = 1/3 map of m = 2, r_inv = 3).

    band (m = 2): None/0 automatic trapezoid bands, > 0 band height, -1 the
    single grid of Eq. map2d.  launch: 0 automatic, 1 grid, 2 x-stream
    (persistent) automaton step for m = 3, block 32, 3 plane stream (m = 3,
    persistent CTAs streaming bricks along x1).  layout (m = 3, beta = 2): 0 packed grid, 1 one block
    range per stack level."""
    if beta is None:
        beta = 3 if r_inv == 3 else (2 if m <= 3 else m)
    h = _vp()
    if band is not None or launch or layout:
        prm = SimplexMapParams(m, r_inv, beta, block, n, side or 0, band or 0, launch, layout)
        _check(_lib.simplex_map_create_ex(ctypes.byref(prm), ctypes.byref(h)), "simplex_map_create_ex")
    elif side is None:
        _check(_lib.simplex_map_create(m, n, r_inv, beta, block, ctypes.byref(h)), "simplex_map_create")
    else:
        _check(_lib.simplex_map_create_padded(m, n, r_inv, beta, block, side, ctypes.byref(h)),
               "simplex_map_create_padded")
    info = SimplexMapInfo()
    _check(_lib.simplex_map_info(h, ctypes.byref(info)), "simplex_map_info")
    return SimplexMap(h.value, info)


def simplex_map_info(mp: SimplexMap) -> dict:
    info = SimplexMapInfo()
    _check(_lib.simplex_map_info(mp.handle, ctypes.byref(info)), "simplex_map_info")
    return info.as_dict()


def simplex_map_block(mp: SimplexMap, mode: int, v: int):
    """Host evaluation of the map for CUDA block v: (tile coordinate tuple, valid)."""
    coord = (ctypes.c_int32 * 4)()
    valid = _i32()
    _check(_lib.simplex_map_block(mp.handle, mode, v, coord, ctypes.byref(valid)), "simplex_map_block")
    return tuple(coord[: mp.m]), bool(valid.value)


def simplex_map_unit(mp: SimplexMap, mode: int, w: int):
    """Host evaluation of plane-stream work unit w: ((y0, x0, first plane, last plane), valid)."""
    unit = (ctypes.c_int32 * 4)()
    valid = _i32()
    _check(_lib.simplex_map_unit(mp.handle, mode, w, unit, ctypes.byref(valid)), "simplex_map_unit")
    return tuple(unit), bool(valid.value)


def simplex_write(mp: SimplexMap, out: torch.Tensor, seed: int, mode: int = SIMPLEX_MODE_H):
    p = _dptr(out, torch.int32, "out", mp.numel) if out.dtype == torch.int32 else \
        _dptr(out, torch.uint32, "out", mp.numel)
    _check(_lib.simplex_write(mp.handle, p, seed & 0xFFFFFFFF, mode, _stream()), "simplex_write")


def simplex_accum(mp: SimplexMap, data: torch.Tensor, add: int = 1, mode: int = SIMPLEX_MODE_H):
    """ACCUM test: data[x] += add (mod 2^32) on every domain cell (int32 or uint32 tensor)."""
    p = _dptr(data, torch.int32, "data", mp.numel) if data.dtype == torch.int32 else \
        _dptr(data, torch.uint32, "data", mp.numel)
    _check(_lib.simplex_accum(mp.handle, p, add & 0xFFFFFFFF, mode, _stream()), "simplex_accum")


def simplex_ca_init(mp: SimplexMap, grid: torch.Tensor, seed: int, threshold: int,
                    live: torch.Tensor | None = None):
    _check(_lib.simplex_ca_init(mp.handle, _dptr(grid, torch.uint8, "grid", mp.numel), seed & 0xFFFFFFFF,
                                threshold & 0xFFFFFFFF, _dptr(live, torch.int64, "live", 1), _stream()),
           "simplex_ca_init")


def simplex_ca_step(mp: SimplexMap, src: torch.Tensor, dst: torch.Tensor, birth: int, survive: int,
                    live: torch.Tensor | None = None, mode: int = SIMPLEX_MODE_H):
    _check(_lib.simplex_ca_step(mp.handle, _dptr(src, torch.uint8, "in", mp.numel),
                                _dptr(dst, torch.uint8, "out", mp.numel), birth, survive,
                                _dptr(live, torch.int64, "live", 1), mode, _stream()), "simplex_ca_step")


def simplex_ca_run(mp: SimplexMap, a: torch.Tensor, b: torch.Tensor, steps: int, birth: int, survive: int,
                   live: torch.Tensor | None = None, use_graph: bool = True, mode: int = SIMPLEX_MODE_H):
    """steps a -> b -> a ...; returns the tensor holding the final state."""
    _check(_lib.simplex_ca_run(mp.handle, _dptr(a, torch.uint8, "a", mp.numel), _dptr(b, torch.uint8, "b", mp.numel),
                               steps, birth, survive, _dptr(live, torch.int64, "live", steps + 1),
                               1 if use_graph else 0, mode, _stream()), "simplex_ca_run")
    return a if steps % 2 == 0 else b


def simplex_ca_run_host(mp: SimplexMap, host_in: torch.Tensor, host_out: torch.Tensor, a: torch.Tensor,
                        b: torch.Tensor, steps: int, birth: int, survive: int,
                        dev_live: torch.Tensor | None = None, host_live: torch.Tensor | None = None,
                        use_graph: bool = True, mode: int = SIMPLEX_MODE_H):
    """End-to-end run from and to host (CPU, ideally pinned) tensors; synchronous."""
    for t, nm in ((host_in, "host_in"), (host_out, "host_out")):
        if t.is_cuda or t.dtype != torch.uint8 or not t.is_contiguous() or t.numel() < mp.numel:
            raise ValueError(f"{nm} must be a contiguous CPU uint8 tensor of {mp.numel} elements")
    if host_live is not None and (host_live.is_cuda or host_live.dtype != torch.int64 or host_live.numel() < steps + 1):
        raise ValueError("host_live must be a CPU int64 tensor of steps + 1 elements")
    _check(_lib.simplex_ca_run_host(mp.handle, host_in.data_ptr(), host_out.data_ptr(),
                                    _dptr(a, torch.uint8, "a", mp.numel), _dptr(b, torch.uint8, "b", mp.numel),
                                    steps, birth, survive, _dptr(dev_live, torch.int64, "dev_live", steps + 1),
                                    None if host_live is None else host_live.data_ptr(), 1 if use_graph else 0,
                                    mode, _stream()), "simplex_ca_run_host")


def simplex_visit_count(mp: SimplexMap, counts: torch.Tensor, level: int, mode: int = SIMPLEX_MODE_H):
    if level == SIMPLEX_LEVEL_BLOCK:
        nb = (mp.n + mp.info.block) // mp.info.block
        need = nb ** mp.m
    else:
        need = mp.numel
    _check(_lib.simplex_visit_count(mp.handle, _dptr(counts, torch.int32, "counts", need), level, mode,
                                    _stream()), "simplex_visit_count")


def simplex_map_test(mp: SimplexMap, cells: torch.Tensor | None = None, mode: int = SIMPLEX_MODE_H):
    """MAP test (the map alone); with `cells` (one int64), the simplex cells of
    every block are added to cells[0]."""
    _check(_lib.simplex_map_test(mp.handle, _dptr(cells, torch.int64, "cells", 1), mode, _stream()),
           "simplex_map_test")


def simplex_edm(mp: SimplexMap, points: torch.Tensor, out: torch.Tensor, mode: int = SIMPLEX_MODE_H):
    """EDM test: out[x1, x2] = |p[x1] - p[n - x2]| (float32) for x1 + x2 <= n;
    points is (n + 1) x dim float32."""
    if points.dim() != 2 or points.shape[0] != mp.n + 1:
        raise ValueError(f"points must be (n + 1) x dim = ({mp.n + 1}, dim), got {tuple(points.shape)}")
    _check(_lib.simplex_edm(mp.handle, _dptr(points, torch.float32, "points", points.numel()), int(points.shape[1]),
                            _dptr(out, torch.float32, "out", mp.numel), mode, _stream()), "simplex_edm")


def simplex_device_status() -> int:
    out = _u32()
    rc = _lib.simplex_device_status(ctypes.byref(out))
    if rc not in (SIMPLEX_OK, SIMPLEX_ETIMEOUT):
        _check(rc, "simplex_device_status")
    return int(out.value)


def simplex_selftest_wait_timeout(limit_ns: int):
    _check(_lib.simplex_selftest_wait_timeout(limit_ns, _stream()), "simplex_selftest_wait_timeout")


class SimplexBatch:
    """A planned batch (owns the C handle); `arena` keeps the bound device memory alive."""

    def __init__(self, handle: int, count: int):
        self.handle = handle
        self.count = count
        self.arena = None

    def close(self):
        if self.handle:
            _lib.simplex_batch_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def simplex_batch_create(instances) -> SimplexBatch:
    """instances: sequence of dicts/tuples with the SimplexInstance fields."""
    arr = (SimplexInstance * len(instances))()
    for k, inst in enumerate(instances):
        if isinstance(inst, dict):
            for f, _ in SimplexInstance._fields_:
                setattr(arr[k], f, inst.get(f, 0))
        else:
            arr[k] = SimplexInstance(*inst)
    h = _vp()
    _check(_lib.simplex_batch_create(arr, len(instances), ctypes.byref(h)), "simplex_batch_create")
    return SimplexBatch(h.value, len(instances))


def simplex_batch_info(b: SimplexBatch) -> dict:
    info = SimplexBatchInfo()
    _check(_lib.simplex_batch_info(b.handle, ctypes.byref(info)), "simplex_batch_info")
    return info.as_dict()


def simplex_batch_bind(b: SimplexBatch, arena: torch.Tensor | None = None) -> torch.Tensor:
    """Binds (allocating a uint8 arena tensor when none is given) and returns the arena."""
    need = simplex_batch_info(b)["arena_bytes"]
    if arena is None:
        arena = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    base = arena.data_ptr()
    off = (-base) % 256
    _check(_lib.simplex_batch_bind(b.handle, base + off, arena.numel() - off, _stream()), "simplex_batch_bind")
    b.arena = arena
    return arena


def simplex_batch_init(b: SimplexBatch):
    _check(_lib.simplex_batch_init(b.handle, _stream()), "simplex_batch_init")


def simplex_batch_run(b: SimplexBatch, steps: int, live: torch.Tensor | None = None, use_graph: bool = True):
    _check(_lib.simplex_batch_run(b.handle, steps, _dptr(live, torch.int64, "live", b.count * (steps + 1)),
                                  1 if use_graph else 0, _stream()), "simplex_batch_run")


def simplex_batch_grid(b: SimplexBatch, i: int, m: int) -> torch.Tensor:
    """Instance i's current grid as a (side,)*m uint8 view into the arena."""
    ptr, side = _vp(), _i64()
    _check(_lib.simplex_batch_grid(b.handle, i, ctypes.byref(ptr), ctypes.byref(side)), "simplex_batch_grid")
    off = ptr.value - b.arena.data_ptr()
    n = side.value ** m
    return b.arena[off: off + n].view((side.value,) * m)


def simplex_batch_run_static(b: SimplexBatch, grids: torch.Tensor, parity: int, steps: int,
                             live: torch.Tensor | None = None):
    """Allocation-free run: `grids` (uint8, 256-byte aligned) holds both grids of
    every instance; the library keeps its own bookkeeping in a fixed array."""
    _check(_lib.simplex_batch_run_static(b.handle, _dptr(grids, torch.uint8, "grids"), grids.numel(), parity, steps,
                                         _dptr(live, torch.int64, "live", b.count * (steps + 1)), _stream()),
           "simplex_batch_run_static")


def simplex_ca_digest(mp: SimplexMap, grid: torch.Tensor, digest: torch.Tensor, live: torch.Tensor | None = None):
    _check(_lib.simplex_ca_digest(mp.handle, _dptr(grid, torch.uint8, "grid", mp.numel),
                                  _dptr(digest, torch.int64, "digest", 1), _dptr(live, torch.int64, "live", 1),
                                  _stream()), "simplex_ca_digest")


class SimplexServer:
    """A serving engine over a torch-allocated arena (owns the C handle)."""

    def __init__(self, hbm_budget: int, max_jobs: int = 4096, max_steps: int = 64, max_items: int = 1 << 18,
                 max_inflight: int = 2, round_steps: int = 0, direct_jobs: int = 0):
        self.params = SimplexServerParams(hbm_budget, max_jobs, max_steps, max_items, max_inflight, round_steps,
                                          direct_jobs)
        need = _u64()
        _check(_lib.simplex_server_arena_bytes(ctypes.byref(self.params), ctypes.byref(need)),
               "simplex_server_arena_bytes")
        self.arena = torch.empty(need.value + 256, dtype=torch.uint8, device="cuda")
        off = (-self.arena.data_ptr()) % 256
        h = _vp()
        _check(_lib.simplex_server_create(ctypes.byref(self.params), self.arena.data_ptr() + off,
                                          self.arena.numel() - off, ctypes.byref(h)), "simplex_server_create")
        self.handle = h.value
        self.count = 0

    def run(self, jobs, arrival_s=None, realtime: bool = True):
        arr = (SimplexJob * len(jobs))()
        for k, d in enumerate(jobs):
            for f, _ in SimplexJob._fields_:
                setattr(arr[k], f, d[f])
        times = None
        if arrival_s is not None:
            times = (ctypes.c_double * len(jobs))(*[float(t) for t in arrival_s])
        _check(_lib.simplex_server_run(self.handle, arr, times, len(jobs), 1 if realtime else 0, _stream()),
               "simplex_server_run")
        self.count = len(jobs)

    def begin(self):
        """Start an online session on the current stream (the server must be idle)."""
        _check(_lib.simplex_server_begin(self.handle, _stream()), "simplex_server_begin")
        self.count = 0

    def submit(self, job: dict) -> int:
        """Queue one job now; returns its id."""
        j = SimplexJob()
        for f, _ in SimplexJob._fields_:
            setattr(j, f, job[f])
        jid = _i64()
        _check(_lib.simplex_server_submit(self.handle, ctypes.byref(j), ctypes.byref(jid)), "simplex_server_submit")
        self.count = jid.value + 1
        return jid.value

    def poll(self) -> int:
        """One non-blocking turn of the serving loop; returns the jobs it finished."""
        n = _i32()
        _check(_lib.simplex_server_poll(self.handle, ctypes.byref(n)), "simplex_server_poll")
        return n.value

    def wait(self, job: int = -1):
        """Serve until job `job` (every submitted job when -1) has finished."""
        _check(_lib.simplex_server_wait(self.handle, job), "simplex_server_wait")

    def result(self, job: int, steps: int | None = None):
        res = SimplexJobResult()
        live = (ctypes.c_uint64 * ((steps or 0) + 1))() if steps else None
        _check(_lib.simplex_server_result(self.handle, job, ctypes.byref(res), live), "simplex_server_result")
        out = res.as_dict()
        if live is not None:
            out["live"] = list(live)
        return out

    def stats(self) -> dict:
        st = SimplexServerStats()
        _check(_lib.simplex_server_stats(self.handle, ctypes.byref(st)), "simplex_server_stats")
        return st.as_dict()

    def close(self):
        if self.handle:
            _lib.simplex_server_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def simplex_last_error() -> str:
    return _lib.simplex_last_error().decode()


def simplex_version() -> str:
    return _lib.simplex_version().decode()


def library_path() -> str:
    return LIB_PATH
