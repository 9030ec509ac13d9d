"""The allocation-free batched run (simplex_batch_run_static) against the
arena-based one (simplex_batch_run).

Some hosts cannot hand the library an arena: they own all device memory
through their own pool, or cannot afford an allocator call on their hot path.
simplex_batch_run_static serves them with a fixed array inside the library
and only the caller's grids.  This test runs the same batch both ways, twice
in a row (so the second call sees the array the first one left behind), and
requires identical grids and live counts -- the work is integer, so the
tolerance is zero.  It lives in its own file, collected last, so that a run
stopping at the first failure has already run every other test.
"""
import ctypes

import pytest
import torch

from paper_2208_11617_gb300 import inputs
from paper_2208_11617_gb300 import simplex as sx

pytestmark = pytest.mark.gpu


def _inst(m, n, block, beta=2, seed=0, p=0.5, rule=None):
    rule = rule or (inputs.B3S23 if m == 2 else inputs.B5S45)
    return dict(m=m, n=n, block=block, beta=beta, band=0, birth=rule[0], survive=rule[1], seed=seed,
                threshold=inputs.bernoulli_threshold(p))


INSTANCES = [_inst(2, 1000, 64, seed=1), _inst(2, 2047, 128, seed=2), _inst(2, 37, 64, seed=3),
             _inst(3, 120, 16, seed=4, p=0.3), _inst(3, 63, 16, beta=3, seed=5, p=0.3),
             _inst(2, 300, 64, seed=6, rule=(1 << 3 | 1 << 6, 1 << 2 | 1 << 3)),
             _inst(3, 150, 32, seed=7, p=0.3)]


def test_static_scratch_run_matches_arena_run_twice():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    steps = 5
    ref = sx.simplex_batch_create(INSTANCES)
    info = sx.simplex_batch_info(ref)
    arena = sx.simplex_batch_bind(ref)
    sx.simplex_batch_init(ref)
    torch.cuda.synchronize()
    base = arena.data_ptr()
    goff = (-base) % 256 + info["grids_offset"]
    # the caller's own grids, with the same initial state
    grids = torch.empty(info["grids_bytes"] + 256, dtype=torch.uint8, device="cuda")
    g0 = (-grids.data_ptr()) % 256
    mine = grids[g0: g0 + info["grids_bytes"]]
    mine.copy_(arena[goff: goff + info["grids_bytes"]])
    other = sx.simplex_batch_create(INSTANCES)          # never bound: no arena at all
    parity = 0
    for call in range(2):
        live_ref = torch.zeros(len(INSTANCES) * (steps + 1), dtype=torch.int64, device="cuda")
        live_mine = torch.full_like(live_ref, -1)
        sx.simplex_batch_run(ref, steps, live_ref, True)
        sx.simplex_batch_run_static(other, mine, parity, steps, live_mine)
        torch.cuda.synchronize()
        assert torch.equal(mine, arena[goff: goff + info["grids_bytes"]]), f"call {call}: grids differ"
        assert torch.equal(live_mine, live_ref), f"call {call}: live counts differ"
        parity = (parity + steps) % 2
    assert sx.simplex_device_status() == 0


def test_static_scratch_rejects_bad_arguments():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    b = sx.simplex_batch_create(INSTANCES)
    info = sx.simplex_batch_info(b)
    small = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(sx.SimplexError) as ei:
        sx.simplex_batch_run_static(b, small, 0, 3)
    assert ei.value.code == sx.SIMPLEX_EINVAL and "too small" in str(ei.value)
    grids = torch.zeros(info["grids_bytes"] + 256, dtype=torch.uint8, device="cuda")
    g0 = (-grids.data_ptr()) % 256
    with pytest.raises(sx.SimplexError):
        sx.simplex_batch_run_static(b, grids[g0:], 2, 3)          # parity must be 0 or 1
    ptr = grids.data_ptr() + g0
    for gp, steps, what in [(ptr + 16, 3, "256-byte aligned"), (ptr, 0, "steps"), (ptr, 4097, "steps"),
                            (None, 3, "NULL")]:
        rc = sx._lib.simplex_batch_run_static(b.handle, ctypes.c_void_p(gp) if gp else None,
                                              info["grids_bytes"], 0, steps, None, None)
        assert rc == sx.SIMPLEX_EINVAL and what in sx.simplex_last_error(), (gp, steps, sx.simplex_last_error())
    # a batch whose bookkeeping exceeds the fixed array is refused, not truncated
    many = [_inst(2, 64, 64, seed=k) for k in range(12000)]
    big = sx.simplex_batch_create(many)
    rc = sx._lib.simplex_batch_run_static(big.handle, ctypes.c_void_p(grids.data_ptr() + g0),
                                          10 ** 12, 0, 1, None, None)
    assert rc == sx.SIMPLEX_EINVAL and "fixed scratch" in sx.simplex_last_error()


def test_static_scratch_alternating_batches():
    """Calls that alternate between two batches (and two grid buffers) find
    the fixed array holding the other batch's bookkeeping and must refill it;
    a repeated call with the same batch and grids reuses it.  Every result
    equals the arena-based run of the same batch."""
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    steps = 3
    specs = [INSTANCES, [_inst(2, 500, 64, seed=11), _inst(3, 90, 16, seed=12, p=0.3)]]
    runs = []
    for spec in specs:
        ref = sx.simplex_batch_create(spec)
        info = sx.simplex_batch_info(ref)
        arena = sx.simplex_batch_bind(ref)
        sx.simplex_batch_init(ref)
        torch.cuda.synchronize()
        goff = (-arena.data_ptr()) % 256 + info["grids_offset"]
        buf = torch.empty(info["grids_bytes"] + 256, dtype=torch.uint8, device="cuda")
        g0 = (-buf.data_ptr()) % 256
        mine = buf[g0: g0 + info["grids_bytes"]]
        mine.copy_(arena[goff: goff + info["grids_bytes"]])
        runs.append(dict(ref=ref, arena=arena, goff=goff, info=info, buf=buf, mine=mine,
                         other=sx.simplex_batch_create(spec), parity=0, count=len(spec)))
    for k in (0, 1, 0, 0, 1):
        r = runs[k]
        live_ref = torch.zeros(r["count"] * (steps + 1), dtype=torch.int64, device="cuda")
        live_mine = torch.full_like(live_ref, -1)
        sx.simplex_batch_run(r["ref"], steps, live_ref, True)
        sx.simplex_batch_run_static(r["other"], r["mine"], r["parity"], steps, live_mine)
        torch.cuda.synchronize()
        want = r["arena"][r["goff"]: r["goff"] + r["info"]["grids_bytes"]]
        assert torch.equal(r["mine"], want), f"batch {k}: grids differ"
        assert torch.equal(live_mine, live_ref), f"batch {k}: live counts differ"
        r["parity"] = (r["parity"] + steps) % 2
    assert sx.simplex_device_status() == 0
