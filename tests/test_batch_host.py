"""Host-side tests of the batched engine's planning (no GPU needed)."""
import math

import pytest

from paper_2208_11617_gb300 import inputs
from paper_2208_11617_gb300 import simplex as sx


def _inst(m, n, block, beta=2, band=0, rule=None, seed=0, thr=1 << 31):
    rule = rule or (inputs.B3S23 if m == 2 else inputs.B5S45)
    return dict(m=m, n=n, block=block, beta=beta, band=band, birth=rule[0], survive=rule[1], seed=seed,
                threshold=thr)


def test_batch_counts_and_layout():
    insts = [_inst(2, 100, 64), _inst(2, 1000, 128), _inst(3, 63, 16), _inst(3, 100, 16, beta=3), _inst(2, 0, 64)]
    b = sx.simplex_batch_create(insts)
    info = sx.simplex_batch_info(b)
    assert info["count"] == 5
    assert info["cells"] == sum(math.comb(d["n"] + d["m"], d["m"]) for d in insts)
    blocks = 0
    items = 0
    for d in insts:
        side = (d["n"] + 128) // 128 * 128
        mp = sx.simplex_map_create(d["m"], d["n"], 2, d["beta"], d["block"], side=side,
                                   band=(min(8, 1 << ((d["n"] + d["block"]) // d["block"]).bit_length() - 1)
                                         if d["m"] == 2 else None))
        blocks += mp.info.h_blocks
        # one work item per run of up to 8 consecutive blocks whose tiles hold
        # cells (blocks that exit in the kernel get no item)
        run = 0
        for v in range(mp.info.h_blocks):
            if sx.simplex_map_block(mp, sx.SIMPLEX_MODE_H, v)[1]:
                run += 1
                if run == 8:
                    items, run = items + 1, 0
            elif run:
                items, run = items + 1, 0
        items += 1 if run else 0
    assert info["blocks"] == blocks
    assert info["items"] == items
    sides = [(d["n"] + 128) // 128 * 128 for d in insts]
    grids = sum(2 * (-(-s ** d["m"] // 256) * 256) for s, d in zip(sides, insts))
    assert info["arena_bytes"] >= grids


@pytest.mark.parametrize("bad", [_inst(2, 100, 32), _inst(3, 63, 64), _inst(3, 63, 8), _inst(4, 31, 16), _inst(2, -1, 64),
                                 _inst(3, 63, 16, beta=4)])
def test_batch_rejects_unsupported_instances(bad):
    with pytest.raises(sx.SimplexError) as ei:
        sx.simplex_batch_create([_inst(2, 10, 64), bad])
    assert "instance 1" in str(ei.value)


def test_batch_rejects_an_empty_list():
    with pytest.raises(sx.SimplexError) as ei:
        sx.simplex_batch_create([])
    assert ei.value.code == sx.SIMPLEX_EINVAL


def test_batch_workload_generator():
    insts = inputs.batch_instances()
    assert len(insts) == 2304
    n2 = [d["n"] for d in insts if d["m"] == 2]
    n3 = [d["n"] for d in insts if d["m"] == 3]
    assert len(n2) == 2048 and min(n2) >= 64 and max(n2) < 2048
    assert len(n3) == 256 and min(n3) >= 32 and max(n3) < 256
    assert insts == inputs.batch_instances()          # seeded
    assert [d["seed"] for d in insts] == list(range(2304))


@pytest.mark.parametrize("field,bad", [("round_steps", 65), ("round_steps", -1), ("direct_jobs", -2),
                                       ("direct_jobs", 65), ("max_inflight", 0)])
def test_server_params_are_validated(field, bad):
    import ctypes
    good = dict(hbm_budget=1 << 30, max_jobs=16, max_steps=8, max_items=1 << 12, max_inflight=2, round_steps=0,
                direct_jobs=0)
    need = ctypes.c_uint64()
    p = sx.SimplexServerParams(**good)
    assert sx._lib.simplex_server_arena_bytes(ctypes.byref(p), ctypes.byref(need)) == 0 and need.value > 0
    for ok in ({"direct_jobs": -1}, {"direct_jobs": 64}, {"round_steps": 64}):
        p = sx.SimplexServerParams(**(good | ok))
        assert sx._lib.simplex_server_arena_bytes(ctypes.byref(p), ctypes.byref(need)) == 0
    p = sx.SimplexServerParams(**(good | {field: bad}))
    assert sx._lib.simplex_server_arena_bytes(ctypes.byref(p), ctypes.byref(need)) == sx.SIMPLEX_EINVAL


def test_serve_trace_generator():
    """The serving workload: Poisson arrivals at the stated rate (count within
    5 sigma, exponential gaps with the right mean), 80/20 m = 2/m = 3, n
    log-uniform in its range (the median near the geometric mean), steps
    uniform in 1..64, the rules of each m and Bernoulli(0.5) initial states."""
    import numpy as np
    rate, secs = 2000.0, 5.0
    jobs, t = inputs.serve_trace(rate=rate, seconds=secs)
    k = len(jobs)
    assert len(t) == k and abs(k - rate * secs) < 5 * math.sqrt(rate * secs)
    assert (np.diff(t) > 0).all() and t[0] >= 0 and t[-1] < secs
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / rate) < 5 / rate / math.sqrt(k)
    m3 = np.array([d["m"] == 3 for d in jobs])
    assert abs(m3.mean() - 0.2) < 5 * math.sqrt(0.2 * 0.8 / k)
    for m, (lo, hi), rule in ((2, (128, 8192), inputs.B3S23), (3, (32, 512), inputs.B5S45)):
        ns = np.array([d["n"] for d in jobs if d["m"] == m])
        assert ns.min() >= lo and ns.max() < hi
        assert abs(np.log(np.median(ns)) - 0.5 * (np.log(lo) + np.log(hi))) < 0.15
        assert all((d["birth"], d["survive"]) == rule for d in jobs if d["m"] == m)
    steps = np.array([d["steps"] for d in jobs])
    assert steps.min() == 1 and steps.max() == 64 and abs(steps.mean() - 32.5) < 1.0
    assert all(d["threshold"] == inputs.bernoulli_threshold(0.5) for d in jobs)
    assert [d["seed"] for d in jobs] == list(range(k))
    again, t2 = inputs.serve_trace(rate=rate, seconds=secs)
    assert again == jobs and (t2 == t).all()        # seeded


def test_static_run_checks_arguments_before_any_device_work():
    """simplex_batch_run_static rejects a NULL or unaligned grids pointer, a
    grids buffer smaller than the batch's grids, a parity other than 0 or 1
    and a step count outside 1 ... 4096 with SIMPLEX_EINVAL before it makes any
    CUDA call (the addresses below are never dereferenced)."""
    import ctypes
    b = sx.simplex_batch_create([_inst(2, 100, 64), _inst(3, 63, 16)])
    need = sx.simplex_batch_info(b)["grids_bytes"]
    fake = 1 << 40  # 256-byte aligned, never touched
    cases = [(None, need, 0, 3, "NULL"), (fake + 16, need, 0, 3, "256-byte aligned"),
             (fake, need - 1, 0, 3, "too small"), (fake, need, 2, 3, "parity"), (fake, need, 0, 0, "steps"),
             (fake, need, 0, 4097, "steps")]
    for ptr, nbytes, parity, steps, what in cases:
        rc = sx._lib.simplex_batch_run_static(b.handle, ctypes.c_void_p(ptr) if ptr else None, nbytes, parity,
                                              steps, None, None)
        assert rc == sx.SIMPLEX_EINVAL and what in sx.simplex_last_error(), (ptr, nbytes, parity, steps)


def test_plane_stream_instances_are_planned():
    """m = 3 instances with block 128 run as plane streams: the batch plans
    them (host only), counts their cells, and the allocation-free run refuses
    them before any device work."""
    import ctypes
    insts = [_inst(2, 100, 64), _inst(3, 200, 128), _inst(3, 0, 128), _inst(3, 63, 16)]
    b = sx.simplex_batch_create(insts)
    info = sx.simplex_batch_info(b)
    assert info["cells"] == sum(math.comb(d["n"] + d["m"], d["m"]) for d in insts)
    assert info["arena_bytes"] > info["grids_bytes"]
    fake = 1 << 40
    rc = sx._lib.simplex_batch_run_static(b.handle, ctypes.c_void_p(fake), info["grids_bytes"], 0, 3, None, None)
    assert rc == sx.SIMPLEX_EUNSUPPORTED and "plane-stream" in sx.simplex_last_error()
    with pytest.raises(sx.SimplexError):
        sx.simplex_batch_create([_inst(3, 70000, 128)])
