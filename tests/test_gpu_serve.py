"""GPU tests of the continuous-batching server: every job's result is the same
in the mix as alone (and as the oracle's for small jobs), admission respects
the HBM budget, and resident jobs really share rounds."""
import numpy as np
import pytest
import torch

import oracle
from paper_2208_11617_gb300 import inputs
from paper_2208_11617_gb300 import simplex as sx

pytestmark = pytest.mark.gpu
SALT = 0x00D16E57


def _oracle_digest(grid, n):
    """Sum over live cells of splitmix32(SALT ^ row-major index on side n + 1)."""
    m = grid.ndim
    d = 0
    for x in np.argwhere(grid):
        lin = 0
        for xi in x:
            lin = lin * (n + 1) + int(xi)
        d += oracle.splitmix32(SALT ^ (lin & 0xFFFFFFFF))
    return d % (1 << 64)


def _alone(job):
    """The job on the single-instance path: final digest and live counts."""
    m, n = job["m"], job["n"]
    side = (n + 16) // 16 * 16
    mp = sx.simplex_map_create(m, n, 2, 2, 64 if m == 2 else 16, side=side)
    a = torch.zeros(mp.numel, dtype=torch.uint8, device="cuda")
    b = torch.zeros_like(a)
    sx.simplex_ca_init(mp, a, job["seed"], job["threshold"])
    live = torch.zeros(job["steps"] + 1, dtype=torch.int64, device="cuda")
    fin = sx.simplex_ca_run(mp, a, b, job["steps"], job["birth"], job["survive"], live, False)
    dig = torch.zeros(1, dtype=torch.int64, device="cuda")
    sx.simplex_ca_digest(mp, fin, dig)
    torch.cuda.synchronize()
    return int(dig.item()) & ((1 << 64) - 1), [int(v) for v in live.cpu().tolist()], fin, mp


def test_jobs_equal_alone_and_in_the_mix():
    jobs, t = inputs.serve_trace(rate=4000, seconds=0.08, seed=11, n2=(16, 1500), n3=(8, 200), max_steps=12)
    assert len(jobs) > 100
    srv = sx.SimplexServer(hbm_budget=2 << 30, max_jobs=512, max_steps=12)
    srv.run(jobs, t, realtime=True)
    st = srv.stats()
    assert st["completed"] == len(jobs) and st["rejected"] == 0
    assert st["mean_active"] > 1.0, st          # resident jobs shared rounds
    assert st["launches"] >= len(jobs) + st["rounds"]   # an init per job and at least one launch per round
    # the same jobs all at once: many resident per round, same results
    burst = sx.SimplexServer(hbm_budget=2 << 30, max_jobs=512, max_steps=12)
    burst.run(jobs, None, realtime=False)
    assert burst.stats()["mean_active"] > 20
    for i, job in enumerate(jobs):
        strip = {"arrival_ms": 0, "admit_ms": 0, "done_ms": 0, "seen_ms": 0}
        assert burst.result(i, job["steps"]) | strip == srv.result(i, job["steps"]) | strip, f"job {i}"
    rng = np.random.default_rng(0)
    sample = set(rng.choice(len(jobs), size=min(60, len(jobs)), replace=False).tolist())
    for i, job in enumerate(jobs):
        res = srv.result(i, job["steps"])
        assert res["status"] == 2
        assert res["done_ms"] >= res["arrival_ms"] - 1.0
        # the host finds a job complete only after its device event
        assert res["seen_ms"] >= res["done_ms"] - 1.0
        if i not in sample:
            continue
        dig, live, fin, mp = _alone(job)
        assert res["digest"] == dig, f"job {i}"
        assert res["live"] == live, f"job {i}"
        if job["n"] <= 512:
            ref, ref_live = oracle.ca_run(job["m"], job["n"], job["steps"], job["birth"], job["survive"],
                                          oracle.ca_init(job["m"], job["n"], job["seed"], job["threshold"]))
            assert [int(v) for v in ref_live] == res["live"]
            assert _oracle_digest(ref, job["n"]) == res["digest"]


def test_direct_and_batched_rounds_agree():
    """Rounds with few resident jobs launch each job's steps on its own grids
    (direct_jobs); the results equal those of batched passes only."""
    jobs, _ = inputs.serve_trace(rate=4000, seconds=0.05, seed=13, n2=(16, 1500), n3=(8, 200), max_steps=12)
    assert len(jobs) > 100
    res = []
    for dj in (-1, 64):
        srv = sx.SimplexServer(hbm_budget=2 << 30, max_jobs=512, max_steps=12, direct_jobs=dj)
        srv.run(jobs, None, realtime=False)   # all at once: batched rounds first, direct ones as jobs finish
        st = srv.stats()
        assert st["completed"] == len(jobs) and st["rejected"] == 0
        res.append([srv.result(i, job["steps"]) for i, job in enumerate(jobs)])
    strip = lambda r: {k: v for k, v in r.items() if not k.endswith("_ms")}
    for i, (a, b) in enumerate(zip(*res)):
        assert strip(a) == strip(b), f"job {i}"
    for i in (0, len(jobs) // 2, len(jobs) - 1):
        dig, live, _, _ = _alone(jobs[i])
        assert res[1][i]["digest"] == dig and res[1][i]["live"] == live


def test_direct_chunks_on_their_own_tiles_match_batched_passes():
    """Direct chunks run m = 3 jobs with n >= 352 on 32^3 tiles and m = 2 jobs
    with 1024 <= n < 2560 on 64 x 64 tiles, while batched passes keep 16^3 and
    128 x 128 tiles on the same grids.  All-batched, all-direct and a mix (a
    job takes batched passes while many are resident, direct chunks as the
    rest drain) give the same results, equal to the single-instance path's."""
    thr = inputs.bernoulli_threshold(0.5)
    rng = np.random.default_rng(21)
    jobs = []
    for k in range(36):
        if k % 3 == 0:
            m, n, rule = 3, int(rng.integers(352, 512)), inputs.B5S45
        else:
            m, rule = 2, inputs.B3S23
            n = int(rng.integers(1024, 2560)) if k % 3 == 1 else int(rng.integers(100, 4000))
        jobs.append(dict(m=m, n=n, steps=int(rng.integers(17, 41)), birth=rule[0], survive=rule[1], seed=k,
                         threshold=thr))
    res = []
    for dj in (-1, 64, 6):
        srv = sx.SimplexServer(hbm_budget=4 << 30, max_jobs=64, max_steps=40, direct_jobs=dj)
        srv.run(jobs, None, realtime=False)
        st = srv.stats()
        assert st["completed"] == len(jobs) and st["rejected"] == 0
        res.append([srv.result(i, job["steps"]) for i, job in enumerate(jobs)])
    strip = lambda r: {k: v for k, v in r.items() if not k.endswith("_ms")}
    for i in range(len(jobs)):
        assert strip(res[0][i]) == strip(res[1][i]) == strip(res[2][i]), f"job {i}"
    for i in (0, 1, 3, 4, len(jobs) - 3):
        dig, live, _, _ = _alone(jobs[i])
        assert res[1][i]["digest"] == dig and res[1][i]["live"] == live, f"job {i}"


def test_round_length_and_queue_depth_do_not_change_results():
    """Batched rounds of 1, 5 and 64 passes (the largest pass count the item
    tags hold), with 1 or 3 rounds queued ahead, give every job the same
    result: a job's steps are split over rounds differently, its grids and
    live counts are not."""
    jobs, _ = inputs.serve_trace(rate=4000, seconds=0.02, seed=19, n2=(16, 1500), n3=(8, 200), max_steps=70)
    assert len(jobs) > 40 and max(j["steps"] for j in jobs) > 64
    strip = lambda r: {k: v for k, v in r.items() if not k.endswith("_ms")}
    ref = None
    for k, depth in ((1, 1), (5, 3), (64, 1), (64, 3), (0, 2)):
        srv = sx.SimplexServer(hbm_budget=2 << 30, max_jobs=512, max_steps=70, round_steps=k, max_inflight=depth,
                               direct_jobs=-1)
        srv.run(jobs, None, realtime=False)
        st = srv.stats()
        assert st["completed"] == len(jobs) and st["rejected"] == 0
        res = [strip(srv.result(i, job["steps"])) for i, job in enumerate(jobs)]
        if ref is None:
            ref = res
        else:
            assert res == ref, (k, depth)
    for i in (0, len(jobs) - 1):
        dig, live, _, _ = _alone(jobs[i])
        assert ref[i]["digest"] == dig and ref[i]["live"] == live


def test_online_submit_poll_wait_matches_trace_run():
    """Jobs submitted one at a time (with polls between) give the results of
    the same jobs run as a trace."""
    jobs, _ = inputs.serve_trace(rate=4000, seconds=0.03, seed=17, n2=(16, 1500), n3=(8, 200), max_steps=12)
    assert len(jobs) > 50
    ref = sx.SimplexServer(hbm_budget=2 << 30, max_jobs=512, max_steps=12)
    ref.run(jobs, None, realtime=False)
    srv = sx.SimplexServer(hbm_budget=2 << 30, max_jobs=512, max_steps=12)
    with pytest.raises(sx.SimplexError):
        srv.submit(jobs[0])                     # no session yet
    srv.begin()
    ids = []
    for k, job in enumerate(jobs):
        ids.append(srv.submit(job))
        if k % 3 == 0:
            srv.poll()
    assert ids == list(range(len(jobs)))
    mid = ids[len(ids) // 2]
    srv.wait(mid)
    assert srv.result(mid)["status"] == 2
    srv.wait()
    strip = lambda r: {k: v for k, v in r.items() if not k.endswith("_ms")}
    for i, job in enumerate(jobs):
        assert strip(srv.result(i, job["steps"])) == strip(ref.result(i, job["steps"])), f"job {i}"
    st = srv.stats()
    assert st["completed"] == len(jobs) and st["rejected"] == 0
    with pytest.raises(sx.SimplexError):
        srv.wait(len(jobs) + 5)
    with pytest.raises(sx.SimplexError):
        srv.submit(dict(jobs[0], steps=13))     # more than max_steps
    # a second session starts clean
    srv.begin()
    assert srv.submit(jobs[1]) == 0
    srv.wait()
    assert strip(srv.result(0, jobs[1]["steps"])) == strip(ref.result(1, jobs[1]["steps"]))


def test_budget_limits_resident_memory_and_rejects_oversized_jobs():
    rule = inputs.B3S23
    thr = inputs.bernoulli_threshold(0.5)
    jobs = [dict(m=2, n=2047, steps=6, birth=rule[0], survive=rule[1], seed=k, threshold=thr) for k in range(12)]
    jobs.append(dict(m=2, n=8191, steps=2, birth=rule[0], survive=rule[1], seed=99, threshold=thr))  # 2 x 64 MiB
    budget = 40 << 20                                                                                # 40 MiB
    srv = sx.SimplexServer(hbm_budget=budget, max_jobs=64, max_steps=8)
    srv.run(jobs, None, realtime=False)
    st = srv.stats()
    assert st["completed"] == 12 and st["rejected"] == 1
    assert st["peak_pool_bytes"] <= budget
    assert srv.result(12)["status"] == 3
    for i in (0, 5, 11):
        dig, live, _, _ = _alone(jobs[i])
        r = srv.result(i, 6)
        assert r["digest"] == dig and r["live"] == live


def test_server_is_reusable_and_rejects_bad_jobs():
    srv = sx.SimplexServer(hbm_budget=256 << 20, max_jobs=16, max_steps=4)
    rule = inputs.B3S23
    good = [dict(m=2, n=100, steps=3, birth=rule[0], survive=rule[1], seed=1, threshold=1 << 31)]
    srv.run(good, None, realtime=False)
    first = srv.result(0, 3)
    srv.run(good, None, realtime=False)
    again = srv.result(0, 3)
    assert (again["digest"], again["live"], again["status"]) == (first["digest"], first["live"], first["status"])
    with pytest.raises(sx.SimplexError):
        srv.run([dict(good[0], steps=9)], None, realtime=False)
    with pytest.raises(sx.SimplexError):
        srv.run([dict(good[0], m=4)], None, realtime=False)
    # empty: a trace without jobs, and a session that waits with nothing submitted
    srv.run([], None, realtime=False)
    assert srv.stats()["submitted"] == 0 and srv.stats()["completed"] == 0
    srv.begin()
    srv.wait()
    assert srv.poll() == 0
    assert sx.simplex_device_status() == 0
