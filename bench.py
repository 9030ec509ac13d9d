"""Benchmark of the simplex automaton hot path (one JSON line on rank 0).

Default workload: the automaton on the 2-simplex, n = 32767 (536,887,296 cells)
in a dense 32768^2 uint8 grid, Bernoulli(0.5), B3/S23, 100 steps, 128 x 128
tiles mapped by H.  One benchmark step = one simplex_ca_run of the 100
automaton steps (CUDA-graph replay, per-step live counts) on device-resident
grids; the grids (1 GiB each) are far larger than L2, so no flush is needed
between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload ca2|ca3|write2|write4]

--impl reference times the CPU oracle on this host's cores on a bounded
sample of the same workload (the reference arm).  Under torchrun (N > 1) every
rank runs an independent replica (the path is not sharded); rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2208_11617_gb300 import inputs  # noqa: E402

METRIC = "simplex cells/s & HBM-roofline % of H vs bounding-box map; serve p99 latency"
UNIT = "cell-updates/s"


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one
# ncu captures of the full-size workloads (dram__bytes_read.sum +
# dram__bytes_write.sum per launch, mean of 3 launches), keyed by a fingerprint
# of the sources the kernel's traffic depends on: a changed kernel reports null
# until it is measured again.
_CSRC = "paper_2208_11617_gb300/csrc/"
_KERNEL_SOURCES = {
    "ca2_step_kernel<128>": ["k_ca2.cu", "ca_tiles.cuh", "common.cuh", "hmap.cuh", "rule.h", "tmap.cpp"],
    "ca3_step_kernel<32>": ["k_ca3.cu", "ca_tiles.cuh", "common.cuh", "hmap.cuh", "rule.h", "tmap.cpp", "kernels.h"],
    "ca3_step_stream": ["k_ca3.cu", "ca_tiles.cuh", "common.cuh", "hmap.cuh", "rule.h", "tmap.cpp", "kernels.h"],
    "ca3_step_planes": ["k_ca3p.cu", "ca_tiles.cuh", "common.cuh", "hmap.cuh", "rule.h", "tmap.cpp", "kernels.h"],
    "write_kernel<2>": ["k_write.cu", "common.cuh", "hmap.cuh", "tile.cuh", "kernels.h"],
}
# ncu dram__bytes_read.sum + dram__bytes_write.sum per launch (mean of 3 launches
# at full size), for the kernel sources with the given fingerprint, at the
# given n and tile size
_KERNEL_TRAFFIC = {("32f88cfef9b587ce", "ca2_step_kernel<128>", 32767, 128): 1_032_765_866,
                   ("ff5e3aa57fa66250", "ca3_step_planes", 1023, 32): 384_356_864,
                   ("afe643cc8e1992fd", "write_kernel<2>", 32767, 128): 2_085_882_453,
                   ("509b2c66697ba39c", "ca3_step_kernel<32>", 1023, 32): 520_881_749,
                   ("509b2c66697ba39c", "ca3_step_stream", 1023, 32): 398_068_906}


def _kernel_fingerprint(kname):
    """Hash of the kernel's sources with comments and whitespace removed: a
    change to the code (not to its comments) drops the recorded traffic."""
    import hashlib
    import re
    h = hashlib.sha1()
    for f in _KERNEL_SOURCES.get(kname, []):
        with open(os.path.join(ROOT, _CSRC + f), encoding="utf-8") as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)   # block comments
        text = re.sub(r"//[^\n]*", " ", text)                # line comments
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------- clocks
class EnergyMeter:
    """Board energy of the GPU over a region: NVML's total-energy counter
    (millijoules since the driver loaded), read through the driver's
    libnvidia-ml with read-only queries.  read() returns joules, or None where
    NVML or the counter is not available."""

    def __init__(self, torch_index: int):
        import ctypes
        self.dev = None
        try:
            import torch
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return
            dev = ctypes.c_void_p()
            pr = torch.cuda.get_device_properties(torch_index)
            bus = getattr(pr, "pci_bus_id", None)
            ok = False
            if bus is not None:
                busid = "%08X:%02X:%02X.0" % (getattr(pr, "pci_domain_id", 0), bus, getattr(pr, "pci_device_id", 0))
                ok = lib.nvmlDeviceGetHandleByPciBusId_v2(busid.encode(), ctypes.byref(dev)) == 0
            if not ok:
                ok = lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(torch_index), ctypes.byref(dev)) == 0
            if ok:
                self.lib, self.dev = lib, dev
        except Exception:
            self.dev = None

    def read(self):
        import ctypes
        if self.dev is None:
            return None
        mj = ctypes.c_ulonglong()
        if self.lib.nvmlDeviceGetTotalEnergyConsumption(self.dev, ctypes.byref(mj)) != 0:
            return None
        return mj.value * 1e-3


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- distributed
def _dist_init():
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and not dist.is_initialized():
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return rank, world, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def aggregate(units_per_rank: float, seconds: float, world: int):
    """Whole-job throughput: units of all ranks over the slowest rank's time."""
    if world > 1:
        import torch
        import torch.distributed as dist
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([seconds, units_per_rank], dtype=torch.float64, device=dev)
        mx = t.clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        sm = t.clone()
        dist.all_reduce(sm, op=dist.ReduceOp.SUM)
        return float(sm[1].item()) / float(mx[0].item()), float(mx[0].item())
    return units_per_rank / seconds, seconds


# ---------------------------------------------------------------- our arm
def _workload(name, args=None):
    import dataclasses
    if name == "ca2":
        wl = inputs.CA_M2
    elif name == "ca3":
        wl = inputs.CA_M3
    elif name == "write2":
        wl = inputs.WRITE_M2
    elif name == "write2hbm":
        wl = inputs.WRITE_M2_HBM
    elif name == "write4":
        wl = inputs.WRITE_M4
    elif name == "accum2":
        wl = inputs.ACCUM_M2
    elif name == "accum3":
        wl = inputs.ACCUM_M3
    elif name == "map2":
        wl = inputs.MAP_M2
    elif name == "map3":
        wl = inputs.MAP_M3
    elif name == "edm":
        wl = inputs.WriteWorkload(f"edm m=2 n={inputs.EDM_N} dim={inputs.EDM_DIM} rho={inputs.EDM_BLOCK}", m=2,
                                  n=inputs.EDM_N, block=inputs.EDM_BLOCK)
    elif name == "batch":
        return "batch"
    elif name == "serve":
        return "serve"
    else:
        raise SystemExit(f"unknown workload {name}")
    if args is not None:
        # smaller or differently tiled cases of the same workload (profiling, sweeps)
        ch = {}
        if args.n is not None:
            ch["n"] = args.n
        if args.block is not None:
            ch["block"] = args.block
        if args.ca_steps is not None and isinstance(wl, inputs.CAWorkload):
            ch["steps"] = args.ca_steps
        if ch:
            ch["name"] = wl.name + " (" + ", ".join(f"{k}={v}" for k, v in ch.items()) + ")"
            wl = dataclasses.replace(wl, **ch)
    return wl


def _single_grid_blocks(info):
    """CUDA blocks of the write, ACCUM, MAP and EDM launches: they take the
    single Eq. map2d grid on the power-of-two side for m = 2 and r = 1/2,
    whatever the plan's trapezoid band (which the automaton uses)."""
    if info["m"] == 2 and info["r_inv"] == 2 and info["band"]:
        N = info["N"]
        return (N // 2) * (N - 1) + N
    return info["h_blocks"]


def _map_name(info):
    if info["m"] == 2 and info.get("r_inv") == 3:
        return "H with r=1/3, beta=3: three squares and three triangles per split, power-of-three lattice"
    if info["m"] == 2 and info["band"]:
        return f"H, trapezoid bands of {info['band']} tile rows (r=1/2, beta=2)"
    if info["m"] == 2:
        return "H, single Eq. map2d grid (r=1/2, beta=2)"
    if info.get("layout") == 1:
        return "H3, one block range per stack level (fully efficient, r=1/2, beta=2)"
    if info.get("launch") == 2:
        return "x-stream: H2 (Eq. map2d) over the tile columns, runs of up to 16 tiles along x3"
    if info.get("launch") == 3:
        return ("plane stream: slabs of planes x1 cut into 32 x 128 bricks, numbered slab by slab, "
                "each brick streamed along x1")
    return f"H (r=1/{info['r_inv']}, beta={info['beta']})"


def _time_region(fn, steps, warmup, world):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    _barrier(world)
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(steps):
        fn()
    e.record()
    torch.cuda.synchronize()
    _barrier(world)
    return s.elapsed_time(e) / 1e3


_ENERGY = True  # --no-energy clears it (e.g. for a profiler run of a few launches)


def _energy_region(meter, fn, per_call_s, units_per_call, seconds=1.5):
    """Board energy of fn: NVML's counter is coarse, so fn runs back to back for
    about `seconds` (apart from the timed region) and the energy is divided
    over the calls.  Returns joules per call, average watts and units per joule."""
    import torch
    if not _ENERGY:
        return {"joules_per_step": None, "note": "not measured (--no-energy)"}
    if meter is None or meter.dev is None:
        return {"joules_per_step": None, "note": "NVML energy counter unavailable"}
    calls = max(1, int(seconds / max(per_call_s, 1e-6)))
    torch.cuda.synchronize()
    t0, j0 = time.perf_counter(), meter.read()
    for _ in range(calls):
        fn()
    torch.cuda.synchronize()
    t1, j1 = time.perf_counter(), meter.read()
    if j0 is None or j1 is None or j1 <= j0:
        return {"joules_per_step": None, "note": "NVML energy counter did not advance"}
    joules = j1 - j0
    return {"joules_per_step": joules / calls, "avg_watts": joules / (t1 - t0),
            "units_per_joule": units_per_call * calls / joules, "calls": calls}


def _per_launch_ms(launch, reps):
    """Average device duration of one kernel launch, CUDA events on the launching stream."""
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    launch()
    torch.cuda.synchronize()
    for s, e in evs:
        s.record()
        launch()
        e.record()
    torch.cuda.synchronize()
    ts = sorted(s.elapsed_time(e) for s, e in evs)
    return statistics.mean(ts), statistics.median(ts)


def run_batch(args, rank, world, compact=False):
    """Batched workload: 2048 + 256 automata, 16 steps per benchmark step, one
    persistent launch per automaton step (graph replay), against looping the
    single-instance path over the instances."""
    import torch
    from paper_2208_11617_gb300 import autotune
    from paper_2208_11617_gb300 import simplex as sx

    base = inputs.batch_instances(n2=args.batch_m2, n3=args.batch_m3)
    if args.batch_nmin is not None or args.batch_nmax is not None:
        lo = args.batch_nmin if args.batch_nmin is not None else 0
        hi = args.batch_nmax if args.batch_nmax is not None else 1 << 62
        base = [d for d in base if lo <= d["n"] <= hi]
    t0 = time.perf_counter()
    table = {} if args.no_tune else autotune.tune(base, cache=args.tune_cache)
    tune_s = time.perf_counter() - t0
    insts = autotune.apply(base, table)
    steps = inputs.BATCH_STEPS
    b = sx.simplex_batch_create(insts)
    info = sx.simplex_batch_info(b)
    sx.simplex_batch_bind(b)
    sx.simplex_batch_init(b)
    live = torch.zeros(len(insts) * (steps + 1), dtype=torch.int64, device="cuda")
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    secs = _time_region(lambda: sx.simplex_batch_run(b, steps, live), args.steps, args.warmup, world)
    clk = clocks.stop()
    cells = info["cells"]
    value, tmax = aggregate(cells * steps * args.steps, secs, world)
    # one automaton step of every instance = one launch: time a live-less run / steps
    run_ms, _ = _per_launch_ms(lambda: sx.simplex_batch_run(b, steps, None), 5)
    step_ms = run_ms / steps
    hbm_peak, peak_kind = _peaks()
    achieved = 2 * cells / (step_ms * 1e-3) / 1e9
    # baseline: the single-instance path looped over the instances (each a graph of 16 steps)
    maps = []
    for d in ([] if args.no_loop else insts):
        side = (d["n"] + 16) // 16 * 16
        plane = d["m"] == 3 and d["block"] == 128  # the plane stream: launch 3 of a single instance
        mp = sx.simplex_map_create(d["m"], d["n"], 2, d["beta"], 32 if plane else d["block"], side=side,
                                   launch=3 if plane else 0)
        a = torch.zeros(mp.numel, dtype=torch.uint8, device="cuda")
        bb = torch.zeros_like(a)
        sx.simplex_ca_init(mp, a, d["seed"], d["threshold"])
        maps.append((mp, a, bb, d))

    def loop():
        for mp, a, bb, d in maps:
            sx.simplex_ca_run(mp, a, bb, steps, d["birth"], d["survive"], None, True)

    secs_loop = _time_region(loop, 1, 1, world) if maps else float("nan")
    value_loop = aggregate(cells * steps, secs_loop, world)[0] if maps else float("nan")
    assert sx.simplex_device_status() == 0
    if compact:
        return {"workload": "2048 m=2 (n log-U[64,2048]) + 256 m=3 (n log-U[32,256]), 16 steps, one persistent "
                            "launch per step, graph replay", "instances": len(insts), "cells": cells,
                "cell_updates_per_s": value, "ms_per_16_steps": tmax / args.steps * 1e3,
                "kernel_ms_per_step": step_ms, "roofline_frac": achieved / hbm_peak, "peak_kind": peak_kind,
                "single_instance_loop_cell_updates_per_s": value_loop, "speedup_over_loop": value / value_loop,
                "autotuned": not args.no_tune, "tune_seconds": tune_s}
    return dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
        ms_per_step=tmax / args.steps * 1e3, higher_is_better=True, scaling="weak", vs_baseline=None,
        dtype="u8", data="synthetic",
        config={"workload": "batched: 2048 m=2 (n log-U[64,2048]) + 256 m=3 (n log-U[32,256]), Bernoulli(0.4), "
                            "B3/S23 / B5/S45, 16 steps", "instances": len(insts), "cells": cells,
                "work_items_per_step": info["items"], "map_blocks_per_step": info["blocks"],
                "autotuned": {f"m={k[0]} log2n={k[1]}": v for k, v in table.items()}, "tune_seconds": tune_s,
                "parallelism": "replicas" if world > 1 else "single"},
        roofline={"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                  "frac": achieved / hbm_peak, "traffic": None, "peak_kind": peak_kind, "kernel": "batch_kernel",
                  "alg_bytes_per_launch": 2 * cells, "launch_ms_mean": step_ms},
        clocks=clk, gpu_launches=args.steps * (steps + 1),
        single_instance_loop={"value": value_loop, "speedup_batched": value / value_loop,
                              "ms_per_step": secs_loop * 1e3},
        e2e={"value": None, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    )


def _fifo_latency(arrivals_s, service_s):
    """FIFO single-server queue (Lindley): completion - arrival per job, seconds."""
    free_at = 0.0
    out = []
    for a, sv in zip(arrivals_s, service_s):
        start = max(a, free_at)
        free_at = start + sv
        out.append(free_at - a)
    return out


def _serve_classes(srv, jobs):
    """Latency by job class (m, and n above or below the class median) and the
    make-up of the jobs at or above the trace's p99 latency."""
    lat = np.array([srv.result(i)["done_ms"] - srv.result(i)["arrival_ms"] for i in range(len(jobs))])
    ms = np.array([d["m"] for d in jobs])
    ns = np.array([d["n"] for d in jobs])
    steps = np.array([d["steps"] for d in jobs])
    out = {}
    for m in (2, 3):
        sel = ms == m
        if not sel.any():
            continue
        med = float(np.median(ns[sel]))
        for part, cond in (("small", ns <= med), ("large", ns > med)):
            l = lat[sel & cond]
            if len(l):
                out[f"m{m}_{part}"] = {"jobs": int(len(l)), "n_range": [int(ns[sel & cond].min()), int(ns[sel & cond].max())],
                                       "p50_ms": float(np.percentile(l, 50)), "p99_ms": float(np.percentile(l, 99))}
    tail = lat >= np.percentile(lat, 99)
    out["tail_p99"] = {"jobs": int(tail.sum()), "m3_share": float((ms[tail] == 3).mean()),
                       "mean_n_m2": float(ns[tail & (ms == 2)].mean()) if (tail & (ms == 2)).any() else None,
                       "mean_n_m3": float(ns[tail & (ms == 3)].mean()) if (tail & (ms == 3)).any() else None,
                       "mean_steps": float(steps[tail].mean())}
    return out


def run_serve(args, rank, world, compact=False):
    """Serving workload: Poisson arrivals at 2000 jobs/s, continuous batching
    under a 64 GiB grid budget; p50/p99 latency and cell-updates/s, against
    serial per-job execution on the single-instance path.  compact: the trace
    and the serial baseline only (no capacity or heavy-load runs)."""
    import torch
    from paper_2208_11617_gb300 import simplex as sx

    seconds = args.serve_seconds
    jobs, t = inputs.serve_trace(seconds=seconds)
    srv = sx.SimplexServer(hbm_budget=inputs.SERVE_BUDGET, max_jobs=8192, max_steps=64, max_items=1 << 18,
                           max_inflight=args.max_inflight, round_steps=args.round_steps, direct_jobs=args.direct_jobs)
    warm, wt = inputs.serve_trace(seconds=0.05, seed=5)
    srv.run(warm, wt, realtime=True)                  # warm-up trace (not timed)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    t0 = time.perf_counter()
    srv.run(jobs, t, realtime=True)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    st = srv.stats()
    value = st["cell_updates"] / wall
    by_class = _serve_classes(srv, jobs)
    # serial per-job execution: service time of each job alone (a sample), then a FIFO queue
    rng = np.random.default_rng(7)
    sample = sorted(rng.choice(len(jobs), size=min(args.serve_sample, len(jobs)), replace=False).tolist())
    svc, cu, mismatches = [], 0, 0
    for i in sample:
        d = jobs[i]
        side = (d["n"] + 16) // 16 * 16
        block = (128 if d["n"] >= 1024 else 64) if d["m"] == 2 else 16
        mp = sx.simplex_map_create(d["m"], d["n"], 2, 2, block, side=side)
        a = torch.zeros(mp.numel, dtype=torch.uint8, device="cuda")
        b = torch.zeros_like(a)
        dig = torch.zeros(1, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        s0 = time.perf_counter()
        sx.simplex_ca_init(mp, a, d["seed"], d["threshold"])
        fin = sx.simplex_ca_run(mp, a, b, d["steps"], d["birth"], d["survive"], None, False)
        sx.simplex_ca_digest(mp, fin, dig)
        torch.cuda.synchronize()
        svc.append(time.perf_counter() - s0)
        cu += mp.info.cells * d["steps"]
        if (int(dig.item()) & ((1 << 64) - 1)) != srv.result(i)["digest"]:
            mismatches += 1
    serial_rate = cu / sum(svc)
    mean_svc = sum(svc) / len(svc)
    # serial latency under the same arrivals, service times resampled from the sample
    svc_all = [svc[k % len(svc)] for k in range(len(jobs))]
    lat = sorted(_fifo_latency(list(t), svc_all))
    q = lambda f: lat[min(len(lat) - 1, int(f * (len(lat) - 1) + 0.5))] * 1e3
    assert mismatches == 0, f"{mismatches} jobs differ between the server and the single-instance path"
    if compact:
        return {"trace": f"Poisson {inputs.SERVE_RATE:g} jobs/s for {seconds:g} s", "jobs": len(jobs),
                "completed": st["completed"], "cell_updates_per_s": value,
                "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                "host_p50_ms": st["host_p50_ms"], "host_p99_ms": st["host_p99_ms"],
                "serial_fifo_p50_ms": q(0.5), "serial_fifo_p99_ms": q(0.99),
                "serial_cell_updates_per_s": serial_rate, "serial_sample_jobs": len(sample),
                "digest_mismatches": mismatches, "gpu_launches": st["launches"],
                "note": "p*_ms: arrival to the device event after the job's result copies; host_p*_ms: arrival to "
                        "the serving loop finding it complete; serial: FIFO queue of the same arrivals served one "
                        "job at a time on the single-instance path"}
    # capacity: the first jobs of the trace all available at once (no arrival gaps)
    cap_jobs = jobs[: args.serve_capacity_jobs]
    t1 = time.perf_counter()
    srv.run(cap_jobs, None, realtime=False)
    cap_wall = time.perf_counter() - t1
    cap = srv.stats()
    cap_svc = [svc[k % len(svc)] for k in range(len(cap_jobs))]
    serial_cap_rate = sum(
        ((d["n"] + 1) * (d["n"] + 2) // 2 if d["m"] == 2 else (d["n"] + 1) * (d["n"] + 2) * (d["n"] + 3) // 6)
        * d["steps"] for d in cap_jobs) / sum(cap_svc)
    # heavier load: where the serial path saturates
    hl_rate = args.serve_high_rate
    hjobs, ht = inputs.serve_trace(rate=hl_rate, seconds=args.serve_high_seconds, seed=9)
    srv.run(hjobs, ht, realtime=True)
    hl = srv.stats()
    hlat = sorted(_fifo_latency(list(ht), [svc[k % len(svc)] for k in range(len(hjobs))]))
    hq = lambda f: hlat[min(len(hlat) - 1, int(f * (len(hlat) - 1) + 0.5))] * 1e3
    assert mismatches == 0, f"{mismatches} jobs differ between the server and the single-instance path"
    assert sx.simplex_device_status() == 0
    return dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=1, warmup=1, ms_per_step=wall * 1e3,
        higher_is_better=True, scaling="weak", vs_baseline=None, dtype="u8", data="synthetic",
        config={"workload": f"serving: Poisson {inputs.SERVE_RATE:g} jobs/s for {seconds:g} s, 80/20 m=2/m=3, "
                            "n log-U[128,8192]/[32,512], steps U{1..64}, Bernoulli(0.5), 64 GiB grid budget",
                "jobs": len(jobs), "parallelism": "replicas" if world > 1 else "single"},
        serve={"p50_ms": st["p50_ms"], "p90_ms": st["p90_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
               "mean_ms": st["mean_ms"], "host_p50_ms": st["host_p50_ms"], "host_p99_ms": st["host_p99_ms"],
               "latency_note": "p*_ms: arrival to the device event after the job's result copies; host_p*_ms: "
                               "arrival to the serving loop finding the job complete", "completed": st["completed"], "rejected": st["rejected"],
               "rounds": st["rounds"], "mean_resident_jobs": st["mean_active"],
               "peak_pool_gib": st["peak_pool_bytes"] / 2 ** 30, "offered_cell_updates_per_s":
                   st["cell_updates"] / seconds},
        serve_by_class=by_class,
        serial={"cell_updates_per_s": serial_rate, "mean_service_ms": mean_svc * 1e3,
                "utilisation_at_this_rate": inputs.SERVE_RATE * mean_svc, "p50_ms": q(0.5), "p99_ms": q(0.99),
                "sample_jobs": len(sample), "digest_mismatches": mismatches},
        host_issue_ms_per_round=st["host_issue_ms"] / max(1, st["rounds"]),
        gpu_ms_per_round=st["gpu_round_ms"],
        gpu_busy_fraction=st["gpu_round_ms"] * st["rounds"] / (wall * 1e3),
        capacity={"jobs": len(cap_jobs), "server_cell_updates_per_s": cap["cell_updates"] / cap_wall,
                  "serial_cell_updates_per_s": serial_cap_rate, "server_over_serial":
                      (cap["cell_updates"] / cap_wall) / serial_cap_rate, "mean_resident_jobs": cap["mean_active"]},
        high_load={"rate_jobs_per_s": hl_rate, "seconds": args.serve_high_seconds, "jobs": len(hjobs),
                   "server_p50_ms": hl["p50_ms"], "server_p99_ms": hl["p99_ms"],
                   "server_host_p50_ms": hl["host_p50_ms"], "server_host_p99_ms": hl["host_p99_ms"],
                   "server_cell_updates_per_s": hl["cell_updates"] / (hl["wall_ms"] * 1e-3),
                   "mean_resident_jobs": hl["mean_active"], "serial_utilisation": hl_rate * mean_svc,
                   "serial_fifo_p50_ms": hq(0.5), "serial_fifo_p99_ms": hq(0.99)},
        roofline=None, clocks=clk, gpu_launches=st["launches"],
        e2e={"value": None, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    )


def run_ours(args, rank, world, local):
    import torch
    from paper_2208_11617_gb300 import simplex as sx

    torch.cuda.set_device(local)
    wl = _workload(args.workload, args)
    if wl == "batch":
        return run_batch(args, rank, world)
    if wl == "serve":
        return run_serve(args, rank, world)
    if args.workload in ("map2", "map3", "edm"):
        return run_diag(args, wl, rank, world)
    hbm_peak, peak_kind = _peaks()
    res = {}
    if isinstance(wl, inputs.CAWorkload):
        # m = 3: the plane stream (the fastest form) unless --launch says otherwise;
        # the other forms are timed beside it below
        launch = args.launch if (args.launch or wl.m != 3) else 3
        mp = sx.simplex_map_create(wl.m, wl.n, 2, 2, wl.block, band=args.band if wl.m == 2 else None,
                                   launch=launch, layout=args.layout if wl.m == 3 else 0, side=args.side)
        info = sx.simplex_map_info(mp)
        cells = info["cells"]
        a = torch.zeros(mp.numel, dtype=torch.uint8, device="cuda")
        b = torch.zeros_like(a)
        sx.simplex_ca_init(mp, a, wl.seed, wl.threshold)
        live = torch.zeros(wl.steps + 1, dtype=torch.int64, device="cuda")
        birth, survive = wl.rule

        def step(mode):
            return lambda: sx.simplex_ca_run(mp, a, b, wl.steps, birth, survive, live, True, mode)

        clocks = ClockSampler(torch.cuda.current_device())
        clocks.start()
        secs = _time_region(step(sx.SIMPLEX_MODE_H), args.steps, args.warmup, world)
        clk = clocks.stop()
        secs_bb = secs if args.no_bb else _time_region(step(sx.SIMPLEX_MODE_BB), args.steps, max(1, args.warmup),
                                                       world)
        units = cells * wl.steps * args.steps
        value, tmax = aggregate(units, secs, world)
        value_bb, _ = aggregate(units, secs_bb, world)
        # dominant kernel: one automaton step; its average launch duration
        nxt = torch.zeros_like(a)
        mean_ms, med_ms = _per_launch_ms(lambda: sx.simplex_ca_step(mp, a, nxt, birth, survive, None), 20)
        mean_bb = mean_ms if args.no_bb else _per_launch_ms(
            lambda: sx.simplex_ca_step(mp, a, nxt, birth, survive, None, sx.SIMPLEX_MODE_BB), 20)[0]
        mean_bbt = mean_ms if args.no_bb else _per_launch_ms(
            lambda: sx.simplex_ca_step(mp, a, nxt, birth, survive, None, sx.SIMPLEX_MODE_BB_THREAD), 10)[0]
        alg_bytes = 2 * cells
        achieved = alg_bytes / (mean_ms * 1e-3) / 1e9
        kname = {2: "ca3_step_stream", 3: "ca3_step_planes"}.get(info["launch"], f"ca{wl.m}_step_kernel<{wl.block}>")
        res.update(
            metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
            ms_per_step=tmax / args.steps * 1e3, higher_is_better=True, scaling="weak", vs_baseline=None,
            dtype="u8", data="synthetic",
            config={"workload": wl.name, "m": wl.m, "n": wl.n, "array": f"{mp.side}^{wl.m} uint8",
                    "tile": f"{wl.block}^{wl.m}", "ca_steps_per_step": wl.steps, "p": wl.p,
                    "rule": "B3/S23" if wl.m == 2 else "B5/S45", "map": _map_name(info),
                    "cells": cells, "parallelism": "replicas" if world > 1 else "single",
                    "l2": "inputs 1 GiB per grid >> 129 MB L2, no flush"},
            roofline={"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                      "frac": achieved / hbm_peak, "peak_kind": peak_kind,
                      "kernel": kname, "alg_bytes_per_launch": alg_bytes,
                      "traffic": _KERNEL_TRAFFIC.get((_kernel_fingerprint(kname), kname, wl.n, wl.block)),
                      "launch_ms_mean": mean_ms, "launch_ms_median": med_ms},
            clocks=clk,
            gpu_launches=args.steps * (wl.steps + 1),
            bb={"value": value_bb, "speedup_h_over_bb": value / value_bb, "launch_ms_mean": mean_bb,
                "kernel_speedup_h_over_bb": mean_bb / mean_ms},
            bb_thread={"launch_ms_mean": mean_bbt, "kernel_speedup_h_over_bb_thread": mean_bbt / mean_ms,
                       "note": "bounding box with a per-thread filter only (the paper's baseline)"},
            blocks={"h": info["h_blocks"], "bb": info["bb_blocks"], "useful": info["useful_blocks"],
                    "wasted_frac_h": 1 - info["useful_blocks"] / info["h_blocks"],
                    "wasted_frac_bb": 1 - info["useful_blocks"] / info["bb_blocks"]},
        )
        meter = EnergyMeter(torch.cuda.current_device())
        res["energy"] = {
            "h": _energy_region(meter, step(sx.SIMPLEX_MODE_H), secs / args.steps, cells * wl.steps),
            "bb": None if args.no_bb else _energy_region(meter, step(sx.SIMPLEX_MODE_BB), secs_bb / args.steps,
                                                          cells * wl.steps),
            "unit": "cell-updates per joule (board energy, NVML, a separate ~1.5 s run per map)"}
        if wl.m == 3 and info["launch"] != 3:
            # the plane-stream form on the same grids
            mpq = sx.simplex_map_create(wl.m, wl.n, 2, 2, wl.block, launch=3, side=args.side)
            mq_ms = _per_launch_ms(lambda: sx.simplex_ca_step(mpq, a, nxt, birth, survive, None), 20)[0]
            ach_q = alg_bytes / (mq_ms * 1e-3) / 1e9
            res["plane_stream"] = {"kernel": "ca3_step_planes", "launch_ms_mean": mq_ms, "achieved": ach_q,
                                   "frac": ach_q / hbm_peak,
                                   "traffic": _KERNEL_TRAFFIC.get((_kernel_fingerprint("ca3_step_planes"),
                                                                   "ca3_step_planes", wl.n, wl.block)),
                                   "note": "same step, plane-stream form (launch 3)"}
        if wl.m == 3 and info["launch"] != 1:
            # the paper's execution model on the same grids: one CTA per block of H3
            mpg = sx.simplex_map_create(wl.m, wl.n, 2, 2, wl.block, launch=1, layout=args.layout, side=args.side)
            mg_ms = _per_launch_ms(lambda: sx.simplex_ca_step(mpg, a, nxt, birth, survive, None), 20)[0]
            ach_g = alg_bytes / (mg_ms * 1e-3) / 1e9
            kg = f"ca3_step_kernel<{wl.block}>"
            res["grid_form"] = {"kernel": kg, "launch_ms_mean": mg_ms, "achieved": ach_g, "frac": ach_g / hbm_peak,
                                "traffic": _KERNEL_TRAFFIC.get((_kernel_fingerprint(kg), kg, wl.n, wl.block)),
                                "note": "same step, one CTA per block of H3 (launch 1, Sec. 4.3 map)"}
        if wl.m == 3 and wl.block == 32 and info["launch"] != 2:
            # the other m = 3 step form on the same grids: persistent CTAs streaming
            # slab columns along x3 (H2 over the tile columns)
            mpx = sx.simplex_map_create(wl.m, wl.n, 2, 2, wl.block, launch=2, side=args.side)
            mx_ms = _per_launch_ms(lambda: sx.simplex_ca_step(mpx, a, nxt, birth, survive, None), 20)[0]
            ach_x = alg_bytes / (mx_ms * 1e-3) / 1e9
            res["x_stream"] = {"kernel": "ca3_step_stream", "launch_ms_mean": mx_ms, "achieved": ach_x,
                               "frac": ach_x / hbm_peak,
                               "traffic": _KERNEL_TRAFFIC.get((_kernel_fingerprint("ca3_step_stream"),
                                                               "ca3_step_stream", wl.n, wl.block)),
                               "note": "same step, x-stream form (launch 2)"}
        # end to end through the C ABI from pinned host memory
        e2e_steps = 0 if args.no_e2e else max(1, min(3, args.steps))
        e2e_val = None
        if e2e_steps:
            h_in = torch.empty(mp.numel, dtype=torch.uint8).pin_memory()
            h_in.copy_(a.cpu())
            h_out = torch.empty_like(h_in).pin_memory()
            h_live = torch.zeros(wl.steps + 1, dtype=torch.int64)
            sx.simplex_ca_run_host(mp, h_in, h_out, a, b, wl.steps, birth, survive, live, h_live)
            torch.cuda.synchronize()
            _barrier(world)
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                sx.simplex_ca_run_host(mp, h_in, h_out, a, b, wl.steps, birth, survive, live, h_live)
            t1 = time.perf_counter()
            e2e_val = aggregate(cells * wl.steps * e2e_steps, t1 - t0, world)[0]
        # the call moves the domain's row prefixes only (host_copy_bytes each way)
        res["e2e"] = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": info["host_copy_bytes"],
                      "d2h_bytes_per_step": info["host_copy_bytes"] + 8 * (wl.steps + 1),
                      "array_bytes": mp.numel}
        assert sx.simplex_device_status() == 0
    else:
        r_inv = args.r_inv if wl.m == 2 else 2
        beta = 3 if r_inv == 3 else (2 if wl.m <= 3 else wl.m)
        mp = sx.simplex_map_create(wl.m, wl.n, r_inv, beta, wl.block,
                                   band=(args.band if r_inv == 2 else -1) if wl.m == 2 else None)
        info = sx.simplex_map_info(mp)
        cells = info["cells"]
        out = torch.zeros(mp.numel, dtype=torch.int32, device="cuda")
        # many launches per benchmark step (the write of one array is a few
        # microseconds), captured in a CUDA graph so the host is off the path
        reps = 100

        accum = args.workload in ("accum2", "accum3")
        if accum or args.workload == "write2hbm":
            reps = 10  # 1 to 4 GiB arrays: a launch moves 1.1 to 2.1 GB

        def launch(mode):
            if accum:
                sx.simplex_accum(mp, out, 1, mode)
            else:
                sx.simplex_write(mp, out, wl.seed, mode)

        def graph_of(mode):
            g = torch.cuda.CUDAGraph()
            launch(mode)  # warm the launch path outside capture
            torch.cuda.synchronize()
            with torch.cuda.graph(g):
                for _ in range(reps):
                    launch(mode)
            return g

        graphs = {m: graph_of(m) for m in (sx.SIMPLEX_MODE_H, sx.SIMPLEX_MODE_BB, sx.SIMPLEX_MODE_BB_THREAD)}

        def step(mode):
            return graphs[mode].replay

        clocks = ClockSampler(torch.cuda.current_device())
        clocks.start()
        secs = _time_region(step(sx.SIMPLEX_MODE_H), args.steps, args.warmup, world)
        clk = clocks.stop()
        secs_bb = secs if args.no_bb else _time_region(step(sx.SIMPLEX_MODE_BB), args.steps, max(1, args.warmup),
                                                       world)
        units = cells * reps * args.steps
        value, tmax = aggregate(units, secs, world)
        value_bb, _ = aggregate(units, secs_bb, world)
        # per launch: a graph of `reps` back-to-back launches, timed by events, / reps
        mean_ms = _per_launch_ms(graphs[sx.SIMPLEX_MODE_H].replay, 10)[0] / reps
        med_ms = mean_ms
        mean_bb = _per_launch_ms(graphs[sx.SIMPLEX_MODE_BB].replay, 10)[0] / reps
        mean_bbt = _per_launch_ms(graphs[sx.SIMPLEX_MODE_BB_THREAD].replay, 10)[0] / reps
        alg_bytes = (8 if accum else 4) * cells  # ACCUM reads and writes each cell
        achieved = alg_bytes / (mean_ms * 1e-3) / 1e9
        res.update(
            metric=METRIC, value=value, unit="cells/s", n_gpus=world, steps=args.steps, warmup=args.warmup,
            ms_per_step=tmax / args.steps * 1e3, higher_is_better=True, scaling="weak", vs_baseline=None,
            dtype="u32", data="synthetic",
            config={"workload": wl.name, "m": wl.m, "n": wl.n, "array": f"{mp.side}^{wl.m} uint32",
                    "tile": f"{wl.block}^{wl.m}", "launches_per_step": reps, "cells": cells,
                    "map": _map_name(info), "parallelism": "replicas" if world > 1 else "single",
                    "l2": ("arrays of 1 / 4 GiB >> 129 MB L2, no flush" if accum
                           else "array re-written back to back (L2-resident when it fits)")},
            roofline={"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                      "frac": achieved / hbm_peak, "peak_kind": peak_kind,
                      "traffic": None if accum else _KERNEL_TRAFFIC.get(
                          (_kernel_fingerprint(f"write_kernel<{wl.m}>"), f"write_kernel<{wl.m}>", wl.n, wl.block)),
                      "kernel": f"{'accum' if accum else 'write'}_kernel<{wl.m}>", "alg_bytes_per_launch": alg_bytes,
                      "launch_ms_mean": mean_ms, "launch_ms_median": med_ms},
            clocks=clk, gpu_launches=args.steps * reps,
            bb={"value": value_bb, "speedup_h_over_bb": value / value_bb, "launch_ms_mean": mean_bb,
                "kernel_speedup_h_over_bb": mean_bb / mean_ms},
            bb_thread={"launch_ms_mean": mean_bbt, "kernel_speedup_h_over_bb_thread": mean_bbt / mean_ms,
                       "note": "bounding box with a per-thread filter only (the paper's baseline)"},
            blocks={"h": _single_grid_blocks(info), "bb": info["bb_blocks"], "useful": info["useful_blocks"]},
        )
        meter = EnergyMeter(torch.cuda.current_device())
        res["energy"] = {
            "h": _energy_region(meter, step(sx.SIMPLEX_MODE_H), secs / args.steps, cells * reps),
            "bb": None if args.no_bb else _energy_region(meter, step(sx.SIMPLEX_MODE_BB), secs_bb / args.steps,
                                                          cells * reps),
            "unit": "cells per joule (board energy, NVML, a separate ~1.5 s run per map)"}
        # end to end: (ACCUM: the array in from pinned host memory,) the kernel,
        # the array back to pinned host memory
        e2e_val = None
        if not args.no_e2e:
            h_out = torch.empty(mp.numel, dtype=torch.int32).pin_memory()
            h_in = h_out.clone().pin_memory() if accum else None
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(3):
                if accum:
                    out.copy_(h_in, non_blocking=True)
                launch(sx.SIMPLEX_MODE_H)
                h_out.copy_(out, non_blocking=True)
                torch.cuda.synchronize()
            t1 = time.perf_counter()
            e2e_val, _ = aggregate(cells * 3, t1 - t0, world)
        res["e2e"] = {"value": e2e_val, "unit": "cells/s", "h2d_bytes_per_step": 4 * mp.numel if accum else 0,
                      "d2h_bytes_per_step": 4 * mp.numel}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(wl, workload=args.workload, n=args.n)
    if args.workload == "ca2" and args.n is None and world == 1 and not args.no_records:
        # the batched engine and the server, briefly, so that the default line
        # carries them too (their own workloads: --workload batch / serve)
        import copy
        ab = copy.copy(args)
        ab.steps, ab.warmup = 3, 3
        res["batch"] = run_batch(ab, rank, world, compact=True)
        asv = copy.copy(args)
        asv.serve_seconds, asv.serve_sample = 5.0, 200
        res["serve"] = run_serve(asv, rank, world, compact=True)
    return res


def run_diag(args, wl, rank, world):
    """The paper's diagnostics (Table 1): MAP (the map alone; time per launch,
    H against the bounding box and against the block-count ratio the theory
    predicts) and EDM (float32 distance matrix of 3-D points, HBM-bound on its
    4-byte stores).  A step is a graph of `reps` back-to-back launches."""
    import torch
    from paper_2208_11617_gb300 import simplex as sx
    hbm_peak, peak_kind = _peaks()
    r_inv = args.r_inv if wl.m == 2 else 2
    beta = 3 if r_inv == 3 else (2 if wl.m <= 3 else wl.m)
    mp = sx.simplex_map_create(wl.m, wl.n, r_inv, beta, wl.block,
                               band=(args.band if r_inv == 2 else -1) if wl.m == 2 else None,
                               layout=args.layout if wl.m == 3 else 0)
    info = sx.simplex_map_info(mp)
    cells = info["cells"]
    edm = args.workload == "edm"
    if edm:
        pts = torch.from_numpy(inputs.edm_points(wl.n, inputs.EDM_DIM)).cuda()
        out = torch.zeros(mp.numel, dtype=torch.float32, device="cuda")
        launch = lambda mode: sx.simplex_edm(mp, pts, out, mode)  # noqa: E731
        reps = 10
    else:
        launch = lambda mode: sx.simplex_map_test(mp, None, mode)  # noqa: E731
        reps = 100

    def graph_of(mode):
        g = torch.cuda.CUDAGraph()
        launch(mode)
        torch.cuda.synchronize()
        with torch.cuda.graph(g):
            for _ in range(reps):
                launch(mode)
        return g

    graphs = {m: graph_of(m) for m in (sx.SIMPLEX_MODE_H, sx.SIMPLEX_MODE_BB, sx.SIMPLEX_MODE_BB_THREAD)}
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    secs = _time_region(graphs[sx.SIMPLEX_MODE_H].replay, args.steps, args.warmup, world)
    clk = clocks.stop()
    secs_bb = _time_region(graphs[sx.SIMPLEX_MODE_BB].replay, args.steps, max(1, args.warmup), world)
    units = cells * reps * args.steps
    value, tmax = aggregate(units, secs, world)
    value_bb, _ = aggregate(units, secs_bb, world)
    mean_ms = _per_launch_ms(graphs[sx.SIMPLEX_MODE_H].replay, 10)[0] / reps
    mean_bb = _per_launch_ms(graphs[sx.SIMPLEX_MODE_BB].replay, 10)[0] / reps
    mean_bbt = _per_launch_ms(graphs[sx.SIMPLEX_MODE_BB_THREAD].replay, 10)[0] / reps
    res = dict(
        metric=METRIC, value=value, unit="cells/s", n_gpus=world, steps=args.steps, warmup=args.warmup,
        ms_per_step=tmax / args.steps * 1e3, higher_is_better=True, scaling="weak", vs_baseline=None,
        dtype="f32" if edm else "i32", data="synthetic",
        config={"workload": wl.name, "m": wl.m, "n": wl.n, "tile": f"{wl.block}^{wl.m}", "launches_per_step": reps,
                "cells": cells, "map": _map_name(info), "parallelism": "replicas" if world > 1 else "single"},
        clocks=clk, gpu_launches=args.steps * reps,
        bb={"value": value_bb, "speedup_h_over_bb": value / value_bb, "launch_ms_mean": mean_bb,
            "kernel_speedup_h_over_bb": mean_bb / mean_ms},
        bb_thread={"launch_ms_mean": mean_bbt, "kernel_speedup_h_over_bb_thread": mean_bbt / mean_ms,
                   "note": "bounding box with a per-thread filter only (the paper's baseline)"},
        blocks={"h": _single_grid_blocks(info), "bb": info["bb_blocks"], "useful": info["useful_blocks"],
                "bb_over_h": info["bb_blocks"] / _single_grid_blocks(info)},
    )
    meter = EnergyMeter(torch.cuda.current_device())
    res["energy"] = {
        "h": _energy_region(meter, graphs[sx.SIMPLEX_MODE_H].replay, secs / args.steps, cells * reps),
        "bb": _energy_region(meter, graphs[sx.SIMPLEX_MODE_BB].replay, secs_bb / args.steps, cells * reps),
        "unit": "cells per joule (board energy, NVML, a separate ~1.5 s run per map)"}
    if edm:
        alg_bytes = 4 * cells + (wl.n + 1) * inputs.EDM_DIM * 4
        achieved = alg_bytes / (mean_ms * 1e-3) / 1e9
        res["config"]["array"] = f"{mp.side}^2 float32, {wl.n + 1} points x {inputs.EDM_DIM}"
        res["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                           "frac": achieved / hbm_peak, "traffic": None, "peak_kind": peak_kind,
                           "kernel": f"edm_kernel<{wl.block}>", "alg_bytes_per_launch": alg_bytes,
                           "launch_ms_mean": mean_ms}
        # end to end: points in from pinned host memory, matrix back to pinned host memory
        h_pts = pts.cpu().pin_memory()
        h_out = torch.empty(mp.numel, dtype=torch.float32).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(2):
            pts.copy_(h_pts, non_blocking=True)
            sx.simplex_edm(mp, pts, out)
            h_out.copy_(out, non_blocking=True)
            torch.cuda.synchronize()
        t1 = time.perf_counter()
        res["e2e"] = {"value": aggregate(cells * 2, t1 - t0, world)[0], "unit": "cells/s",
                      "h2d_bytes_per_step": h_pts.numel() * 4, "d2h_bytes_per_step": 4 * mp.numel}
    else:
        # the MAP test moves no memory: its bound is launching and retiring blocks
        res["roofline"] = None
        res["roofline_note"] = "MAP moves no memory; compare launch_ms against bb and blocks.bb_over_h"
        res["theory_speedup"] = {2: 2.0, 3: 6.0}.get(wl.m)
        res["e2e"] = {"value": None, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    if rank == 0 and world == 1 and not args.no_cpu_baseline and edm:
        res["cpu_baseline"] = cpu_baseline(wl, edm=True, workload="edm")
    return res


# ---------------------------------------------------------------- oracle (CPU) arm
def _oracle_sample(wl, steps_sample):
    """Time the oracle on a bounded sample of the workload; returns (units/s, note, cores)."""
    import oracle
    cores = oracle.num_threads()
    if isinstance(wl, inputs.CAWorkload):
        g = oracle.ca_init(wl.m, wl.n, wl.seed, wl.threshold)
        cells = oracle.count_cells(wl.m, wl.n)
        t0 = time.perf_counter()
        for _ in range(steps_sample):
            g, _ = oracle.ca_step(wl.m, wl.n, wl.rule[0], wl.rule[1], g)
        dt = time.perf_counter() - t0
        note = f"{steps_sample} automaton step(s) of the full n={wl.n} grid ({cells} cells each)"
        return cells * steps_sample / dt, note, cores, dt
    if wl.name.startswith("accum"):
        # ACCUM on a smaller array of the same simplex dimension (the workload's
        # 1 / 4 GiB arrays would spend the time copying, not adding)
        ns = min(wl.n, 4095 if wl.m == 2 else 511)
        data = np.zeros(oracle.dense_shape(wl.m, ns), dtype=np.uint32)
        cells = oracle.count_cells(wl.m, ns)
        t0 = time.perf_counter()
        for _ in range(steps_sample):
            data = oracle.accum(wl.m, ns, data, 1)
        dt = time.perf_counter() - t0
        return cells * steps_sample / dt, f"{steps_sample} ACCUM pass(es) of n={ns} (array copy included)", cores, dt
    # the write of a smaller array of the same simplex dimension past n = 8191
    # (the 4 GiB array would spend the time allocating and zeroing)
    ns = min(wl.n, 8191)
    cells = oracle.count_cells(wl.m, ns)
    t0 = time.perf_counter()
    for _ in range(steps_sample):
        oracle.write(wl.m, ns, wl.seed)
    dt = time.perf_counter() - t0
    return cells * steps_sample / dt, f"{steps_sample} full write(s) of n={ns}", cores, dt


def _oracle_edm_sample(n_sample):
    """The oracle's distance matrix at a smaller n (whole triangle), cells/s."""
    import oracle
    pts = inputs.edm_points(n_sample, inputs.EDM_DIM)
    t0 = time.perf_counter()
    oracle.edm(n_sample, pts)
    dt = time.perf_counter() - t0
    return oracle.count_cells(2, n_sample) / dt, f"the whole EDM triangle at n={n_sample}", oracle.num_threads(), dt


def _cpu_model() -> str:
    """The host CPU's model string (lscpu, else /proc/cpuinfo, else platform)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "hardware")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


# One bounded oracle sample in a child process with OpenMP limited to one
# thread (the oracle's parallel loops then run serially); prints JSON.
_SINGLE_THREAD_PROBE = r"""
import dataclasses, json, sys
sys.path.insert(0, sys.argv[1])
import bench
wl = bench._workload(sys.argv[2])
if sys.argv[3] != "-":
    wl = dataclasses.replace(wl, n=int(sys.argv[3]))
if sys.argv[4] == "edm":
    v, note, cores, dt = bench._oracle_edm_sample(int(sys.argv[5]))
else:
    v, note, cores, dt = bench._oracle_sample(wl, int(sys.argv[5]))
print(json.dumps({"value": v, "sample": note, "cores": cores, "seconds": dt}))
"""


def _oracle_single_thread(workload, n, edm, sample):
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", _SINGLE_THREAD_PROBE, ROOT, workload, str(n) if n is not None else "-",
                            "edm" if edm else "-", str(sample)], capture_output=True, text=True, timeout=600,
                           env=env)
        if r.returncode == 0:
            return json.loads(r.stdout.strip().splitlines()[-1])
        return {"error": r.stderr.strip().splitlines()[-1] if r.stderr.strip() else f"exit {r.returncode}"}
    except (OSError, subprocess.SubprocessError, ValueError) as exc:
        return {"error": str(exc)}


def cpu_baseline(wl, edm=False, workload=None, n=None):
    """The oracle on all host cores (OpenMP) on a bounded sample, plus the same
    oracle on one thread (a smaller sample) and the CPU model string."""
    if edm:
        v, note, cores, dt = _oracle_edm_sample(8191)
        res = {"value": v, "unit": "cells/s", "cores": cores, "kind": "oracle", "sample": note, "seconds": dt}
        one = _oracle_single_thread("edm", None, True, 4095)
    else:
        ca = isinstance(wl, inputs.CAWorkload)
        v, note, cores, dt = _oracle_sample(wl, 2 if ca else 5)
        res = {"value": v, "unit": UNIT if ca else "cells/s", "cores": cores,
               "kind": "oracle", "sample": note, "seconds": dt}
        one = _oracle_single_thread(workload, n, False, 1) if workload else {"error": "no workload name"}
    res["cpu_model"] = _cpu_model()
    res["single_thread"] = one if "error" in one else {"value": one["value"], "unit": res["unit"], "cores": 1,
                                                       "sample": one["sample"], "seconds": one["seconds"]}
    return res


def run_reference(args, rank, world):
    if rank != 0:
        return None
    wl = _workload(args.workload, args)
    if wl in ("batch", "serve") or args.workload in ("map2", "map3"):
        return {"impl": "reference", "unavailable": f"the oracle arm times the single-instance workloads "
                f"(ca2, ca3, write2, write2hbm, write4, accum2, accum3, edm), not {args.workload}"}
    unit = UNIT if isinstance(wl, inputs.CAWorkload) else "cells/s"
    if args.workload == "edm":
        sample = lambda k: _oracle_edm_sample(8191)  # noqa: E731
    else:
        sample = lambda k: _oracle_sample(wl, k)  # noqa: E731
    for _ in range(args.warmup):
        sample(1)
    vals, dts = [], []
    cores, note = 1, ""
    for _ in range(args.steps):
        v, note, cores, dt = sample(1)
        vals.append(v)
        dts.append(dt)
    total = sum(dts)
    value = len(vals) / sum(1.0 / v for v in vals)  # units over total time
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": unit, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / len(dts) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.workload == "edm" else ("u8" if unit == UNIT else "u32"),
            "data": "synthetic", "config": {"workload": wl.name, "m": wl.m, "n": wl.n},
            "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle",
                             "sample": f"each step: {note}"},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ca2",
                    choices=["ca2", "ca3", "write2", "write2hbm", "write4", "accum2", "accum3", "map2", "map3", "edm", "batch",
                             "serve"])
    ap.add_argument("--serve-seconds", type=float, default=inputs.SERVE_SECONDS, help="serve: trace length")
    ap.add_argument("--serve-sample", type=int, default=400, help="serve: jobs re-run alone for the serial baseline")
    ap.add_argument("--serve-capacity-jobs", type=int, default=4000, help="serve: jobs of the offline capacity run")
    ap.add_argument("--serve-high-rate", type=float, default=8000.0, help="serve: arrival rate of the heavy-load run")
    ap.add_argument("--serve-high-seconds", type=float, default=5.0, help="serve: length of the heavy-load run")
    ap.add_argument("--round-steps", type=int, default=0, help="serve: automaton steps per batched round (0: the default, 16)")
    ap.add_argument("--max-inflight", type=int, default=2, help="serve: rounds the host may queue ahead of the GPU")
    ap.add_argument("--direct-jobs", type=int, default=0,
                    help="serve: rounds with at most this many resident jobs launch each job's steps directly "
                         "(0: the default, 24; -1: never)")
    ap.add_argument("--no-tune", action="store_true", help="batch: untuned tile choices")
    ap.add_argument("--tune-cache", default=None,
                    help="batch: JSON file of tuned tile choices, read if it exists, else written after tuning")
    ap.add_argument("--no-loop", action="store_true", help="batch: skip the single-instance loop baseline")
    ap.add_argument("--batch-m2", type=int, default=2048, help="batch: number of m = 2 instances")
    ap.add_argument("--batch-m3", type=int, default=256, help="batch: number of m = 3 instances")
    ap.add_argument("--batch-nmin", type=int, default=None, help="batch: keep only the instances with n >= this")
    ap.add_argument("--batch-nmax", type=int, default=None, help="batch: keep only the instances with n <= this")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-bb", action="store_true", help="skip the bounding-box comparison")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-buffer run")
    ap.add_argument("--no-energy", action="store_true", help="skip the NVML energy runs")
    ap.add_argument("--no-records", action="store_true",
                    help="ca2: leave out the short batched and serving records of the default line")
    ap.add_argument("--n", type=int, default=None, help="override n (smaller case of the workload)")
    ap.add_argument("--block", type=int, default=None, help="override the tile side")
    ap.add_argument("--side", type=int, default=None,
                    help="automaton: padded array side (cells per row, a multiple of 16; default n + 1 rounded up)")
    ap.add_argument("--band", type=int, default=None, help="m = 2: trapezoid band height (-1: single H2 grid)")
    ap.add_argument("--r-inv", type=int, default=2, choices=[2, 3],
                    help="write, ACCUM, MAP, EDM with m = 2: scale factor 1/r of the map (3: the r = 1/3, beta = 3 map)")
    ap.add_argument("--launch", type=int, default=0,
                    help="automaton step form: 0 auto (m = 3: the plane stream), 1 grid, 2 x-stream, "
                         "3 plane stream (m = 3)")
    ap.add_argument("--ca-steps", type=int, default=None, help="override automaton steps per bench step")
    ap.add_argument("--layout", type=int, default=0,
                    help="m = 3 H3 layout: 0 packed grid (Sec. 4.3), 1 one block range per stack level")
    args = ap.parse_args()
    global _ENERGY
    _ENERGY = not args.no_energy
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    rank, world, local = _dist_init()
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    else:
        res = run_ours(args, rank, world, local)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
