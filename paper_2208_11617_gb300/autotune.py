"""Autotuner for the batched engine: picks the tile side and (r, beta) per
(m, n) size class by timing the candidates on the GPU.

Size class of an instance: (m, floor(log2 n)).  Candidates (r = 1/2 is the
only scale factor implemented):
  m = 2: tile 64 or 128 (H in trapezoid form, band chosen by the plan);
  m = 3: tile 16 or 32 with beta = 2 (H3 with the hinge) or beta = 3 (every
         corner recursed); 32^3 tiles run in a second launch per step; or
         block 128, the plane stream (bricks of 32 x 128 cells streamed along
         x1), in a launch of its own.
For each class the tuner builds a batch of that class's instances alone for
every candidate, runs a few graph-captured steps, and keeps the candidate with
the most cell-updates per second.  Results can be cached in a JSON file.
"""
from __future__ import annotations

import json
import math
import os
import time

CANDIDATES = {2: [dict(block=64, beta=2), dict(block=128, beta=2)],
              3: [dict(block=16, beta=2), dict(block=16, beta=3), dict(block=32, beta=2), dict(block=32, beta=3),
                  dict(block=128, beta=2)]}


def size_class(m: int, n: int):
    return (m, int(math.floor(math.log2(max(n, 1)))))


def default_config(m: int, n: int) -> dict:
    """Untuned choice: 128-cell tiles from n = 1024 up, else 64 (m = 2); 16^3, beta = 2 (m = 3)."""
    if m == 2:
        return dict(block=128 if n >= 1024 else 64, beta=2)
    return dict(block=16, beta=2)


def apply(instances, table=None):
    """Instances with block/beta filled from the tuned table (or the defaults)."""
    out = []
    for d in instances:
        cfg = (table or {}).get(size_class(d["m"], d["n"])) or default_config(d["m"], d["n"])
        e = dict(d)
        e.update(block=cfg["block"], beta=cfg["beta"], band=cfg.get("band", 0))
        out.append(e)
    return out


def _time_batch(sx, torch, insts, steps: int, reps: int) -> float:
    b = sx.simplex_batch_create(insts)
    sx.simplex_batch_bind(b)
    sx.simplex_batch_init(b)
    for _ in range(2):                      # capture + warm up
        sx.simplex_batch_run(b, steps)
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        sx.simplex_batch_run(b, steps)
    e.record()
    torch.cuda.synchronize()
    cells = sx.simplex_batch_info(b)["cells"]
    b.close()
    return cells * steps * reps / (s.elapsed_time(e) * 1e-3)


def tune(instances, steps: int = 16, reps: int = 3, max_per_class: int = 256, cache: str | None = None):
    """Returns {size class: config}; reads/writes `cache` (JSON) when given.  Each
    candidate runs `steps` steps per graph (the batched workload's 16: with fewer,
    a small class's fixed graph-launch cost decides the choice)."""
    import torch
    from . import simplex as sx
    if cache and os.path.exists(cache):
        with open(cache) as f:
            raw = json.load(f)
        return {tuple(json.loads(k)): v for k, v in raw.items()}
    classes = {}
    for d in instances:
        classes.setdefault(size_class(d["m"], d["n"]), []).append(d)
    table = {}
    t0 = time.perf_counter()
    for cls, members in sorted(classes.items()):
        members = members[:max_per_class]
        best, best_rate = None, -1.0
        for cand in CANDIDATES[cls[0]]:
            insts = [dict(d, block=cand["block"], beta=cand["beta"], band=0) for d in members]
            rate = _time_batch(sx, torch, insts, steps, reps)
            if rate > best_rate:
                best, best_rate = dict(cand, rate=rate), rate
        table[cls] = best
    table_meta = time.perf_counter() - t0
    if cache:
        os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
        with open(cache, "w") as f:
            json.dump({json.dumps(list(k)): v for k, v in table.items()}, f, indent=1)
    tune.last_seconds = table_meta
    return table


# ---------------------------------------------------------------------------
# The (r, beta) question of Thm. 3 (Sec. 6), on the host.
#
# A self-similar set S of orthotopes with scale factor r = 1/k and replication
# beta has volume (Eq. generic-m)
#     V(S_n^m) = (n^m - beta^(log_k n)) / (k^m - beta),
# against V(Delta) = C(n + m - 1, m) (the paper's side-length count).  Its
# extra volume tends to alpha = m! / (k^m - beta) - 1 (Lemma 5 gives it for
# k = beta = 2: 5/7 at m = 4, 3 at m = 5, 39 at m = 7).  Thm. 3 asks for the
# (k, beta) minimising |V(S) - V(Delta)| subject to beta > 1 and k, beta
# integers; a set can only cover the simplex if V(S) >= V(Delta).  The paper
# states the bound 1/r > beta, which its own r = 1/2, beta = 2 sets break, so
# the search uses beta < k^m (the series converges) and reports the paper's
# bound beside each candidate.  Volume alone does not say whether a set
# covers Delta geometrically: the maps built here are r = 1/2 with beta = 2
# (m = 2, 3) and beta = m (m = 3, 4), and their cover is checked block by
# block by the tests.

def set_volume(m: int, n: int, k: int, beta: int) -> float:
    """V(S_n^m) of Eq. generic-m for r = 1/k (n a power of k)."""
    levels = round(math.log(n, k))
    return (n ** m - beta ** levels) / (k ** m - beta)


def simplex_volume(m: int, n: int) -> int:
    """V(Delta_n^m) with n the side length, as Sec. 6 counts it: C(n + m - 1, m)."""
    return math.comb(n + m - 1, m)


def extra_volume_limit(m: int, k: int, beta: int) -> float:
    """alpha(S, Delta) as n -> infinity: m! / (k^m - beta) - 1 (Lemma 5 for k = beta = 2)."""
    return math.factorial(m) / (k ** m - beta) - 1.0


def search_r_beta(m: int, n: int, k_max: int = 8):
    """Candidates (k = 1/r, beta) of Thm. 3 for the m-simplex of side n (a
    power of k is not required: the volume formula is evaluated at n), sorted
    by |V(S) - V(Delta)|; each entry says whether V(S) >= V(Delta) at this n
    and whether the paper's bound 1/r > beta holds."""
    out = []
    vd = simplex_volume(m, n)
    for k in range(2, k_max + 1):
        for beta in range(2, k ** m):
            vs = (n ** m - beta ** math.log(n, k)) / (k ** m - beta)
            out.append(dict(k=k, beta=beta, volume=vs, extra=vs / vd - 1.0, covers_volume=vs >= vd,
                            paper_bound=k > beta, alpha=extra_volume_limit(m, k, beta)))
    out.sort(key=lambda c: abs(c["volume"] - vd))
    return out
