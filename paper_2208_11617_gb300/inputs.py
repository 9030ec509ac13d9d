"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds workload definitions only -- sizes, seeds, rule masks and
Bernoulli thresholds -- and none of the method's arithmetic.  Both the CUDA path
and the CPU oracle receive these numbers as plain arguments.

The paper measures on synthetic n-sweeps (Sec. 5.1, Table 1) and publishes no
dataset; the workloads below are the same shapes: dense n^m arrays holding the
discrete orthogonal m-simplex x_1 + ... + x_m <= n.
"""
from __future__ import annotations

from dataclasses import dataclass
from fractions import Fraction

DEFAULT_SEED = 0x22081161

# Automaton rules as (birth, survive) bit masks: bit k = "k live neighbours".
B3S23 = (1 << 3, (1 << 2) | (1 << 3))          # Conway's Life, Moore-8 (m = 2)
B5S45 = (1 << 5, (1 << 4) | (1 << 5))          # Moore-26 rule used for m = 3


def bernoulli_threshold(p) -> int:
    """floor(p * 2^32) computed exactly from the decimal value of p (0 <= p < 1)."""
    q = Fraction(str(p))
    if not (0 <= q < 1):
        raise ValueError("p must be in [0, 1)")
    return int(q * (1 << 32))


@dataclass(frozen=True)
class WriteWorkload:
    name: str
    m: int
    n: int
    block: int
    seed: int = DEFAULT_SEED


@dataclass(frozen=True)
class CAWorkload:
    name: str
    m: int
    n: int
    block: int
    steps: int
    p: float
    rule: tuple
    seed: int = DEFAULT_SEED

    @property
    def threshold(self) -> int:
        return bernoulli_threshold(self.p)


# Write test on the 2-simplex: n = 1023 (524,800 cells) in a 1024^2 uint32 array,
# 16 x 16 tiles.
WRITE_M2 = WriteWorkload("write m=2 n=1023 rho=16", m=2, n=1023, block=16)
# Write test on the 2-simplex at a size past the L2: n = 32767 (536,887,296
# cells, 2.1 GB of stores) in a 32768^2 uint32 array (4 GiB), 128 x 128 tiles.
WRITE_M2_HBM = WriteWorkload("write m=2 n=32767 rho=128", m=2, n=32767, block=128)
# Write test on the 4-simplex: n = 127 (11,716,640 cells) in a 128^4 uint32 array,
# 8^4 tiles.
WRITE_M4 = WriteWorkload("write m=4 n=127 rho=8", m=4, n=127, block=8)
# ACCUM test (Table 1, read-add-write of one uint32 per cell) at sizes well
# past the L2: the 2-simplex n = 16383 (134,225,920 cells, 16384^2 array) in
# 64 x 64 tiles and the 3-simplex n = 1023 (179,481,600 cells, 1024^3 array)
# in 16^3 tiles.
ACCUM_M2 = WriteWorkload("accum m=2 n=16383 rho=64", m=2, n=16383, block=64)
ACCUM_M3 = WriteWorkload("accum m=3 n=1023 rho=16", m=3, n=1023, block=16)
# Automaton on the 2-simplex: n = 32767 in a 32768^2 uint8 array, Bernoulli(0.5),
# B3/S23, 100 steps; the same run at n = 4095 is the size the oracle finishes in
# seconds.
CA_M2 = CAWorkload("ca m=2 n=32767 B3/S23", m=2, n=32767, block=128, steps=100,
                   p=0.5, rule=B3S23)
CA_M2_SMALL = CAWorkload("ca m=2 n=4095 B3/S23", m=2, n=4095, block=128, steps=100,
                         p=0.5, rule=B3S23)
# Automaton on the 3-simplex: n = 1023 in a 1024^3 uint8 array, Bernoulli(0.3),
# B5/S45, 50 steps.
CA_M3 = CAWorkload("ca m=3 n=1023 B5/S45", m=3, n=1023, block=32, steps=50,
                   p=0.3, rule=B5S45)


# Batched workload: 2048 automata on 2-simplices with n log-uniform in
# [64, 2048] and 256 on 3-simplices with n log-uniform in [32, 256], each
# Bernoulli(0.4) seeded by its index, B3/S23 (m = 2) or B5/S45 (m = 3), 16 steps.
BATCH_STEPS = 16


def log_uniform_sizes(rng, count: int, lo: int, hi: int):
    """n = floor(exp(U(ln lo, ln hi))), drawn from a numpy Generator."""
    import numpy as np
    return np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))).astype(np.int64)


def batch_instances(seed: int = 1, n2: int = 2048, n3: int = 256, p: float = 0.4):
    """The batched workload as a list of dicts (m, n, rule, seed, threshold);
    tile sizes are left to the caller (autotuner or defaults)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    sizes2 = log_uniform_sizes(rng, n2, 64, 2048)
    sizes3 = log_uniform_sizes(rng, n3, 32, 256)
    thr = bernoulli_threshold(p)
    out = []
    for i, n in enumerate(sizes2):
        out.append(dict(m=2, n=int(n), birth=B3S23[0], survive=B3S23[1], seed=i, threshold=thr))
    for j, n in enumerate(sizes3):
        out.append(dict(m=3, n=int(n), birth=B5S45[0], survive=B5S45[1], seed=n2 + j, threshold=thr))
    return out


# Serving workload: Poisson arrivals at 2000 jobs/s for 60 s; each job is an
# automaton on a 2-simplex (80 %, n log-uniform in [128, 8192], B3/S23) or a
# 3-simplex (20 %, n log-uniform in [32, 512], B5/S45), steps uniform in
# 1..64, Bernoulli(0.5) seeded by the job's index; 64 GiB grid budget.
SERVE_RATE = 2000.0
SERVE_SECONDS = 60.0
SERVE_BUDGET = 64 << 30


def serve_trace(rate: float = SERVE_RATE, seconds: float = SERVE_SECONDS, seed: int = 2,
                n2=(128, 8192), n3=(32, 512), max_steps: int = 64, p: float = 0.5):
    """(jobs, arrival times in seconds) of the serving workload."""
    import numpy as np
    rng = np.random.default_rng(seed)
    arr_rng = np.random.default_rng(seed + 1)
    gaps = arr_rng.exponential(1.0 / rate, size=int(rate * seconds * 1.2) + 16)
    t = np.cumsum(gaps)
    t = t[t < seconds]
    count = len(t)
    is3 = rng.random(count) < 0.2
    sizes2 = log_uniform_sizes(rng, count, *n2)
    sizes3 = log_uniform_sizes(rng, count, *n3)
    steps = rng.integers(1, max_steps + 1, size=count)
    thr = bernoulli_threshold(p)
    jobs = []
    for i in range(count):
        m = 3 if is3[i] else 2
        rule = B5S45 if m == 3 else B3S23
        jobs.append(dict(m=m, n=int(sizes3[i] if m == 3 else sizes2[i]), steps=int(steps[i]), birth=rule[0],
                         survive=rule[1], seed=i, threshold=thr))
    return jobs, t


# Diagnostics of Table 1.  MAP: the map alone, 16 x 16 threads per block on
# the 2-simplex n = 32767 and 8 x 8 x 8 on the 3-simplex n = 1023 (the block
# sizes the paper found fastest).  EDM: the distance matrix of 32768 points in
# 3-D (coordinates uniform in [0, 1), float32) on the 2-simplex n = 32767,
# 32 x 32 tiles.
MAP_M2 = WriteWorkload("map m=2 n=32767 rho=16", m=2, n=32767, block=16)
MAP_M3 = WriteWorkload("map m=3 n=1023 rho=8", m=3, n=1023, block=8)
EDM_N = 32767
EDM_DIM = 3
EDM_BLOCK = 32


def edm_points(n: int, dim: int = EDM_DIM, seed: int = DEFAULT_SEED):
    """(n + 1) x dim float32 points, uniform in [0, 1), from numpy's seeded generator."""
    import numpy as np
    return np.random.default_rng(seed).random((n + 1, dim), dtype=np.float32)
