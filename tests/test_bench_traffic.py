"""The recorded DRAM traffic in bench.py belongs to the kernels as committed.

bench.py reports a kernel's ncu traffic only while the fingerprint of its
sources (the code without comments) equals the one the traffic was captured
with.  These tests keep the table and the profiles that quote it in step with
the sources: a kernel change must come with a new capture.
"""
import math
import os
import re

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# profile file prefix -> kernel name in bench._KERNEL_SOURCES
PROFILE_KERNELS = {
    "ca2_step_kernel_m2_": "ca2_step_kernel<128>",
    "ca3_step_kernel_m3_": "ca3_step_kernel<32>",
    "ca3_step_stream_m3_": "ca3_step_stream",
    "ca3_step_planes_m3_": "ca3_step_planes",
    "write_kernel_m2_": "write_kernel<2>",
}

# bytes per domain cell of one launch: automaton steps read and write one
# uint8 each, the write test stores one uint32
BYTES_PER_CELL = {"ca2_step_kernel<128>": (2, 2), "ca3_step_kernel<32>": (3, 2), "ca3_step_stream": (3, 2),
                  "ca3_step_planes": (3, 2), "write_kernel<2>": (2, 4)}


@pytest.mark.parametrize("key", sorted(bench._KERNEL_TRAFFIC), ids=lambda k: f"{k[1]}-n{k[2]}")
def test_traffic_entry_matches_current_sources(key):
    fp, kname, n, block = key
    assert kname in bench._KERNEL_SOURCES
    assert bench._kernel_fingerprint(kname) == fp, f"{kname}: sources changed since its traffic was captured"


@pytest.mark.parametrize("key", sorted(bench._KERNEL_TRAFFIC), ids=lambda k: f"{k[1]}-n{k[2]}")
def test_traffic_entry_is_near_the_algorithmic_bytes(key):
    _, kname, n, _ = key
    m, width = BYTES_PER_CELL[kname]
    alg = width * math.comb(n + m, m)
    ratio = bench._KERNEL_TRAFFIC[key] / alg
    # below 1: the last writes of a launch still sit in L2; far above: re-reads
    assert 0.9 < ratio < 1.6, (kname, ratio)


def test_profiles_quote_the_current_fingerprints():
    pdir = os.path.join(ROOT, "profiles")
    seen = 0
    for name in sorted(os.listdir(pdir)):
        kname = next((k for p, k in PROFILE_KERNELS.items() if name.startswith(p)), None)
        if kname is None:
            continue
        with open(os.path.join(pdir, name), encoding="utf-8") as f:
            m = re.search(r"fingerprint[^:\n]*:\s*([0-9a-f]{16})", f.read())
        assert m, f"{name} quotes no kernel source fingerprint"
        assert m.group(1) == bench._kernel_fingerprint(kname), f"{name}: fingerprint of other sources"
        seen += 1
    assert seen == len(PROFILE_KERNELS)
