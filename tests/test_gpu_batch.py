"""GPU parity of the batched engine: every instance of a mixed batch equals
the oracle (and the single-instance path) bit for bit."""
import numpy as np
import pytest
import torch

import oracle
from paper_2208_11617_gb300 import autotune, inputs
from paper_2208_11617_gb300 import simplex as sx

pytestmark = pytest.mark.gpu


def _inst(m, n, block, beta=2, band=0, rule=None, seed=0, p=0.5):
    rule = rule or (inputs.B3S23 if m == 2 else inputs.B5S45)
    return dict(m=m, n=n, block=block, beta=beta, band=band, birth=rule[0], survive=rule[1], seed=seed,
                threshold=inputs.bernoulli_threshold(p))


MIXED = [
    _inst(2, 0, 64, seed=1), _inst(2, 17, 64, seed=2), _inst(2, 100, 64, seed=3), _inst(2, 255, 128, seed=4),
    _inst(2, 1000, 64, seed=5), _inst(2, 1000, 128, band=4, seed=6),
    _inst(2, 300, 64, rule=(1 << 3 | 1 << 6, 1 << 2 | 1 << 3), seed=7, p=0.4),
    _inst(2, 200, 128, rule=(1, 0), seed=8, p=0.3),
    _inst(3, 0, 16, seed=9), _inst(3, 20, 16, seed=10, p=0.3), _inst(3, 63, 16, seed=11, p=0.3),
    _inst(3, 100, 16, beta=3, seed=12, p=0.3), _inst(3, 150, 16, rule=(1 << 4, 1 << 2 | 1 << 3 | 1 << 4), seed=13),
    _inst(2, 4095, 128, seed=14), _inst(3, 255, 16, seed=15, p=0.3),
    _inst(3, 0, 32, seed=16), _inst(3, 31, 32, seed=17, p=0.3), _inst(3, 100, 32, beta=3, seed=18, p=0.3),
    _inst(3, 200, 32, seed=19, p=0.3), _inst(3, 150, 32, rule=(1 << 4, 1 << 2 | 1 << 3 | 1 << 4), seed=20),
    # plane-stream instances (block 128): a launch of their own per step
    _inst(3, 0, 128, seed=24), _inst(3, 1, 128, seed=25), _inst(3, 64, 128, seed=26, p=0.3),
    _inst(3, 200, 128, seed=27, p=0.3), _inst(3, 150, 128, rule=(1 << 4, 1 << 2 | 1 << 3 | 1 << 4), seed=28),
    _inst(3, 255, 128, beta=3, seed=29, p=0.3), _inst(3, 300, 128, seed=30, p=0.3),
]

ONLY32 = [_inst(3, 64, 32, seed=21, p=0.3), _inst(3, 255, 32, seed=22, p=0.3), _inst(3, 17, 32, seed=23)]
ONLYPLANE = [_inst(3, 64, 128, seed=31, p=0.3), _inst(3, 255, 128, seed=32, p=0.3), _inst(3, 17, 128, seed=33),
             _inst(3, 500, 128, seed=34, p=0.3), _inst(3, 2, 128, rule=(1, 0), seed=35, p=0.3)]


def _batch_side(d):
    """The batch's grid side: whole 128-byte rows, round_up(n + 1, 128)."""
    return (d["n"] + 128) // 128 * 128


def _logical(t, n):
    return t[tuple(slice(0, n + 1) for _ in range(t.dim()))].cpu().numpy()


@pytest.mark.parametrize("use_graph", [True, False])
def test_mixed_batch_matches_oracle(use_graph):
    b = sx.simplex_batch_create(MIXED)
    sx.simplex_batch_bind(b)
    sx.simplex_batch_init(b)
    refs = [oracle.ca_init(d["m"], d["n"], d["seed"], d["threshold"]) for d in MIXED]
    for steps in (5, 3):                    # two runs: parity 0 then parity 1
        live = torch.zeros(len(MIXED) * (steps + 1), dtype=torch.int64, device="cuda")
        sx.simplex_batch_run(b, steps, live, use_graph)
        torch.cuda.synchronize()
        live = live.view(len(MIXED), steps + 1).cpu().numpy().astype(np.uint64)
        for i, d in enumerate(MIXED):
            ref, ref_live = oracle.ca_run(d["m"], d["n"], steps, d["birth"], d["survive"], refs[i])
            g = sx.simplex_batch_grid(b, i, d["m"])
            np.testing.assert_array_equal(_logical(g, d["n"]), ref, err_msg=f"instance {i}")
            np.testing.assert_array_equal(live[i], ref_live, err_msg=f"instance {i} live")
            refs[i] = ref
    assert sx.simplex_device_status() == 0


@pytest.mark.parametrize("insts", [ONLY32, ONLYPLANE], ids=["32cubed", "plane"])
def test_batch_of_one_launch_set_matches_oracle(insts):
    """A batch whose every instance runs in the second launch set (32^3 tiles),
    or in the plane-stream launch (m = 3, block 128)."""
    ONLY32 = insts
    b = sx.simplex_batch_create(ONLY32)
    sx.simplex_batch_bind(b)
    sx.simplex_batch_init(b)
    steps = 4
    live = torch.zeros(len(ONLY32) * (steps + 1), dtype=torch.int64, device="cuda")
    sx.simplex_batch_run(b, steps, live)
    torch.cuda.synchronize()
    live = live.view(len(ONLY32), steps + 1).cpu().numpy().astype(np.uint64)
    for i, d in enumerate(ONLY32):
        ref, ref_live = oracle.ca_run(d["m"], d["n"], steps, d["birth"], d["survive"],
                                      oracle.ca_init(d["m"], d["n"], d["seed"], d["threshold"]))
        np.testing.assert_array_equal(_logical(sx.simplex_batch_grid(b, i, d["m"]), d["n"]), ref)
        np.testing.assert_array_equal(live[i], ref_live)
    assert sx.simplex_device_status() == 0


def test_batch_workload_equals_single_instance_path():
    """The batched workload (2048 + 256 instances, 16 steps): every instance's
    final grid and live counts equal simplex_ca_run on that instance alone."""
    insts = autotune.apply(inputs.batch_instances())
    steps = inputs.BATCH_STEPS
    b = sx.simplex_batch_create(insts)
    sx.simplex_batch_bind(b)
    sx.simplex_batch_init(b)
    live = torch.zeros(len(insts) * (steps + 1), dtype=torch.int64, device="cuda")
    sx.simplex_batch_run(b, steps, live)
    torch.cuda.synchronize()
    live = live.view(len(insts), steps + 1)
    rng = np.random.default_rng(5)
    oracle_check = set(rng.choice(len(insts), size=12, replace=False).tolist())
    for i, d in enumerate(insts):
        side = _batch_side(d)
        mp = sx.simplex_map_create(d["m"], d["n"], 2, d["beta"], 32 if d["m"] == 3 else d["block"], side=side)
        a = torch.zeros(mp.numel, dtype=torch.uint8, device="cuda")
        bb = torch.zeros_like(a)
        sx.simplex_ca_init(mp, a, d["seed"], d["threshold"])
        l1 = torch.zeros(steps + 1, dtype=torch.int64, device="cuda")
        fin = sx.simplex_ca_run(mp, a, bb, steps, d["birth"], d["survive"], l1, False)
        g = sx.simplex_batch_grid(b, i, d["m"])
        assert torch.equal(g.reshape(-1), fin), f"instance {i}"
        assert torch.equal(live[i], l1), f"instance {i} live"
        if i in oracle_check and d["n"] <= 600:
            ref, ref_live = oracle.ca_run(d["m"], d["n"], steps, d["birth"], d["survive"],
                                          oracle.ca_init(d["m"], d["n"], d["seed"], d["threshold"]))
            np.testing.assert_array_equal(_logical(g, d["n"]), ref)
    assert sx.simplex_device_status() == 0
