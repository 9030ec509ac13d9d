"""bench.py's reference arm (the oracle timed on the host cores) on CPU: one
JSON line with the contract's keys, alone and under torchrun with two ranks
(gloo), where rank 0 alone prints."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _lines(cmd):
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    return [json.loads(ln) for ln in r.stdout.splitlines() if ln.startswith("{")]


def _check(line, workload, n_gpus):
    assert line["impl"] == "reference" and line["n_gpus"] == n_gpus
    assert line["value"] > 0 and line["unit"] == "cells/s" and line["higher_is_better"] is True
    assert line["config"]["workload"] == workload
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_single_process():
    out = _lines([sys.executable, "bench.py", "--impl", "reference", "--workload", "write2", "--steps", "2",
                  "--warmup", "1"])
    assert len(out) == 1
    _check(out[0], "write m=2 n=1023 rho=16", 1)


def test_reference_arm_two_ranks_rank0_prints_once():
    out = _lines([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                  "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl",
                  "reference", "--gpus", "2", "--workload", "write2", "--steps", "1", "--warmup", "0"])
    assert len(out) == 1
    _check(out[0], "write m=2 n=1023 rho=16", 2)


def test_reference_arm_names_the_workloads_it_does_not_time():
    out = _lines([sys.executable, "bench.py", "--impl", "reference", "--workload", "serve", "--steps", "1"])
    assert len(out) == 1 and out[0]["impl"] == "reference" and "unavailable" in out[0]
