"""Host logic of the batched engine's tuner: size classes, the untuned
defaults, applying a tuned table and reading a cached one (no GPU work)."""
import json

import pytest

from paper_2208_11617_gb300 import autotune


@pytest.mark.parametrize("m,n,cls", [(2, 64, (2, 6)), (2, 127, (2, 6)), (2, 128, (2, 7)), (2, 2047, (2, 10)),
                                     (3, 32, (3, 5)), (3, 255, (3, 7)), (3, 256, (3, 8)), (2, 1, (2, 0)),
                                     (2, 0, (2, 0))])
def test_size_class_is_m_and_floor_log2_n(m, n, cls):
    assert autotune.size_class(m, n) == cls


def test_default_config():
    assert autotune.default_config(2, 1023) == dict(block=64, beta=2)
    assert autotune.default_config(2, 1024) == dict(block=128, beta=2)
    assert autotune.default_config(3, 255) == dict(block=16, beta=2)


def test_candidates_are_buildable_choices():
    # m = 2: H2 tiles of 64 or 128 cells; m = 3: 16^3 / 32^3 tiles with beta 2
    # or 3, or block 128 (the plane stream)
    assert {c["block"] for c in autotune.CANDIDATES[2]} == {64, 128}
    assert all(c["beta"] == 2 for c in autotune.CANDIDATES[2])
    assert {(c["block"], c["beta"]) for c in autotune.CANDIDATES[3]} == {(16, 2), (16, 3), (32, 2), (32, 3), (128, 2)}


def test_apply_takes_the_table_else_the_defaults_and_copies():
    insts = [dict(m=2, n=1500, seed=1), dict(m=2, n=100, seed=2), dict(m=3, n=200, seed=3), dict(m=3, n=40, seed=4)]
    table = {(2, 10): dict(block=64, beta=2, rate=1.0), (3, 7): dict(block=128, beta=2, band=0, rate=2.0)}
    out = autotune.apply(insts, table)
    assert [(d["block"], d["beta"], d["band"]) for d in out] == [(64, 2, 0), (64, 2, 0), (128, 2, 0), (16, 2, 0)]
    assert [d["seed"] for d in out] == [1, 2, 3, 4]
    assert all("block" not in d for d in insts)          # the caller's dicts are left alone
    assert [d["block"] for d in autotune.apply(insts)] == [128, 64, 16, 16]


def test_tune_reads_a_cached_table(tmp_path):
    cache = tmp_path / "tune.json"
    raw = {json.dumps([2, 10]): dict(block=128, beta=2, rate=3.5), json.dumps([3, 7]): dict(block=128, beta=2, rate=1.5)}
    cache.write_text(json.dumps(raw))
    table = autotune.tune([dict(m=2, n=1500), dict(m=3, n=200)], cache=str(cache))
    assert table == {(2, 10): raw[json.dumps([2, 10])], (3, 7): raw[json.dumps([3, 7])]}
    out = autotune.apply([dict(m=3, n=200)], table)
    assert out[0]["block"] == 128
