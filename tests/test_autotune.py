"""The autotuner's host logic on the CPU: coordinate descent finds the fastest value of each
tunable against a fake step whose time depends on the settings, keeps the old value when nothing
is faster, and its cache stores and re-applies the choice per GPU and workload signature (and
ignores unknown names). Only sg_tune_set / sg_tune_get are called: no GPU work."""
import json

import pytest

import paper_2010_10055_gb300 as sg
from paper_2010_10055_gb300 import autotune


@pytest.fixture
def restore_tunables():
    saved = sg.tunables()
    yield
    for k, v in saved.items():
        sg.tune(k, v)


def fake_timer(cost):
    calls = []

    def timer(step, reps):
        step()
        calls.append(dict(sg.tunables()))
        return cost(sg.tunables())

    return timer, calls


def test_descent_picks_the_fastest_value_per_tunable(restore_tunables):
    sg.tune("bloom_bits", 8)
    sg.tune("spgemm_blocks_per_sm", 16)
    # bloom_bits best at 10, blocks best at 4; independent costs
    cost = lambda t: abs(t["bloom_bits"] - 10) * 1.0 + abs(t["spgemm_blocks_per_sm"] - 4) * 0.5 + 3.0
    timer, calls = fake_timer(cost)
    space = {"bloom_bits": [6, 8, 10, 12], "spgemm_blocks_per_sm": [2, 4, 8, 16]}
    steps = []
    res = autotune.autotune(lambda: steps.append(1), space=space, timer=timer)
    assert res["params"]["bloom_bits"] == 10
    assert res["params"]["spgemm_blocks_per_sm"] == 4
    assert sg.tunables()["bloom_bits"] == 10 and sg.tunables()["spgemm_blocks_per_sm"] == 4
    assert res["ms"] == pytest.approx(3.0)
    # one baseline timing + every candidate except the current value of each tunable
    assert res["trials"] == 1 + 3 + 3 == len(calls) == len(steps)


def test_descent_keeps_current_value_when_nothing_is_faster(restore_tunables):
    sg.tune("tr_blocks_per_sm", 32)
    timer, _ = fake_timer(lambda t: 1.0 if t["tr_blocks_per_sm"] == 32 else 2.0)
    res = autotune.autotune(lambda: None, space={"tr_blocks_per_sm": [4, 8, 16, 32]}, timer=timer)
    assert res["params"]["tr_blocks_per_sm"] == 32 and res["ms"] == 1.0


def test_cache_store_load_per_device_and_signature(tmp_path, restore_tunables):
    path = str(tmp_path / "cache.json")
    sg.tune("bloom_bits", 12)
    autotune.store(path, "wl-a", {"params": {"bloom_bits": 12, "no_such_tunable": 5}, "ms": 1.0}, device="GPU-X|152")
    sg.tune("bloom_bits", 8)
    assert not autotune.load(path, "wl-a", device="GPU-Y|152")   # other GPU
    assert not autotune.load(path, "wl-b", device="GPU-X|152")   # other workload
    assert sg.tunables()["bloom_bits"] == 8
    assert autotune.load(path, "wl-a", device="GPU-X|152")
    assert sg.tunables()["bloom_bits"] == 12
    data = json.load(open(path))
    assert list(data) == ["GPU-X|152|wl-a"]
    assert not autotune.load(str(tmp_path / "missing.json"), "wl-a", device="GPU-X|152")


def test_cache_skips_out_of_range_values(tmp_path, restore_tunables):
    path = str(tmp_path / "cache.json")
    autotune.store(path, "wl", {"params": {"bloom_bits": 1000, "tr_blocks_per_sm": 8}, "ms": 1.0}, device="G|1")
    sg.tune("tr_blocks_per_sm", 32)
    assert autotune.load(path, "wl", device="G|1")
    assert sg.tunables()["tr_blocks_per_sm"] == 8
    assert sg.tunables()["bloom_bits"] != 1000
