"""The autotuner's search and cache on the host alone: the step timer is
replaced by a cost function of the library's current knob settings (set and
read through the C ABI, which needs no GPU), so the search logic is checked
without timing anything.  Coordinate descent reaches the optimum of a
separable cost with one trial per option; the full sweep reaches the optimum
of a coupled one; results are cached per device and key, reused without
timing, and re-tuned on request; the fastest setting is left set."""
import json

import pytest
import torch

import paper_2603_00413_gb300 as dt
from paper_2603_00413_gb300 import autotune


@pytest.fixture(autouse=True)
def _restore_tuning(monkeypatch):
    from paper_2603_00413_gb300 import build
    build.build()
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "test-device")
    saved = dt.get_tuning()
    yield
    dt.set_tuning(**saved)


SPACE = {"trace_steps": (32, 64, 128, 192), "trace_refill": (4, 8, 16), "shade_blocks_per_sm": (4, 8, 16)}
BEST = {"trace_steps": 128, "trace_refill": 4, "shade_blocks_per_sm": 16}


def _separable(**_):
    t = dt.get_tuning()
    return 1.0 + sum(abs(SPACE[k].index(t[k]) - SPACE[k].index(BEST[k])) for k in SPACE)


def _fake_time(cost, calls):
    def timer(step, reps):
        calls.append(dict(dt.get_tuning()))
        return cost()
    return timer


def test_coordinate_descent_finds_a_separable_optimum(monkeypatch, tmp_path):
    calls = []
    monkeypatch.setattr(autotune, "_time", _fake_time(_separable, calls))
    dt.set_tuning(trace_steps=32, trace_refill=16, shade_blocks_per_sm=4)
    res = autotune.tune(lambda: None, "sep", space=SPACE, cache_path=str(tmp_path / "c.json"))
    assert {k: res["tuning"][k] for k in SPACE} == BEST and res["ms"] == 1.0
    assert {k: dt.get_tuning()[k] for k in SPACE} == BEST
    # the starting point plus one trial per other option of each knob
    assert len(calls) == 1 + sum(len(v) - 1 for v in SPACE.values()) == len(res["trials"])


def test_full_sweep_finds_a_coupled_optimum(monkeypatch, tmp_path):
    space = {"trace_steps": (32, 64, 128), "trace_refill": (4, 8, 16)}

    def coupled():
        t = dt.get_tuning()
        # best only in the corner (32, 16); one knob at a time from (128, 4) cannot leave the start
        table = {(32, 16): 1.0, (128, 4): 2.0}
        return table.get((t["trace_steps"], t["trace_refill"]), 3.0)

    calls = []
    monkeypatch.setattr(autotune, "_time", _fake_time(coupled, calls))
    dt.set_tuning(trace_steps=128, trace_refill=4)
    res = autotune.tune(lambda: None, "cpl", space=space, cache_path=str(tmp_path / "a.json"), coordinate=True)
    assert (res["tuning"]["trace_steps"], res["tuning"]["trace_refill"]) == (128, 4)
    dt.set_tuning(trace_steps=128, trace_refill=4)
    res = autotune.tune(lambda: None, "cpl", space=space, cache_path=str(tmp_path / "b.json"), coordinate=False)
    assert (res["tuning"]["trace_steps"], res["tuning"]["trace_refill"]) == (32, 16) and res["ms"] == 1.0
    assert len(res["trials"]) == 1 + 9


def test_results_are_cached_per_device_and_key(monkeypatch, tmp_path):
    path = str(tmp_path / "cache.json")
    calls = []
    monkeypatch.setattr(autotune, "_time", _fake_time(_separable, calls))
    dt.set_tuning(trace_steps=32, trace_refill=16, shade_blocks_per_sm=4)
    first = autotune.tune(lambda: None, "k1", space=SPACE, cache_path=path)
    n = len(calls)
    stored = json.load(open(path))
    assert list(stored) == ["test-device|k1"] and stored["test-device|k1"]["tuning"] == first["tuning"]
    # a cached key is set without timing anything
    dt.set_tuning(trace_steps=32, trace_refill=16, shade_blocks_per_sm=4)
    again = autotune.tune(lambda: None, "k1", space=SPACE, cache_path=path)
    assert len(calls) == n and again["tuning"] == first["tuning"]
    assert {k: dt.get_tuning()[k] for k in SPACE} == BEST
    # another key, or retune, runs the search again and both keys stay cached
    autotune.tune(lambda: None, "k2", space=SPACE, cache_path=path)
    assert len(calls) > n
    m = len(calls)
    autotune.tune(lambda: None, "k1", space=SPACE, cache_path=path, retune=True)
    assert len(calls) > m
    assert sorted(json.load(open(path))) == ["test-device|k1", "test-device|k2"]
