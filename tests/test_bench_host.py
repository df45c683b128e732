"""The bench's host-side bookkeeping: the clock summary taken from
nvidia-smi rows (median SM clock under load, the highest maximum clock, the
throttle reasons seen as Active) and the DRAM traffic read from the
committed ncu summary (scaled to the launch's units, and withheld once the
kernel's sources differ from the captured ones)."""
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_host_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _row(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return ["0", str(sm), str(mx), "900.5", "0x0", hw, hwt, swt, cap]


def test_clock_summary(bench):
    c = bench.ClockSampler()
    assert c.summary()["reasons"] == ["no nvidia-smi samples"]
    c.rows = [_row(2070, 2070), _row(1900, 2070, cap="Active"), _row(2070, 2070), _row("[N/A]", "[N/A]"),
              ["garbage"]]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 5
    c.rows = [_row(1500, 2070, hw="Active"), _row(1400, 2070, hwt="Active", swt="Active"), _row(1600, 2070)]
    s = c.summary()
    assert s["sm_mhz"] == 1500.0
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_ncu_traffic_scales_and_goes_stale(bench, tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "ncu_traffic.json").write_text(json.dumps(
        {"k_trace": {"kernel_sources": "abc", "dram_bytes_per_unit": 75.0, "unit": "segment"}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_sources_hash", lambda k: "abc")
    assert bench.ncu_traffic("k_trace", 1000.0) == 75000.0
    assert bench.ncu_traffic("k_shade", 1000.0) is None  # never captured
    monkeypatch.setattr(bench, "kernel_sources_hash", lambda k: "changed")
    assert bench.ncu_traffic("k_trace", 1000.0) is None
    (prof / "ncu_traffic.json").write_text("{not json")
    assert bench.ncu_traffic("k_trace", 1000.0) is None


def test_kernel_sources_hash_follows_the_kernel_files(bench):
    h = bench.kernel_sources_hash("k_trace")
    assert h == bench.kernel_sources_hash("k_shade")  # the same translation unit
    assert len(h) == 16 and h != bench.kernel_sources_hash("k_adjoint")
