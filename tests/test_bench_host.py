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


def test_issue_roofline_from_the_committed_instruction_count(bench, tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "ncu_traffic.json").write_text(json.dumps(
        {"k_trace": {"kernel_sources": "abc", "dram_bytes_per_unit": 75.0, "inst_per_unit": 180.0,
                     "threads_per_inst": 16.0},
         "k_shade": {"kernel_sources": "abc", "dram_bytes_per_unit": 110.0}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_sources_hash", lambda k: "abc")
    assert bench.ncu_issue("k_trace") == (180.0, 16.0)
    assert bench.ncu_issue("k_shade") is None  # no instruction count captured
    r = bench.issue_roofline(180.0, 16.0, 1e7, 2.0, 152, 2000.0)
    assert r["peak"] == pytest.approx(1216.0) and r["achieved"] == pytest.approx(900.0)
    assert r["frac"] == pytest.approx(900.0 / 1216.0)
    monkeypatch.setattr(bench, "kernel_sources_hash", lambda k: "changed")
    assert bench.ncu_issue("k_trace") is None


def test_kernel_sources_hash_follows_the_kernel_files(bench):
    h = bench.kernel_sources_hash("k_trace")
    assert h == bench.kernel_sources_hash("k_shade")  # the same translation unit
    assert len(h) == 16 and h != bench.kernel_sources_hash("k_adjoint")


def test_summary_digest_keeps_every_workload_short(bench):
    """The digest printed last on the bench line: the headline numbers of each
    workload that ran, None-safe for workloads left out, and short enough for
    a log tail of 1500 characters to hold it whole."""
    rates = {str(r): {"batched": {"p50_ms": 3.0, "p99_ms": 12.0, "requests_per_s": float(r)},
                      "one_per_launch": {"p50_ms": 3.1, "p99_ms": 14.0, "requests_per_s": float(r)}}
             for r in (10, 30, 100, 300, 1000, 2000)}
    leg = {"ms_per_step": 50.9, "segments_per_s": 1.2e9, "rebuild_ms": 4.5}
    out = {"value": 3.27e9, "fwd_segments_per_s": 3.9e9, "ms_per_step": 37.35, "e2e": {"value": 3.28e9},
           "roofline": {"ms_per_launch": 2.8, "frac": 0.049, "l2": {"frac": 0.47}},
           "large": {"checkpoint": leg, "full": leg, "mesh_update": {"ms": 6.9, "optimisation_step_ms": 57.9}},
           "batch": {"batched_ms": 26.1, "graph_ms": 25.9, "plain_ms": 109.9, "graph_segments_per_s": 2.3e9},
           "c0": {"eager_ms_per_frame": 0.27, "graph_ms_per_frame": 0.245},
           "medium": {"sigma_only": {"ms_per_step": 37.2}, "hash_texture": {"ms_per_step": 461.0}, "clocks": None},
           "paper_loss": {"ms": 0.21}, "serve": {"rates": rates}}
    g = bench.summary_digest(out)
    assert g["fwd_bwd_gseg_s"] == 3.27 and g["e2e_gseg_s"] == 3.28
    assert g["large"]["ckpt_ms"] == 50.9 and g["batch"]["graph_ms"] == 25.9 and g["c0"]["graph_ms_per_frame"] == 0.245
    assert set(g["medium_ms"]) == {"sigma_only", "hash_texture"}
    assert [k for k in g["serve"] if k[0].isdigit()] == ["10", "30", "100", "300", "1000", "2000"]
    assert len(json.dumps(g)) < 1400
    bare = {k: out[k] for k in ("value", "fwd_segments_per_s", "ms_per_step", "roofline")}
    bare.update(e2e=None, large=None, batch=None, c0=None, medium=None, paper_loss=None, serve=None)
    g = bench.summary_digest(bare)
    assert g["e2e_gseg_s"] is None and "large" not in g and "serve" not in g
