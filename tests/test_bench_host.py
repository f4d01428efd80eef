"""Host logic of bench.py that decides whether a benchmark line is valid: the summary of the
nvidia-smi clock samples taken during the timed region (the median SM clock under load, the
maximum clock, and the throttle reasons that were active)."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
bench = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(bench)

IDLE = "Not Active"


def line(sm, mx, hw=IDLE, hwt=IDLE, swt=IDLE, cap=IDLE, power="850.25"):
    return f"0, {sm}, {mx}, {power}, 0x0000000000000000, {hw}, {hwt}, {swt}, {cap}\n"


def test_steady_clocks_no_reasons():
    s = bench.summarize_clocks([line(2070, 2070)] * 3)
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}


def test_idle_samples_do_not_pull_the_median_down():
    s = bench.summarize_clocks([line(345, 2070), line(2070, 2070), line(2055, 2070), line(2070, 2070)])
    assert s["sm_mhz"] == 2070.0 and s["samples"] == 4


def test_reasons_are_collected_by_name():
    s = bench.summarize_clocks([line(1980, 2070, cap="Active"), line(1900, 2070, hwt="Active"), line(2070, 2070)])
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clock_stuck_low_shows_in_the_median():
    # a leftover clock lock: every sample well below the maximum, no reason active
    s = bench.summarize_clocks([line(1005, 2070)] * 5)
    assert s["sm_mhz"] == 1005.0 and s["sm_max_mhz"] == 2070.0 and s["reasons"] == []


def test_unavailable_fields_and_empty_output():
    s = bench.summarize_clocks([line("[N/A]", "[N/A]"), line(2070, 2070)])
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert bench.summarize_clocks([]) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
    assert bench.summarize_clocks(["garbage\n"])["reasons"] == ["no samples"]


def test_sampler_runs_the_tool_and_summarizes(tmp_path, monkeypatch):
    # a stand-in nvidia-smi on PATH that prints samples until it is terminated
    tool = tmp_path / "nvidia-smi"
    tool.write_text("#!/bin/sh\nwhile true; do echo '0, 2070, 2070, 700.0, 0x0, Not Active, Not Active, "
                    "Not Active, Active'; sleep 0.05; done\n")
    tool.chmod(0o755)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    s = bench.ClockSampler(0)
    s.start()
    import time
    time.sleep(0.3)
    out = s.stop()
    assert out["sm_mhz"] == 2070.0 and out["reasons"] == ["sw_power_cap"] and out["samples"] >= 2


def test_sampler_without_the_tool(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    s = bench.ClockSampler(0)
    s.start()
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_ncu_traffic_only_for_the_captured_source(monkeypatch):
    # a recorded capture counts only while the kernel's source file hashes as it did then
    src = "panel_flat.cu"
    digest = bench.source_digest(src)
    assert digest is not None and len(digest) == 16
    monkeypatch.setitem(bench.NCU_TRAFFIC, "probe", (1234, 1.0, src, digest))
    assert bench.ncu_traffic("probe") == 1234
    # captured on half the units the bench runs: the bytes scale in proportion
    monkeypatch.setitem(bench.NCU_TRAFFIC, "probe", (1000, 16384, src, digest))
    assert bench.ncu_traffic("probe", 32768) == 2000
    monkeypatch.setitem(bench.NCU_TRAFFIC, "probe", (1234, 1.0, src, "0" * 16))
    assert bench.ncu_traffic("probe") is None
    assert bench.ncu_traffic("no such kernel") is None
