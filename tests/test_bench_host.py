"""Host logic of bench.py: the DRAM traffic records (valid only for the kernel
sources they were captured on), the clock-sample summary that decides whether a
run was throttled, and the workload list."""
import importlib.util
import json
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_committed_traffic_records_match_the_committed_kernels(bench):
    # a record taken on other kernel sources would be reported as null by the bench
    with open(os.path.join(ROOT, "profiles", "search_kernel_traffic.json")) as f:
        ig1 = json.load(f)["ig1"]
    assert bench.recorded_traffic("ig1", 4096, 1 << 20) == pytest.approx(ig1["bytes_per_sample"] * 4096 * (1 << 20))
    with open(os.path.join(ROOT, "profiles", "msd_pass_traffic.json")) as f:
        msd = json.load(f)["msd_pass_f32"]
    assert bench.recorded_msd_traffic("f32", 4096, 1 << 20) == pytest.approx(msd["bytes_per_sample"] * 4096 * (1 << 20))
    # traffic close to the algorithmic bytes (no re-reads): 10 B/sample search, 4 B/sample pass
    assert 9.5 < ig1["bytes_per_sample"] < 10.5 and 3.9 < msd["bytes_per_sample"] < 4.1


def test_traffic_record_of_other_sources_or_types_is_null(bench, tmp_path, monkeypatch):
    assert bench.recorded_msd_traffic("f16", 10, 10) is None   # no record for that input type
    assert bench.recorded_traffic("bd32", 10, 10) is None      # nor for that grid
    # a copy of the tree whose pass kernel differs by one byte: the record no longer applies
    for rel in bench.MSD_SOURCES + bench.SEARCH_SOURCES:
        dst = tmp_path / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(ROOT, rel), dst)
    (tmp_path / "profiles").mkdir()
    for name in ("msd_pass_traffic.json", "search_kernel_traffic.json"):
        shutil.copy(os.path.join(ROOT, "profiles", name), tmp_path / "profiles" / name)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_msd_traffic("f32", 10, 10) is not None
    with open(tmp_path / bench.MSD_SOURCES[0], "ab") as f:
        f.write(b"\n")
    assert bench.recorded_msd_traffic("f32", 10, 10) is None
    assert bench.recorded_traffic("ig1", 10, 10) is not None  # the search kernels did not change


def test_clock_summary_reports_median_and_throttle_reasons(bench, tmp_path):
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1200.5, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage line"]
    p = tmp_path / "clocks.csv"
    p.write_text("\n".join(rows) + "\n")
    cs = bench.ClockSampler(0)
    cs.path = str(p)
    s = cs.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    p.write_text("0, 1500, 2070, 1000, 0x8, Active, Not Active, Active, Not Active\n")
    cs.path = str(p)
    assert cs.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_workloads_and_defaults(bench, monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert (a.gpus, a.workload, a.algo, a.dtype, a.warmup) == (1, "ska_mid", "ig1", "f32", 3)
    assert (a.ndm, a.nt, a.s_end) == (4096, 1 << 20, 8192)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "noise_stats"])
    assert bench.parse().workload == "noise_stats"
