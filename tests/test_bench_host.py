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
    rows = ["2026/12/04 10:00:00.000, 0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "2026/12/04 10:00:00.100, 0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
            "2026/12/04 10:00:00.200, 0, 2070, 2070, 1200.5, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage line"]
    p = tmp_path / "clocks.csv"
    p.write_text("\n".join(rows) + "\n")
    cs = bench.ClockSampler(0)
    cs.path = str(p)
    s = cs.summary()  # no timed region marked: every sample
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"] and not s["in_timed_region"]
    p.write_text("2026/12/04 10:00:00.000, 0, 1500, 2070, 1000, 0x8, Active, Not Active, Active, Not Active\n")
    cs.path = str(p)
    assert cs.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_keeps_the_samples_of_the_timed_region(bench, tmp_path):
    # samples before the region (an idle clock, a throttle reason) are left out
    rows = ["2026/12/04 10:00:00.000, 0, 990, 2070, 100.0, 0x1, Not Active, Not Active, Not Active, Active",
            "2026/12/04 10:00:01.000, 0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "2026/12/04 10:00:01.020, 0, 2055, 2070, 910.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "2026/12/04 10:00:01.040, 0, 2070, 2070, 905.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    p = tmp_path / "clocks.csv"
    p.write_text("\n".join(rows) + "\n")
    cs = bench.ClockSampler(0)
    cs.path = str(p)
    cs.t0 = bench.ClockSampler._stamp("2026/12/04 10:00:00.900")
    cs.t1 = bench.ClockSampler._stamp("2026/12/04 10:00:01.050")
    s = cs.summary()
    assert s["samples"] == 3 and s["in_timed_region"] and s["reasons"] == [] and s["sm_mhz"] == 2070.0


def test_binding_roofline_takes_the_longer_of_hbm_and_alu_time(bench):
    # 152 SMs: ALU peak 1.3422e13 candidates/s; at 6784.5 GB/s and 10 B/sample the
    # balance point is ~19.8 candidates per sample
    r = bench.binding_roofline(7.0, 10, 1 << 30, 2.0, 152, 6784.5)
    assert r["bound"] == "hbm" and abs(r["balance_candidates_per_sample"] - 19.78) < 0.05
    assert r["frac"] == pytest.approx(r["frac_hbm"]) and r["frac_alu"] < r["frac_hbm"]
    r = bench.binding_roofline(31.9, 10, 1 << 30, 5.0, 152, 6784.5)
    assert r["bound"] == "alu" and r["frac"] == pytest.approx(31.9 * (1 << 30) / 5e-3 / 1.3422e13, rel=1e-3)
    # IG(2) (15 candidates per sample) and BD-8 (16) sit below the balance: HBM-bound
    for c in (15.0, 16.0):
        assert bench.binding_roofline(c, 10, 1 << 30, 5.0, 152, 6784.5)["bound"] == "hbm"


def test_workloads_and_defaults(bench, monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert (a.gpus, a.workload, a.algo, a.dtype, a.warmup) == (1, "ska_mid", "ig1", "f32", 3)
    assert (a.ndm, a.nt, a.s_end) == (4096, 1 << 20, 8192)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "noise_stats"])
    assert bench.parse().workload == "noise_stats"


def test_search_launches_of_each_grid(bench):
    import paper_1910_08324_gb300 as spd
    for algo, n in (("ig1", 1), ("bd16", 1), ("bd12", 2), ("bd24", 2)):
        plan = spd.spd_plan_create(ndm=1, nt=1 << 16, s_end=8192, **bench.ALGOS[algo])
        assert bench.search_launches(algo, plan.widths()[0]) == n, algo
    low = spd.spd_plan_create(ndm=1, nt=1 << 16, s_end=40, **bench.ALGOS["bd12"])  # levels 0-1 only
    assert bench.search_launches("bd12", low.widths()[0]) == 1
