"""Host-side logic of bench.py that needs no GPU: the clock-sample summary,
the peak lookup, the workload description and the traffic record."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _summary(tmp_path, lines):
    s = bench.ClockSampler(0)
    p = tmp_path / "clocks.csv"
    p.write_text("\n".join(lines) + "\n")

    class F:
        name = str(p)
    s.fh = F()
    return s.summary()


def test_clock_summary_median_max_and_reasons(tmp_path):
    rows = ["0, 2070, 2070, 880.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2055, 2070, 1010.2, 0x0, Not Active, Not Active, Not Active, Not Active"]
    d = _summary(tmp_path, rows)
    assert d["sm_mhz"] == 2055.0 and d["sm_max_mhz"] == 2070.0 and d["samples"] == 3
    assert d["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_thermal_and_skips_bad_rows(tmp_path):
    rows = ["garbage", "0, N/A, 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1500, 2070, 700.0, 0x40, Active, Not Active, Active, Not Active"]
    d = _summary(tmp_path, rows)
    assert d["samples"] == 1 and d["sm_mhz"] == 1500.0
    assert d["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples(tmp_path):
    assert _summary(tmp_path, ["not, a, sample"]) is None


def test_measured_peak_is_read_from_the_repository():
    hbm, kind = bench.measured_peaks()
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            assert hbm == float(json.load(fh)["hbm_gbs"]) and kind == "measured"
    else:
        assert (hbm, kind) == (6800.0, "fallback")


def test_workload_config_names_the_workload():
    c = bench.workload_config(256)
    assert c["grid"] == [256, 256, 256] and c["workload"].startswith("drops256_walls_z")
    assert "l2" in c and "parallelism" in c and "model" not in c


def test_traffic_record_points_at_a_kernel_source():
    for cls, rec in bench.NCU_TRAFFIC.items():
        assert cls in ("smooth0", "restrict0", "prolong0", "matvec0", "resid64")
        assert rec["bytes_per_launch"] > 0
        assert len(bench.kernel_source_sha(rec["source"])) == 16


def test_viscous_oracle_sample_extrapolates_to_the_stored_counts():
    import paris_inputs as pi
    pr = pi.config2(n=16)
    s = bench.viscous_oracle_sample(pr, 0.05, {"components": [{"iters": 10}, {"iters": 20}, {"iters": 30}]})
    assert s["cg_iters_full"] == [10, 20, 30] and s["cg_iters_sampled"][0] == 1
    assert s["cg_iters_sampled"][1] >= 9 and s["s_per_cg_iter"] >= 0.0 and s["setup_s"] >= 0.0
    assert s["step_s"] >= 3 * s["setup_s"] + 60 * s["s_per_cg_iter"]
    # no stored solves: a small grid's full oracle solves are run and counted
    full = bench.viscous_oracle_sample(pr, 0.01, None)["cg_iters_full"]
    assert len(full) == 3 and all(k > 0 for k in full)
    with pytest.raises(FileNotFoundError):
        bench.viscous_oracle_sample(pi.config2(n=80), 0.01, None)


def test_oracle_sample_counts_small_grids_and_refuses_large_ones_without_a_stored_solve():
    import paris_inputs as pi
    s = bench.oracle_sample(pi.config2(n=16), 0.05, None)
    assert s["cg_iters_full"] > 0 and s["solve_s"] > 0
    with pytest.raises(FileNotFoundError):
        bench.oracle_sample(pi.config2(n=80), 0.01, None)
