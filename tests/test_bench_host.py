"""CPU: the host logic of bench.py that needs no GPU -- the summary of nvidia-smi clock samples
taken during the timed region, the roofline denominators and the workload description."""
import os
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

NA = "Not Active"


def _row(sm, mx, hw=NA, hw_th=NA, sw_th=NA, cap=NA):
    return f"0, {sm}, {mx}, 912.40, 0x0000000000000000, {hw}, {hw_th}, {sw_th}, {cap}"


def _summary(lines):
    s = bench.ClockSampler(0)
    s.lines = list(lines)
    return s.summary()


def test_clock_summary_median_max_and_reasons():
    out = _summary([_row(2070, 2070), _row(1980, 2070, cap="Active"), _row(2055, 2070), "", "garbage"])
    assert out["sm_mhz"] == 2055 and out["sm_max_mhz"] == 2070 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_summary_reports_every_rejecting_reason():
    out = _summary([_row(1500, 2070, hw="Active"), _row(1400, 2070, hw_th="Active", sw_th="Active")])
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert out["sm_mhz"] == 1450


def test_clock_summary_skips_unreadable_samples():
    out = _summary([_row("[N/A]", 2070), "0, 2070"])
    assert out == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
    assert _summary([])["reasons"] == ["no nvidia-smi samples"]


def test_peaks_have_the_roofline_denominators():
    peaks, source = bench.measured_peaks()
    assert source in ("measured", "fallback")
    for k in ("hbm_gbs", "bf16_tflops"):
        assert float(peaks[k]) > 0
    if source == "fallback":
        assert peaks["hbm_gbs"] == 6800.0 and peaks["bf16_tflops"] == 1900.0


def test_workload_description_names_sizes_and_l2_rule():
    args = types.SimpleNamespace(buses=60, columns=525600, seed=3, tol=1e-10)
    f, cfg = bench.workload(args)
    assert cfg["buses"] == 60 and cfg["pq_buses"] == f.n_pq == 59 and cfg["columns"] == 525600
    assert "60-bus" in cfg["workload"] and "525,600" in cfg["workload"]
    assert 0 < cfg["load_scale"] <= 1
    assert "%.1f GB" % (525600 * 59 * 16 / 1e9) in cfg["l2"]


def test_cpu_newton_leg_converges_and_agrees_with_the_oracle():
    from paper_2403_04578_gb300 import inputs as G

    f = G.make_feeder(60, 2)
    S = G.load_tensor(f, 4096, 2)
    r = bench.cpu_newton_leg(f, S, 4096, columns=8)
    assert r["converged"] == 8 and r["cores"] == 1 and r["value"] > 0
    assert 1 <= r["mean_iterations"] <= 10
    assert r["max_abs_err_pu_vs_fpi_oracle"] <= 1e-9
    for k in ("value", "unit", "cores", "kind", "sample"):
        assert k in r


def test_secondary_leg_failure_is_recorded_not_fatal(capsys):
    def boom(x):
        raise ValueError(f"bad {x}")

    assert bench.secondary(lambda a, b: {"value": a + b}, 1, 2) == {"value": 3}
    assert bench.secondary(boom, 7) == {"error": "ValueError: bad 7"}
    assert "ValueError" in capsys.readouterr().err
