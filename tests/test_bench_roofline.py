"""Host logic of the benchmark's roofline object: the dominant phase is the
one with the most event time; achieved = its algorithmic work / its time;
the peak follows the phase's bound (the measured copy bandwidth, the bf16
burst peak -- the phases are timed with every kernel alone -- scaled by the
precision's nominal ratio or by six slice products, or the nominal FP64
rate); traffic comes from the ncu captures, per n^2 for the sweeps and as a
ratio to algorithmic bytes where one was captured.  Every phase with at least
1 % of the dominant one's time gets its own entry.  Synthetic phase records;
no GPU."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def phases(**ms):
    base = {p: {"launches": 0, "ms": 0.0, "flops": 0.0, "bytes": 0.0} for p in
            ["convert", "leaf", "trailing", "solve", "resid", "panel", "trailing_x3", "resid_df32", "resid_tc"]}
    for k, (launches, t, flops, by) in ms.items():
        base[k] = {"launches": launches, "ms": t, "flops": flops, "bytes": by}
    return base


def test_sweeps_dominant_hbm_with_traffic_scaled_by_n2():
    peaks, _ = bench.load_peaks()
    n = 16384
    ph = phases(solve=(10, 15.0, 0.0, 10 * 4.0 * n * n), leaf=(100, 5.0, 1e9, 1e8))
    r = bench.roofline(ph, [{"prec_used": "fp16"}], n)
    assert r["kernel_phase"] == "solve" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(10 * 4.0 * n * n / 15e-3 / 1e9)
    assert r["peak"] == peaks["hbm_gbs"] and r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["avg_launch_ms"] == pytest.approx(1.5)
    assert r["algorithmic_per_launch"] == pytest.approx(4.0 * n * n)
    # traffic of one pair: the capture's bytes per n^2, times n^2
    assert r["traffic"] == pytest.approx(bench.MEASURED_TRAFFIC["solve"][0] * n * n)
    assert 4.0 < bench.MEASURED_TRAFFIC["solve"][0] < 4.3  # one triangle of float32 per sweep, plus a few %


def test_fp32_updates_dominant_tensor_against_six_slice_products():
    peaks, _ = bench.load_peaks()
    burst = peaks["bf16_tflops"]
    sus = peaks.get("bf16_tflops_sustained", burst)
    ph = phases(trailing_x3=(500, 36.0, 2.9e12, 5.0e10), solve=(10, 15.0, 0.0, 1e10),
                leaf=(10, 0.1, 1e6, 1e6))
    r = bench.roofline(ph, [{"prec_used": "fp32"}], 16384)
    assert r["kernel_phase"] == "trailing_x3" and r["bound"] == "tensor"
    assert r["achieved"] == pytest.approx(2.9e12 / 36e-3 / 1e12)
    assert r["peak"] == pytest.approx(burst / 6)
    assert r["frac_of_sustained"] == pytest.approx(r["achieved"] / (sus / 6))
    if "trailing_x3" in bench.MEASURED_TRAFFIC_RATIO:
        ratio = bench.MEASURED_TRAFFIC_RATIO["trailing_x3"][0]
        assert r["traffic"] == pytest.approx(ratio * 5.0e10 / 500)
    else:
        assert r["traffic"] is None
    # every phase above 1 % of the dominant one's time has its own entry
    assert set(r["phases"]) == {"trailing_x3", "solve"}
    assert r["phases"]["solve"]["bound"] == "hbm"


@pytest.mark.parametrize("prec,scale", [("fp16", 1.0), ("bf16", 1.0), ("tf32", 0.5), ("fp8", 2.0)])
def test_low_precision_updates_take_their_precision_peak(prec, scale):
    peaks, _ = bench.load_peaks()
    bf16 = peaks["bf16_tflops"]
    ph = phases(trailing=(100, 10.0, 1e13, 1e9))
    r = bench.roofline(ph, [{"prec_used": prec}], 8192)
    assert r["bound"] == "tensor" and r["peak"] == pytest.approx(bf16 * scale)
    assert r["traffic"] is None  # no capture for this phase


def test_float64_residual_against_the_fp64_rate():
    ph = phases(resid=(4, 40.0, 4 * 2.0 * 16384 ** 2 * 16, 4 * 8.0 * 16384 ** 2))
    r = bench.roofline(ph, [{"prec_used": "fp32"}], 16384)
    assert r["bound"] == "alu" and r["peak"] == bench.FP64_PEAK_TFLOPS
    assert r["achieved"] == pytest.approx(4 * 2.0 * 16384 ** 2 * 16 / 40e-3 / 1e12)


def test_tensor_core_residual_is_hbm_bound():
    peaks, _ = bench.load_peaks()
    by = 4 * 20.0 * 16384 ** 2
    ph = phases(resid_tc=(4, 3.3, 0.0, by))
    r = bench.roofline(ph, [{"prec_used": "fp16"}], 16384)
    assert r["bound"] == "hbm" and r["peak"] == peaks["hbm_gbs"]
    assert r["achieved"] == pytest.approx(by / 3.3e-3 / 1e9)


def test_leaf_dominant_is_measured_against_one_sm():
    """The leaves are one CTA each by design: their ceiling is one SM's FP32
    rate; the fraction of the whole GPU is reported beside it."""
    ph = phases(leaf=(650, 26.0, 650 * 128 ** 3 / 3.0, 650 * 128 * 128 * 4.0), solve=(23, 22.0, 0.0, 23 * 4.0 * 16384 ** 2))
    r = bench.roofline(ph, [{"prec_used": "fp16"}], 16384)
    assert r["kernel_phase"] == "leaf" and r["bound"] == "alu"
    assert r["peak"] == pytest.approx(bench.FP32_SM_PEAK_TFLOPS)
    assert r["achieved"] == pytest.approx(650 * 128 ** 3 / 3.0 / 26e-3 / 1e12)
    assert r["frac_of_gpu"] == pytest.approx(r["achieved"] / bench.FP32_SIMT_PEAK_TFLOPS)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
