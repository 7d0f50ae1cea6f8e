"""The bench's roofline arithmetic on synthetic profile statistics (host only).

`roofline` turns the library's per-kernel CUDA-event times and algorithmic byte
and flop counts into the JSON line's `roofline` object.  These checks fix what
the line promises: frac = bytes per launch / mean launch time / measured copy
bandwidth for the kernel with the largest share of the profiled step; the
derived FP32 peak comes from the SM count and the sampled clock; the traffic
field scales the ncu DRAM/algorithmic ratio only for the kernel it was taken on.
"""
import math

import pytest

import bench


def _stats(op_ms, upd_ms=10.0, pupd_ms=5.0):
    """Synthetic profile: p = 2 mechanics dominant unless told otherwise; op_ms is
    the per-class operator time [p1 mech, p1 scal, p2 mech, p2 scal, p3 mech, p3 scal]."""
    launches = [100, 0, 200, 0, 0, 0]
    bytes_ = [2e9, 0.0, 1.2e10, 0.0, 0.0, 0.0]
    flops = [6e10, 0.0, 4e11, 0.0, 0.0, 0.0]
    n = sum(launches)
    return {
        "op_class_launches": launches, "op_class_ms": op_ms, "op_class_bytes": bytes_,
        "op_class_flops": flops, "op_class_active_frac": [0.7, 0.0, 0.6, 0.0, 0.0, 0.0],
        "op_launches": n, "op_ms": sum(op_ms), "op_bytes": sum(bytes_), "op_flops": sum(flops),
        "op_active_frac": 0.65,
        "update_ms": upd_ms, "update_bytes": n * 1e8, "pupdate_ms": pupd_ms, "pupdate_bytes": n * 6e7,
        "finalize_ms": 1.0, "residual_launches": 7, "residual_ms": 4.0,
    }


PEAKS = {"hbm_gbs": 6780.4, "sm_max_mhz": 2070.0}


def test_headline_is_the_hbm_fraction_of_the_dominant_kernel():
    st = _stats([5.0, 0.0, 20.0, 0.0, 0.0, 0.0])
    out = bench.roofline(st, 100.0, PEAKS, "measured", {"sm_mhz": 2070.0}, 152)
    assert out["kernel"] == "k_operator<p=2,mech,f32>"
    k = out["kernels"]["k_operator<p=2,mech,f32>"]
    bpl = 1.2e10 / 200
    mean_ms = 20.0 / 200
    achieved = bpl / (mean_ms / 1e3) / 1e9
    assert k["bytes_per_launch"] == pytest.approx(bpl)
    assert k["mean_launch_ms"] == pytest.approx(mean_ms)
    assert out["achieved"] == pytest.approx(achieved)
    assert out["frac"] == pytest.approx(achieved / 6780.4)
    assert out["peak"] == 6780.4 and out["unit"] == "GB/s" and out["bound"] == "hbm"
    assert k["share_of_step"] == pytest.approx(0.2)


def test_derived_fp32_peak_and_alu_fraction():
    st = _stats([5.0, 0.0, 20.0, 0.0, 0.0, 0.0])
    out = bench.roofline(st, 100.0, PEAKS, "measured", {"sm_mhz": 1800.0}, 148)
    peak = 148 * 128 * 2 * 1800e6 / 1e12
    assert out["peaks"]["fp32_tflops"] == pytest.approx(peak)
    assert "148 SM" in out["peaks"]["fp32_kind"] and "1800 MHz" in out["peaks"]["fp32_kind"]
    k = out["kernels"]["k_operator<p=2,mech,f32>"]
    tflops = 4e11 / (20.0 / 1e3) / 1e12
    assert k["tflops"] == pytest.approx(tflops)
    assert out["alu_frac_derived"] == pytest.approx(tflops / peak)
    # the binding roof is the larger of the two fractions
    assert out["binding_roof"] == ("alu" if tflops / peak >= out["frac"] else "hbm")


def test_traffic_only_for_the_captured_kernel():
    st = _stats([5.0, 0.0, 20.0, 0.0, 0.0, 0.0])
    out = bench.roofline(st, 100.0, PEAKS, "measured", {"sm_mhz": 2070.0}, 152)
    ratio = bench.TRAFFIC_CAPTURE["dram_bytes"] / bench.TRAFFIC_CAPTURE["algorithmic_bytes"]
    assert bench.TRAFFIC_CAPTURE["ratio"] == pytest.approx(ratio)
    assert out["traffic"] == pytest.approx(ratio * 1.2e10 / 200)
    # a step dominated by the vector update: no ncu capture of it, so no traffic figure
    st = _stats([1.0, 0.0, 2.0, 0.0, 0.0, 0.0], upd_ms=60.0)
    out = bench.roofline(st, 100.0, PEAKS, "measured", {"sm_mhz": 2070.0}, 152)
    assert out["kernel"] == "k_update"
    assert out["traffic"] is None
    assert out["frac"] == pytest.approx(300 * 1e8 / 300 / (60.0 / 300 / 1e3) / 1e9 / 6780.4)


def test_all_instances_entry_is_never_the_headline():
    # the sum over operator instances has the largest share by construction
    st = _stats([30.0, 0.0, 31.0, 0.0, 0.0, 0.0])
    out = bench.roofline(st, 100.0, PEAKS, "measured", {"sm_mhz": 2070.0}, 152)
    assert out["kernels"]["k_operator (all instances)"]["share_of_step"] == pytest.approx(0.61)
    assert out["kernel"] == "k_operator<p=2,mech,f32>"
    assert math.isfinite(out["frac"])
