"""The bench's roofline arithmetic on the host: the achieved rate is the
algorithmic FLOPs of all timed steps over the dominant kernel's CUDA-event
time, the fraction divides by the stated peak, and the DRAM traffic of a
capture is reported only while the workload and the kernels' sources match
it (hand-computed values; no GPU)."""
import copy

import pytest

import bench

ALU_PEAK = 152 * 128 * 2 * 2070.0e6 / 1e12   # TFLOP/s


def _prof(fft=(30.0, 20.0), tc=(0.0, 0.0), simt=(0.0, 0.0), n=4):
    keys = ("conv_forward_fft", "conv_adjoint_fft", "conv_forward_tc", "conv_adjoint_tc",
            "conv_forward", "conv_adjoint")
    ms = fft + tc + simt
    return {k: {"total_ms": t, "launches": n if t else 0} for k, t in zip(keys, ms)}


WORK = {"fft_flops": 1.0e11, "conv_flops": 6.0e11, "mma_flops": 3.0e12}


def test_fft_roofline_arithmetic():
    steps = 10
    r = bench._roofline(_prof(), WORK, steps, "another workload")
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    # 1e11 FLOP per step x 10 steps over 50 ms of FFT time
    assert r["achieved"] == pytest.approx(20.0, rel=1e-12)
    assert r["peak"] == pytest.approx(ALU_PEAK, rel=1e-12)
    assert r["frac"] == pytest.approx(20.0 / ALU_PEAK, rel=1e-12)
    # per launch: 8 launches of the two FFT directions
    assert r["flops_per_launch"] == pytest.approx(1.0e12 / 8, rel=1e-12)
    assert r["ms_per_launch"] == pytest.approx(50.0 / 8, rel=1e-12)
    # the direct-convolution equivalent: 2 passes x 6e11 x 10 steps over 50 ms
    assert r["direct_equivalent_tflops"] == pytest.approx(240.0, rel=1e-12)
    assert r["traffic"] is None   # no capture of this workload


def test_captured_traffic_only_for_matching_sources(monkeypatch):
    wl = bench._CAPTURES["workload"]
    r = bench._roofline(_prof(), WORK, 10, wl)
    fb = bench._CAPTURES["conv_forward_fft"]["bytes"]
    ab = bench._CAPTURES["conv_adjoint_fft"]["bytes"]
    assert r["traffic"] == pytest.approx(0.5 * (fb + ab))
    stale = copy.deepcopy(bench._CAPTURES)
    stale["conv_forward_fft"]["sha"] = "0" * 16
    monkeypatch.setattr(bench, "_CAPTURES", stale)
    assert bench._roofline(_prof(), WORK, 10, wl)["traffic"] is None


def test_tensor_and_simt_kernels_when_they_dominate():
    r = bench._roofline(_prof(fft=(0.0, 0.0), tc=(40.0, 40.0)), WORK, 10, "w")
    assert r["bound"] == "tensor"
    assert r["achieved"] == pytest.approx(2.0 * 6.0e11 * 10 / 0.08 / 1e12, rel=1e-12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-12)
    assert r["tensor_issued_tflops"] == pytest.approx(3.0e12 * 10 / 0.08 / 1e12, rel=1e-12)
    s = bench._roofline(_prof(fft=(0.0, 0.0), simt=(50.0, 50.0)), WORK, 10, "w")
    assert s["bound"] == "alu" and s["kernel"].startswith("k_conv ")
    assert s["achieved"] == pytest.approx(2.0 * 6.0e11 * 10 / 0.1 / 1e12, rel=1e-12)


def test_kernel_hbm_fraction():
    wl = bench._CAPTURES["workload"]
    prof = {"gather_accumulate": {"total_ms": 15.0, "launches": 10}}
    out = bench._kernel_hbm(prof, wl)["gather_accumulate"]
    b = bench._CAPTURES["gather_accumulate"]["bytes"]
    assert out["ms_per_launch"] == pytest.approx(1.5)
    assert out["achieved_gbs"] == pytest.approx(b / 1.5e-3 / 1e9)
    assert out["frac"] == pytest.approx(out["achieved_gbs"] / out["peak_gbs"])
