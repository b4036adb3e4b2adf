"""The benchmark's roofline arithmetic (host logic, no GPU): algorithmic bytes and FLOPs per launch,
the choice of the binding roof, and the FP32 ALU peak derived from unit counts and clocks."""
import importlib.util
import os
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


# The 256-element ULA case: M = B = N = 256, L = 512, 64 blocks; stage 2 = 6 (TF32x3 tensor cores).
C2 = SimpleNamespace(M=256, N=256, B=256, L=512, S_time=2, P_time=512, P_space_x=512, P_gs=1024,
                     P_rec=512, S_rec=2, stage2=6)
PEAKS = {"hbm_gbs": 6690.8, "bf16_tflops": 1972.2, "sm_max_mhz": 2070.0}
FP32 = {"tflops": 72.5, "source": "measured (test value)"}
# The 1024-element ULA: M = B = 1024, N = 512, L = 1024; stage 2 = 6 (TF32x3 tensor cores).
ULA1024 = SimpleNamespace(M=1024, N=512, B=1024, L=1024, S_time=2, P_time=1024, P_space_x=2048, P_gs=2048,
                          P_rec=1024, S_rec=2, stage2=6)


def test_tf32x3_stage2_bytes_flops_and_bound():
    b = _bench()
    # Compulsory bytes of one 64-block launch: G as FP32 re/im planes, w read once, bhat written.
    g_bytes = 256 * 2 * 256 * 512 * 4
    w_bytes = 256 * 512 * 64 * 8
    out_bytes = 256 * 256 * 64 * 8
    assert (g_bytes, w_bytes, out_bytes) == (268435456, 67108864, 33554432)
    # 8 N L flops per beam-block (complex multiply-add), 3 split-TF32 products per complex term.
    assert b.flop_model(C2)["stage2"] * 64 == 8 * 256 * 512 * 256 * 64
    # At the measured peaks HBM binds: 369.1 MB / 6690.8 GB/s = 55.2 us against
    # 3 x 17.18 GFLOP / (0.5 x 1972.2 TFLOP/s) = 52.3 us of tensor work.
    r = b.roofline("stage2", C2, 64, 0.1, PEAKS, "measured", FP32)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6690.8
    assert r["achieved"] == pytest.approx((g_bytes + w_bytes + out_bytes) / 1e-4 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6690.8)
    # With a much slower memory the same launch is tensor-bound, against the TF32 peak (bf16 / 2).
    r = b.roofline("stage2", C2, 64, 0.1, dict(PEAKS, hbm_gbs=20000.0), "measured", FP32)
    assert r["bound"] == "tensor" and r["peak"] == pytest.approx(986.1)
    assert r["achieved"] == pytest.approx(3 * 8 * 256 * 512 * 256 * 64 / 1e-4 / 1e12)


def test_fft_kernels_are_reported_against_the_fp32_alu_peak():
    b = _bench()
    r = b.roofline("czt_time", C2, 64, 0.0765, PEAKS, "measured", FP32)
    # The ALU roof is the FP32 peak handed in (the benchmark measures it on the GPU).
    assert r["bound"] == "alu" and r["peak"] == 72.5 and r["peak_source"] == FP32["source"]
    # Its nominal form: 152 SMs x 128 FP32 lanes x 2 flops per FMA x 2070 MHz.
    assert b.nominal_fp32_peak(152, 2070.0)["tflops"] == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12)
    # One forward and S = 2 inverse transforms of 512 points per sensor-block, 5 P log2 P each,
    # plus the chirp and spectrum multiplies (6 flops per complex multiply).
    per_sensor = 3 * 5 * 512 * 9 + 6 * (256 + 2 * 512 + 512)
    assert b.flop_model(C2)["czt_time"] == per_sensor * 256
    assert r["achieved"] == pytest.approx(per_sensor * 256 * 64 / 0.0765e-3 / 1e12)


def test_nulling_bracket_roofline():
    b = _bench()
    # C2N: B = 256, L = 512, two interferers, 64 blocks. Operator planes 8 B L P L = 1073741824 bytes,
    # w in + nulled w out 2 x 8 x 64 x 256 x 512 = 134217728 bytes: 180.5 us at 6690.8 GB/s, against
    # 3 x 8 B L P L nblk = 3 x 68.72 GFLOP = 209.1 us at 986.1 TFLOP/s: tensor-bound.
    flops = 8 * 256 * 512 * 2 * 512 * 64
    assert flops == 68719476736
    r = b.null_roofline(256, 512, 2, 64, 0.25, "tf32x3", PEAKS, "measured", FP32)
    assert r["bound"] == "tensor" and r["peak"] == pytest.approx(986.1)
    assert r["achieved"] == pytest.approx(3 * flops / 0.25e-3 / 1e12)
    # One interferer: 80.2 us of operator + 20.1 us of w against 104.5 us of tensor work: still
    # tensor-bound; at a slower memory (3000 GB/s) the same launch is HBM-bound.
    r = b.null_roofline(256, 512, 1, 64, 0.2, "tf32x3", PEAKS, "measured", FP32)
    assert r["bound"] == "tensor"
    r = b.null_roofline(256, 512, 1, 64, 0.2, "tf32x3", dict(PEAKS, hbm_gbs=3000.0), "measured", FP32)
    assert r["bound"] == "hbm" and r["peak"] == 3000.0
    assert r["achieved"] == pytest.approx((8 * 256 * 512 * 512 + 2 * 8 * 64 * 256 * 512) / 0.2e-3 / 1e9)
    # The FP32 CUDA-core contraction is reported against the FP32 ALU peak.
    r = b.null_roofline(256, 512, 2, 64, 1.0, "fp32", PEAKS, "measured", FP32)
    assert r["bound"] == "alu" and r["achieved"] == pytest.approx(flops / 1e-3 / 1e12)


def test_whole_path_bytes_are_32_per_beam_sample_at_m_equal_b():
    b = _bench()
    # y in (8 M N), bhat out (8 B N) and one generator per beam (8 B L) per block: at M = B and
    # L = 2N that is 8 (N + N + 2N) B / (B N) = 32 bytes per beam-sample.
    assert b.path_bytes(ULA1024, 64) == 8.0 * 64 * (1024 * 512 + 1024 * 512 + 1024 * 1024)
    assert b.path_bytes(ULA1024, 64) / (64 * 1024 * 512) == 32.0
    assert b.path_bytes(C2, 64) / (64 * 256 * 256) == 32.0


def test_path_roofline_takes_the_binding_roof():
    b = _bench()
    # ULA1024, TF32x3: 2.15 GB of compulsory bytes (0.32 ms at 6690.8 GB/s) against the FFT flops
    # on the FP32 roof plus 3 split-TF32 products on the tensor roof.
    fm = b.flop_model(ULA1024)
    t_alu = (fm["czt_time"] + fm["czt_space"]) * 64 / 72.5e12
    t_tc = 3 * fm["stage2"] * 64 / (0.5 * 1972.2e12)
    r = b.path_roofline(ULA1024, 64, 2.0, PEAKS, FP32)
    assert r["bound"] == "compute"
    assert r["t_roof_ms"] == pytest.approx((t_alu + t_tc) * 1e3)
    assert r["frac"] == pytest.approx((t_alu + t_tc) / 2e-3)
    assert r["bytes_per_beam_sample"] == 32.0
    # With an absurdly fast FP32 roof the bytes bind.
    r = b.path_roofline(SimpleNamespace(**dict(vars(ULA1024), stage2=2)), 64, 2.0, PEAKS, {"tflops": 1e9, "source": ""})
    assert r["bound"] == "hbm"
