"""Parity of the CUDA path (called through the C ABI) with the FP64 oracle on seeded inputs.

Tolerance: relative L2 error <= 1e-5 for every FP32 result (the end-to-end bar), and <= 2e-6 for
the stage-1 outputs alone. Outputs are poisoned with NaN before each call so an unwritten entry
fails. Sizes span several CTA tiles and ragged tails (M, B not multiples of the tile widths).
"""
import numpy as np
import pytest

import oracle as O
from synth import configs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_E2E = 1e-5
TOL_STAGE1 = 2e-6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_08887_gb300.build import build
    build()


def _fb():
    import paper_2512_08887_gb300 as fb
    return fb


def make(kind, mx, my, bx, by, N, frac_bw, stage2="auto", delta_rel=1e-3, max_blocks=64, gamma=(2, 1), eps=1.01):
    fb = _fb()
    plan = fb.Plan(fb.make_geometry(kind, mx, my, bx, by), N,
                   fb.make_band(frac_bw, epsilon=eps, gamma=gamma, delta=delta_rel, stage2=stage2,
                                max_blocks=max_blocks))
    i = plan.info
    pb = O.make_problem(kind, mx, my, bx, by, N, frac_bw=i.fb_num / i.fb_den, epsilon=i.eps_num / i.eps_den,
                        delta=i.delta, L=i.L)
    return plan, pb


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def nan_like(shape):
    return torch.full(shape, complex(np.nan, np.nan), dtype=torch.complex64, device="cuda")


def crandn(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


def per_beam_err(got, ref):
    """max over beams of ||got_b - ref_b|| / max(||ref_b||, rms over beams of ||ref_b||), arrays
    (nblk, nbeams, N): a weak beam is held to the typical beam's scale (stage 1's rounding spreads
    over all beams of a frequency), a wrongly formed beam is off by its own norm."""
    e = np.linalg.norm(got - ref, axis=(0, 2))
    n = np.linalg.norm(ref, axis=(0, 2))
    return float(np.max(e / np.maximum(n, np.sqrt(np.mean(n ** 2)))))


def run(plan, fn, x, out_shape, nblk):
    out = nan_like(out_shape)
    getattr(plan, fn)(dev(x), out, nblk)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("M,N", [(16, 64), (13, 24), (256, 256), (40, 512), (8, 1024)])
def test_czt_time_matches_oracle(rng, M, N):
    # (8, 1024): L = 2048 outputs (P = 2048), the largest block a plan accepts (its
    # Gohberg-Semencul circulants then have the largest size, 2L = 4096).
    plan, pb = make("ula", M, 1, M, 1, N, 0.5)
    y = crandn(rng, 3, M, N)
    got = run(plan, "czt_time", y, (3, pb.L, M), 3)
    ref = O.stage1_time(pb, y).transpose(0, 2, 1)
    assert O.rel_l2(got, ref) < TOL_STAGE1


@pytest.mark.parametrize("case", [
    ("ula", 16, 1, 16, 1, 64, 0.5), ("ula", 13, 1, 10, 1, 24, 0.37), ("ula", 256, 1, 256, 1, 256, 0.5),
    ("ula", 100, 1, 150, 1, 64, 0.8), ("ura", 4, 4, 4, 4, 32, 0.3), ("ura", 8, 8, 8, 8, 64, 0.3),
    ("ula", 1024, 1, 1024, 1, 32, 0.5), ("ula", 2048, 1, 2048, 1, 16, 0.5),
])
def test_czt_matches_oracle(rng, case):
    # The last two: spatial transforms of P = 2048 and P = 4096 (the largest).
    kind, mx, my, bx, by, N, fbw = case
    plan, pb = make(kind, mx, my, bx, by, N, fbw)
    y = crandn(rng, 2, pb.M, N)
    got = run(plan, "czt", y, (2, pb.B, pb.L), 2)
    ref = O.fan_coefficients(pb, y)
    assert O.rel_l2(got, ref) < TOL_STAGE1


@pytest.mark.parametrize("case", [("ula", 16, 1, 16, 1, 64, 0.5), ("ula", 13, 1, 10, 1, 24, 0.37),
                                  ("ura", 4, 4, 4, 4, 32, 0.3)])
def test_levinson_generators_match_dense_solve(case):
    kind, mx, my, bx, by, N, fbw = case
    plan, pb = make(kind, mx, my, bx, by, N, fbw)
    x = plan.generators()
    for b in range(pb.B):
        ref = np.linalg.solve(O.gram(pb, b), np.eye(pb.L)[:, 0])
        assert O.rel_l2(x[b], ref) < 1e-9


@pytest.mark.parametrize("stage2", ["gs_ir1", "dense_fp32", "gs"])
@pytest.mark.parametrize("case", [("ula", 16, 1, 16, 1, 64, 0.5), ("ula", 13, 1, 10, 1, 24, 0.37),
                                  ("ura", 8, 8, 8, 8, 64, 0.3), ("ula", 64, 1, 64, 1, 512, 0.5),
                                  ("ula", 1, 1, 1, 1, 16, 0.5), ("ula", 4, 1, 4, 1, 1024, 0.5)])
def test_toeplitz_apply_matches_oracle(rng, stage2, case):
    # The last case has L = 2048: Gohberg-Semencul circulants of P = 4096 (the largest).
    # White-noise input puts energy where A_b is smallest (the worst case for FP32). Plain GS in
    # FP32 loses about eps32 * cond(A_b) ~ 6e-8 * 2/delta_rel to the difference of its two
    # triangular products, so it is held to 2e-4; the refined and dense variants to 1e-5.
    kind, mx, my, bx, by, N, fbw = case
    plan, pb = make(kind, mx, my, bx, by, N, fbw, stage2=stage2)
    y = crandn(rng, 3, pb.M, N)
    w = O.fan_coefficients(pb, y).astype(np.complex64)
    got = run(plan, "toeplitz_apply", w, (3, pb.B, N), 3)
    ref = O.Stage2Factors(pb).apply(w)
    assert O.rel_l2(got, ref) < (2e-4 if stage2 == "gs" else TOL_E2E)


def test_execute_c1_matches_oracle():
    d = configs.config_data("C1")
    for stage2 in ("gs_ir1", "dense_fp32"):
        plan, pb = make("ula", 16, 1, 16, 1, 64, 0.5, stage2=stage2)
        got = run(plan, "execute", d["y"], (1, 16, 64), 1)
        ref = O.fbst(pb, d["y"])
        assert O.rel_l2(got, ref) < TOL_E2E, stage2


def test_execute_c2_full_size_sampled_beams():
    # The benchmark's workload and launch configuration: 64 blocks of 256 snapshots, one launch
    # sequence with max_blocks = 64; the oracle evaluates a spread of beams on every block.
    d = configs.config_data("C2")
    plan, pb = make("ula", 256, 1, 256, 1, 256, 0.5, max_blocks=64)
    got = run(plan, "execute", d["y"], (64, 256, 256), 64)
    beams = np.array([0, 1, 37, 64, 127, 128, 200, 254, 255])
    ref = O.fbst(pb, d["y"], beams=beams)
    assert O.rel_l2(got[:, beams], ref) < TOL_E2E
    assert per_beam_err(got[:, beams], ref) < TOL_E2E
    assert np.isfinite(got).all()


def test_execute_c3_ura_sampled_beams():
    d = configs.config_data("C3", nblk=2, Q=64)
    plan, pb = make("ura", 32, 32, 32, 32, 512, 0.3, max_blocks=2)
    got = run(plan, "execute", d["y"], (2, 1024, 512), 2)
    beams = np.array([0, 31, 32, 500, 528, 777, 1023])
    ref = O.fbst(pb, d["y"], beams=beams)
    assert O.rel_l2(got[:, beams], ref) < TOL_E2E
    assert per_beam_err(got[:, beams], ref) < TOL_E2E
    assert np.isfinite(got).all()


@pytest.mark.parametrize("case", [("ula", 13, 1, 10, 1, 24, 0.37), ("ula", 1, 1, 1, 1, 16, 0.5),
                                  ("ula", 33, 1, 7, 1, 50, 1.2), ("ura", 3, 5, 3, 5, 20, 0.45)])
def test_execute_ragged_and_degenerate(rng, case):
    kind, mx, my, bx, by, N, fbw = case
    plan, pb = make(kind, mx, my, bx, by, N, fbw)
    y = crandn(rng, 5, pb.M, N)
    got = run(plan, "execute", y, (5, pb.B, N), 5)
    assert O.rel_l2(got, O.fbst(pb, y)) < TOL_E2E


def test_chunking_host_path_and_determinism(rng):
    y = crandn(rng, 7, 40, 64)
    p1, pb = make("ula", 40, 1, 24, 1, 64, 0.5, max_blocks=64)
    p2, _ = make("ula", 40, 1, 24, 1, 64, 0.5, max_blocks=3)
    a = run(p1, "execute", y, (7, 24, 64), 7)
    b = run(p2, "execute", y, (7, 24, 64), 7)
    c = run(p1, "execute", y, (7, 24, 64), 7)
    assert np.array_equal(a, b) and np.array_equal(a, c)
    host_out = np.full((7, 24, 64), np.nan, dtype=np.complex64)
    p2.execute_host(np.ascontiguousarray(y), host_out, 7)
    assert np.array_equal(a, host_out)
    assert O.rel_l2(a, O.fbst(pb, y)) < TOL_E2E


@pytest.mark.parametrize("stage2", ["gs_ir1", "dense_tf32x3", "dense_f16x3", "dense_fp32"])
def test_pipelined_host_path_equals_device_path(rng, stage2):
    # fbst_execute_host overlaps its copies with the kernels: stage 1 and the copies in run in block
    # parts; stage 2 and the copies out run in block parts (Gohberg-Semencul), in beam ranges with
    # strided copies (TF32x3) or in one piece (other dense variants). Every part computes exactly
    # what the device path computes, so the results are bitwise equal. 7 blocks in chunks of 3: the
    # parts are uneven and the beam count (37) does not split evenly.
    y = crandn(rng, 7, 40, 96)
    p, pb = make("ula", 40, 1, 37, 1, 96, 0.45, stage2=stage2, max_blocks=3)
    a = run(p, "execute", y, (7, 37, 96), 7)
    host_out = np.full((7, 37, 96), np.nan, dtype=np.complex64)
    p.execute_host(np.ascontiguousarray(y), host_out, 7)
    assert p.sync_status() == 0
    assert np.array_equal(a, host_out)
    assert O.rel_l2(host_out, O.fbst(pb, y)) < TOL_E2E


@pytest.mark.parametrize("stage2", ["gs_ir1", "dense_tf32x3", "dense_f16x3"])
def test_host_path_with_pinned_output_writes_in_place(rng, stage2):
    # A pinned output buffer is written by stage 2 through its device address (no copy out).
    y = crandn(rng, 7, 40, 96)
    p, pb = make("ula", 40, 1, 37, 1, 96, 0.45, stage2=stage2, max_blocks=3)
    a = run(p, "execute", y, (7, 37, 96), 7)
    y_pin = torch.from_numpy(np.ascontiguousarray(y)).pin_memory()
    out_pin = torch.full((7, 37, 96), float("nan"), dtype=torch.complex64).pin_memory()
    p.execute_host(y_pin, out_pin, 7)
    assert p.sync_status() == 0
    assert np.array_equal(a, out_pin.numpy())


def test_zero_blocks_is_a_noop_and_bad_args_raise():
    fb = _fb()
    plan, _ = make("ula", 16, 1, 16, 1, 64, 0.5)
    out = nan_like((1, 16, 64))
    plan.execute(0, out, 0)
    torch.cuda.synchronize()
    assert torch.isnan(out.real).all()
    with pytest.raises(fb.FBSTError):
        plan.execute(0, out, 1)          # null input
    with pytest.raises(fb.FBSTError):
        plan.execute(out, out, -1)


def test_on_grid_plane_wave_is_reproduced_on_gpu():
    from synth import Source, array_record, waveform
    rs = np.random.default_rng(7)
    plan, pb = make("ula", 32, 1, 32, 1, 64, 0.5)
    b = 21
    Q = 64
    src = Source(pb.directions[b, 0], 0.0, (rs.standard_normal(Q) + 1j * rs.standard_normal(Q)) * np.sqrt(0.5 / Q),
                 rs.uniform(-0.5, 0.5, Q))
    y = array_record(pb.geom, [src], 0.5, 64, None, None)[None].astype(np.complex64)
    got = run(plan, "execute", y, (1, 32, 64), 1)
    assert O.rel_l2(got[0, b], waveform(src, np.arange(64))) < 1e-2


TC_TOL = {"dense_tf32x3": TOL_E2E, "dense_f16x3": TOL_E2E, "dense_bf16x3": 1e-3, "dense_tf32": 3e-2}


@pytest.mark.parametrize("stage2", ["dense_tf32x3", "dense_f16x3", "dense_bf16x3", "dense_tf32"])
@pytest.mark.parametrize("case", [("ula", 16, 1, 16, 1, 64, 0.5, 3), ("ula", 13, 1, 10, 1, 24, 0.37, 5),
                                  ("ura", 8, 8, 8, 8, 64, 0.3, 2), ("ula", 48, 1, 40, 1, 256, 0.5, 70),
                                  ("ula", 40, 1, 160, 1, 200, 0.45, 27)])
def test_dense_tensor_core_matches_oracle(rng, stage2, case):
    # Tensor-core dense apply (tcgen05, TMA, TMEM). The first cases have N < 128 (row tiles partly
    # outside G_b) and up to 16 blocks (single-tile CTAs for TF32x3). 70 blocks: two block groups of
    # 64 (persistent TF32x3 CTAs), 2 row tiles. 27 blocks: one partial group of 32, N = 200 (a
    # partial second row tile), L = 400 (a partial last K chunk of 32) and 320 tiles, more than
    # the SMs, so persistent CTAs walk several tiles.
    kind, mx, my, bx, by, N, fbw, nblk = case
    plan, pb = make(kind, mx, my, bx, by, N, fbw, stage2=stage2, max_blocks=nblk)
    y = crandn(rng, nblk, pb.M, N)
    w = O.fan_coefficients(pb, y).astype(np.complex64)
    got = run(plan, "toeplitz_apply", w, (nblk, pb.B, N), nblk)
    assert plan.sync_status() == 0
    ref = O.Stage2Factors(pb).apply(w)
    err = O.rel_l2(got, ref)
    assert err < TC_TOL[stage2], f"{stage2}: {err:.3e}"


def test_execute_c3_precision_split_sampled_beams():
    # Config C3: URA 32x32, N = 512, B = 32x32, fb = 0.3; stage 2 on the tensor cores, each variant's
    # error against the FP64 oracle printed. Bars: 1e-5 for TF32x3 (FP32-class: split operands and
    # the K loop split over several tensor-memory accumulators), 1e-3 for BF16x3 (the tensor-core
    # bar) and 3e-2 for plain TF32.
    d = configs.config_data("C3", nblk=4, Q=64)
    beams = np.array([0, 33, 500, 777, 1023])
    errs, ref = {}, None
    for stage2 in ("dense_tf32x3", "dense_f16x3", "dense_bf16x3", "dense_tf32"):
        plan, pb = make("ura", 32, 32, 32, 32, 512, 0.3, stage2=stage2, max_blocks=4)
        got = run(plan, "execute", d["y"], (4, 1024, 512), 4)
        assert plan.sync_status() == 0
        if ref is None:
            ref = O.fbst(pb, d["y"], beams=beams)
        errs[stage2] = O.rel_l2(got[:, beams], ref)
        plan.close()
    print("C3 rel L2 error vs FP64 oracle:", {k: f"{v:.2e}" for k, v in errs.items()})
    assert errs["dense_tf32x3"] < TOL_E2E and errs["dense_f16x3"] < TOL_E2E, errs
    assert errs["dense_bf16x3"] < 1e-3 and errs["dense_tf32"] < 3e-2, errs


def test_execute_c2_full_size_tf32x3_sampled_beams():
    # The benchmark's headline configuration: C2 (64 blocks in one launch sequence) with the
    # FP32-class tensor-core stage 2; beams spread over the grid, every block.
    d = configs.config_data("C2")
    plan, pb = make("ula", 256, 1, 256, 1, 256, 0.5, stage2="dense_tf32x3", max_blocks=64)
    got = run(plan, "execute", d["y"], (64, 256, 256), 64)
    assert plan.sync_status() == 0
    beams = np.array([0, 1, 37, 64, 127, 128, 200, 254, 255])
    ref = O.fbst(pb, d["y"], beams=beams)
    assert O.rel_l2(got[:, beams], ref) < TOL_E2E
    assert per_beam_err(got[:, beams], ref) < TOL_E2E
    assert np.isfinite(got).all()


@pytest.mark.parametrize("stage2", ["dense_tf32x3", "dense_f16x3", "dense_bf16x3"])
def test_tensor_core_wait_that_runs_out_reports_timeout_and_recovers(rng, stage2):
    # Failure detection without a fault: a wait limit of 1 ns makes the pipeline waits of the
    # tensor-core kernel run out (nothing can complete that fast). The kernel must record
    # FBST_ERR_TIMEOUT, drain its own copies and MMAs, free tensor memory and return; the status is
    # read and cleared by fbst_sync_status, and the next call with the default limit is correct.
    plan, pb = make("ula", 64, 1, 64, 1, 512, 0.5, stage2=stage2, max_blocks=16)
    y = crandn(rng, 16, 64, 512)
    w = O.fan_coefficients(pb, y[:2]).astype(np.complex64)
    wd = dev(np.concatenate([w, np.zeros((14,) + w.shape[1:], np.complex64)]))
    out = nan_like((16, 64, 512))
    plan.set_wait_limit(1)
    plan.toeplitz_apply(wd, out, 16)
    assert plan.sync_status() == -5                    # FBST_ERR_TIMEOUT
    assert plan.sync_status() == 0                     # read and cleared
    plan.set_wait_limit(0)
    out2 = nan_like((16, 64, 512))
    plan.toeplitz_apply(wd, out2, 16)
    assert plan.sync_status() == 0
    got = out2.cpu().numpy()[:2]
    assert O.rel_l2(got, O.Stage2Factors(pb).apply(w)) < TC_TOL[stage2]


def test_f16x3_block_scales_keep_accuracy_across_magnitudes(rng):
    # The FP16 split scales G per beam and w per block by powers of two chosen from their largest
    # magnitudes, so every block keeps FP32-class accuracy however large or small it is, in one
    # call with blocks 50 orders of magnitude apart and an all-zero block (scale 1, output 0).
    plan, pb = make("ula", 48, 1, 40, 1, 256, 0.5, stage2="dense_f16x3", max_blocks=6)
    y = crandn(rng, 6, 48, 256)
    w = O.fan_coefficients(pb, y).astype(np.complex64)
    mags = np.array([1e-25, 1e-3, 1.0, 1e3, 1e25, 0.0], dtype=np.float32)
    ws = (w * mags[:, None, None]).astype(np.complex64)
    got = run(plan, "toeplitz_apply", ws, (6, pb.B, 256), 6)
    assert plan.sync_status() == 0
    ref = O.Stage2Factors(pb).apply(w)
    for i, m in enumerate(mags):
        if m == 0:
            assert not got[i].any()
        else:
            err = O.rel_l2(got[i] / np.float64(m), ref[i])
            assert err < TOL_E2E, f"block scaled by {m:g}: {err:.3e}"


@pytest.mark.parametrize("case", [("ula", 48, 1, 40, 1, 256, 0.5, 5), ("ura", 8, 8, 8, 8, 64, 0.3, 3)])
def test_f16x3_block_scales_from_stage1_equal_separate_pass(rng, case):
    # On a linear array the spatial chirp-z finds each block's largest |re|, |im| as it writes w, and
    # stage 2 uses it; toeplitz_apply on the same w finds it with a pass of its own. The maximum is
    # exact either way, so both give the same scales and bitwise the same output. (A rectangular
    # array takes the separate pass in both.) Chunks of 2 blocks: each chunk has its own maxima.
    kind, mx, my, bx, by, N, fbw, nblk = case
    plan, pb = make(kind, mx, my, bx, by, N, fbw, stage2="dense_f16x3", max_blocks=2)
    y = crandn(rng, nblk, pb.M, N)
    a = run(plan, "execute", y, (nblk, pb.B, N), nblk)
    w = run(plan, "czt", y, (nblk, pb.B, pb.L), nblk)
    b = run(plan, "toeplitz_apply", w, (nblk, pb.B, N), nblk)
    assert plan.sync_status() == 0
    assert np.array_equal(a, b)
    assert O.rel_l2(a, O.fbst(pb, y)) < TOL_E2E
    chunks = (nblk + 1) // 2
    assert plan.launch_count(nblk) == chunks * (2 + (1 if kind == "ula" else 2))
