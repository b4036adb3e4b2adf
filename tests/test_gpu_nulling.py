"""Parity of the beamspace interference nulling (Sec. VIII-B, Eq. (14)) through the C ABI with the
FP64 oracle, on seeded scenes with interferers 20 dB above the source.

The library applies the bracket of Eq. (14) as w_b - sum_p G_{b,p} w_p with G_{b,p} = F_b^H F_p
A_p^{-1} built once in FP64 and rounded to complex64, contracted in FP32 on the CUDA cores (products
rounded to 2^-24) or on the tensor cores in split TF32 (hi*hi + hi*lo + lo*hi with lo truncated to
TF32 by the MMA: about 2^-21 per product). The correction sum_p G_{b,p} w_p is a sum of P*L terms of
the size of w_p whose total is the interferer's share of w_b, and what remains after the
subtraction is about a tenth of w_b at 20 dB: the rounding of the terms, not of the result, sets
the error. So each contraction is compared with a model of its own arithmetic (bracket_model
below: the oracle's FP64 matrices with the GPU's roundings, in numpy, on the same input), and the
bars, fixed before the measurement, are:

* FP32 contraction (the default): the bracket (fbst_null_apply, on the oracle's w rounded to
  complex64) within 2x of the model over the array (error / ||w||) and within 3x per beam
  (error_b / max(|w_b|, rms_b |w_b|), a maximum over beams and so a noisier statistic); end to end
  (fbst_null_execute from y, the model adding a stage-1 perturbation of the measured FP32 stage-1
  size, 2.5e-7) within 2x of the model relative to the nulled output;
* both contractions, end to end: within the transform's own bar, 1e-5, relative to the plain
  output of the same input (the scale every rounding is taken at). The tensor cores accumulate in
  FP32 without IEEE round-to-nearest semantics, which the model does not describe, so for the
  split-TF32 contraction the model figure is printed, not asserted.
Outputs are poisoned with NaN first.
"""
import numpy as np
import pytest

import oracle as O
from synth import configs, interference_config

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_E2E = 1e-5           # of the plain transform's output
MODEL_GLOBAL = 2.0       # GPU error <= 2 x the model's (array-wide figures)
MODEL_PER_BEAM = 3.0     # GPU error <= 3 x the model's (maximum over beams)
STAGE1_REL = 2.5e-7      # measured relative error of the FP32 stage 1, for the end-to-end model


def _tf32(x, rna):
    """float32 -> TF32 (10 stored mantissa bits): round to nearest, ties away (cvt.rna), or truncate
    (what the tensor core does with the low bits of an FP32 register)."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    b = ((b + np.uint32(0x1000)) if rna else b) & np.uint32(0xFFFFE000)
    return b.view(np.float32)


def _contract(rhs, G, contraction):
    """rhs (n, K) complex64 times G^T (G: (L, K) complex64) with the GPU kernel's roundings."""
    if contraction == "fp32":
        # The CUDA-core kernel sums every K chunk of 32 in FP32, then adds the chunk sums in FP32.
        acc = np.zeros((rhs.shape[0], G.shape[0]), np.complex64)
        for k0 in range(0, G.shape[1], 32):
            acc = (acc + (rhs[:, k0:k0 + 32] @ G[:, k0:k0 + 32].T).astype(np.complex64)).astype(np.complex64)
        return acc

    def prod(a, b):                                    # real (n, K) x (K, L), split TF32
        ah, bh = _tf32(a, True), _tf32(b, True)
        al, bl = _tf32(a - ah, False), _tf32(b - bh, False)
        return (ah @ bh).astype(np.float32) + ((ah @ bl) + (al @ bh)).astype(np.float32)

    A = G.T
    re = prod(rhs.real, A.real) - prod(rhs.imag, A.imag)
    im = prod(rhs.real, A.imag) + prod(rhs.imag, A.real)
    return (re + 1j * im).astype(np.complex64)


def bracket_model(pb, w32, ints, beams, contraction):
    """The bracket of Eq. (14) with the GPU's roundings: G_{b,p} from the oracle's FP64 matrices
    rounded to complex64, the contraction of `contraction`, the subtraction in complex64.
    w32: (nblk, B, L) complex64; returns (nblk, len(beams), L) complex64."""
    rhs = w32[:, ints].reshape(w32.shape[0], -1)
    ainv = [np.linalg.inv(O.gram(pb, p)) for p in ints]
    out = np.empty((w32.shape[0], len(beams), pb.L), np.complex64)
    for i, b in enumerate(beams):
        G = np.concatenate([O.cross_gram(pb, b, p) @ a for p, a in zip(ints, ainv)], axis=1).astype(np.complex64)
        out[:, i] = w32[:, b] - _contract(rhs, G, contraction)
    return out


def _per_beam(err, ref):
    e = np.linalg.norm(err, axis=(0, 2))
    n = np.linalg.norm(ref, axis=(0, 2))
    return float(np.max(e / np.maximum(n, np.sqrt(np.mean(n ** 2)))))


def e2e_model_error(pb, y, ints, beams, contraction):
    """Relative error (to the nulled output) of the FP32 pipeline model: w with a stage-1-sized
    perturbation (seeded), rounded to complex64, the bracket model, then the FP64 stage 2."""
    fac = O.NullingFactors(pb, ints, beams)
    w64 = O.fan_coefficients(pb, y)
    ref = fac.out.apply(fac.coefficients(w64[:, beams], w64[:, ints]))
    g = np.random.default_rng(123)
    col = np.linalg.norm(w64, axis=1, keepdims=True) / np.sqrt(pb.B)
    w32 = (w64 + STAGE1_REL * col * (g.standard_normal(w64.shape) + 1j * g.standard_normal(w64.shape))
           / np.sqrt(2)).astype(np.complex64)
    got = fac.out.apply(bracket_model(pb, w32, ints, beams, contraction).astype(np.complex128))
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_08887_gb300.build import build
    build()


def _fb():
    import paper_2512_08887_gb300 as fb
    return fb


def make(kind, mx, my, bx, by, N, frac_bw, stage2="auto", max_blocks=64):
    fb = _fb()
    plan = fb.Plan(fb.make_geometry(kind, mx, my, bx, by), N,
                   fb.make_band(frac_bw, delta=1e-3, stage2=stage2, max_blocks=max_blocks))
    i = plan.info
    pb = O.make_problem(kind, mx, my, bx, by, N, frac_bw=i.fb_num / i.fb_den, epsilon=i.eps_num / i.eps_den,
                        delta=i.delta, L=i.L)
    return plan, pb


def scene(pb, kind, mx, my, N, frac_bw, ints, nblk, seed):
    """A unit source half a grid away from the first interferer, interferers on grid beams at 20 dB."""
    dirs = pb.directions
    src = tuple(dirs[(ints[0] + pb.B // 2) % pb.B])
    return interference_config(kind, mx, my, N, nblk, frac_bw, [src], [tuple(dirs[p]) for p in ints],
                               20.0, 10.0, seed, Q=64)["y"]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def nan_like(shape):
    return torch.full(shape, complex(np.nan, np.nan), dtype=torch.complex64, device="cuda")


CASES = [
    ("ula", 16, 1, 16, 1, 64, 0.5, [5]),              # L = 128
    ("ula", 40, 1, 48, 1, 96, 0.45, [3, 30]),         # L = 192: 1.5 row tiles of 128, B not a multiple of 16
    ("ura", 4, 4, 4, 4, 32, 0.3, [5]),                # rectangular array, both axis factors
    ("ula", 24, 1, 24, 1, 40, 0.5, [0, 11, 23]),      # three interferers, grid edges, L = 80
]


@pytest.mark.parametrize("contraction", ["tf32x3", "fp32"])
@pytest.mark.parametrize("case", CASES)
def test_bracket_of_eq14_matches_oracle(case, contraction):
    kind, mx, my, bx, by, N, fb_, ints = case
    plan, pb = make(kind, mx, my, bx, by, N, fb_, max_blocks=2)
    nblk = 3                                           # two chunks, the second ragged
    y = scene(pb, kind, mx, my, N, fb_, ints, nblk, 77)
    w = O.fan_coefficients(pb, y).astype(np.complex64)
    with _fb().Nulling(plan, ints, contraction) as nl:
        out = nan_like((nblk, pb.B, pb.L))
        nl.apply(dev(w), out, nblk)
        assert plan.sync_status() == 0
    got = out.cpu().numpy()
    w64 = w.astype(np.complex128)
    ref = O.NullingFactors(pb, ints).coefficients(w64, w64[:, ints])
    model = bracket_model(pb, w, ints, list(range(pb.B)), contraction).astype(np.complex128)
    err, m_err = np.linalg.norm(got - ref) / np.linalg.norm(w64), np.linalg.norm(model - ref) / np.linalg.norm(w64)
    per, m_per = _per_beam(got - ref, w64), _per_beam(model - ref, w64)
    print(f"bracket {kind}{mx} {contraction}: {err:.2e} of ||w|| (model {m_err:.2e}), per beam {per:.2e} "
          f"(model {m_per:.2e})")
    if contraction == "fp32":
        assert err <= MODEL_GLOBAL * m_err, (err, m_err)
        assert per <= MODEL_PER_BEAM * m_per, (per, m_per)


def test_bracket_in_place_equals_out_of_place():
    plan, pb = make("ula", 40, 1, 48, 1, 96, 0.45)
    y = scene(pb, "ula", 40, 1, 96, 0.45, [3, 30], 2, 5)
    w = dev(O.fan_coefficients(pb, y).astype(np.complex64))
    with _fb().Nulling(plan, [3, 30]) as nl:
        out = nan_like(tuple(w.shape))
        nl.apply(w, out, 2)
        nl.apply(w, w, 2)
        torch.cuda.synchronize()
    assert torch.equal(out, w)


@pytest.mark.parametrize("stage2", ["auto", "dense_tf32x3", "dense_f16x3"])
@pytest.mark.parametrize("contraction", ["tf32x3", "fp32"])
@pytest.mark.parametrize("case", CASES[:3])
def test_nulled_transform_matches_oracle(case, contraction, stage2):
    kind, mx, my, bx, by, N, fb_, ints = case
    plan, pb = make(kind, mx, my, bx, by, N, fb_, stage2=stage2, max_blocks=2)
    nblk = 3
    y = scene(pb, kind, mx, my, N, fb_, ints, nblk, 91)
    with _fb().Nulling(plan, ints, contraction) as nl:
        out = nan_like((nblk, pb.B, N))
        nl.execute(dev(y), out, nblk)
        assert plan.sync_status() == 0
        # the nulled w was not written by stage 1b, so the FP16 split finds its block scales itself
        assert nl.launch_count(nblk) == 2 * (5 + (1 if stage2 in ("auto", "dense_tf32x3") else 2))
        # the plain transform's own stage 1b writes them on a linear array, so its stage 2 is one launch
        assert plan.launch_count(nblk) == 2 * (2 + (2 if stage2 == "dense_f16x3" and kind != "ula" else 1))
    got = out.cpu().numpy()
    ref = O.fbst_nulled(pb, y, ints)
    err = np.linalg.norm(got - ref) / np.linalg.norm(O.fbst(pb, y))
    rel, model = O.rel_l2(got, ref), e2e_model_error(pb, y, ints, list(range(pb.B)), contraction)
    print(f"nulled {case[0]}{case[1]} {contraction} {stage2}: {err:.2e} of plain, {rel:.2e} of nulled "
          f"(model {model:.2e})")
    assert err < TOL_E2E, (err, rel)
    if contraction == "fp32":
        assert rel <= MODEL_GLOBAL * model, (rel, model)


def test_interferer_removed_on_the_gpu():
    # Physics through the CUDA path: a plane wave from a grid beam is removed from every beam.
    M, N, nblk = 16, 64, 4
    plan, pb = make("ula", M, 1, M, 1, N, 0.5)
    y = interference_config("ula", M, 1, N, nblk, 0.5, [], [tuple(pb.directions[4])], 20.0, None, 3, Q=64)["y"]
    plain = nan_like((nblk, M, N))
    nul = nan_like((nblk, M, N))
    plan.execute(dev(y), plain, nblk)
    with _fb().Nulling(plan, [4]) as nl:
        nl.execute(dev(y), nul, nblk)
    torch.cuda.synchronize()
    ratio = float(torch.linalg.vector_norm(nul) / torch.linalg.vector_norm(plain))
    assert ratio < 2e-2, ratio


def test_full_size_workload_on_sampled_beams():
    # The benchmark's launch configuration: the 256-element ULA, 256 beams, N = 256, 64 blocks per
    # call, interferers on beams 64 and 96, tensor-core stage 2 and contraction. Checked against the
    # oracle on 2 blocks for the interferer beams, their neighbours, the source beam and an edge beam.
    c = configs.NULLING["C2N"]
    d = configs.nulling_data("C2N")
    plan, pb = make("ula", 256, 1, 256, 1, 256, 0.5, stage2="dense_tf32x3", max_blocks=64)
    contraction = "fp32"
    with _fb().Nulling(plan, c["interferers"], contraction) as nl:
        out = nan_like((64, 256, 256))
        nl.execute(dev(d["y"]), out, 64)
        assert plan.sync_status() == 0
    got = out.cpu().numpy()
    assert np.isfinite(got).all()
    beams = [63, 64, 65, 96, 160, 255]
    ref = O.fbst_nulled(pb, d["y"][:2], c["interferers"], beams=beams)
    err = np.linalg.norm(got[:2, beams] - ref) / np.linalg.norm(O.fbst(pb, d["y"][:2], beams=beams))
    rel, model = O.rel_l2(got[:2, beams], ref), e2e_model_error(pb, d["y"][:2], c["interferers"], beams, contraction)
    print(f"C2N: {err:.2e} of plain, {rel:.2e} of nulled (model {model:.2e})")
    assert err < TOL_E2E, (err, rel)
    if contraction == "fp32":
        assert rel <= MODEL_GLOBAL * model, (rel, model)


def test_invalid_arguments_are_rejected():
    fb = _fb()
    plan, pb = make("ula", 16, 1, 16, 1, 64, 0.5)
    for ints in ([], [16], [-1], [3, 3], list(range(17))):
        with pytest.raises(fb.FBSTError) as e:
            fb.Nulling(plan, ints)
        assert e.value.status == -1
    with fb.Nulling(plan, [2]) as nl:
        y = torch.zeros((1, 16, 64), dtype=torch.complex64, device="cuda")
        out = torch.zeros((1, 16, 64), dtype=torch.complex64, device="cuda")
        raw = torch.zeros(16 * 64 * 2 + 4, dtype=torch.float32, device="cuda")
        with pytest.raises(fb.FBSTError):
            nl.execute(raw.data_ptr() + 4, out, 1)      # misaligned input: rejected, nothing launched
        nl.execute(y, out, 0)                            # empty call is a no-op
        assert nl.launch_count(0) == 0
        assert plan.sync_status() == 0


OFFGRID_CASES = [("ula", 16, 1, 32, 1, 64, 0.5, [[-0.3, 0.0]]), ("ula", 40, 1, 80, 1, 96, 0.45, [[0.11, 0.0], [-0.52, 0.0]]),
                 ("ura", 4, 4, 8, 8, 32, 0.3, [[0.2, -0.33]])]


@pytest.mark.parametrize("contraction", ["fp32", "tf32x3"])
@pytest.mark.parametrize("case", OFFGRID_CASES)
def test_offgrid_interferers_match_oracle(case, contraction):
    # Interferers between grid beams (Sec. VIII-B: no alignment with the grid needed): their vectors
    # interpolated from the grid (Sec. VIII-A), G from their own F_p. The bracket on the oracle's w
    # within 2e-6 of ||w|| (the grid-interferer bracket measures 2.4-9.3e-7 with the same arithmetic),
    # end to end within the transform's 1e-5 of the plain output.
    kind, mx, my, bx, by, N, fb_, dirs = case
    plan, pb = make(kind, mx, my, bx, by, N, fb_, max_blocks=2)
    nblk = 3
    src = tuple(pb.directions[(pb.B // 2 + 3) % pb.B])
    y = interference_config(kind, mx, my, N, nblk, fb_, [src], [tuple(d) for d in dirs], 20.0, 10.0, 19, Q=64)["y"]
    fac = O.OffGridNullingFactors(pb, dirs)
    w = O.fan_coefficients(pb, y).astype(np.complex64)
    w64 = w.astype(np.complex128)
    with _fb().Nulling(plan, contraction=contraction, directions=dirs) as nl:
        out = nan_like((nblk, pb.B, pb.L))
        nl.apply(dev(w), out, nblk)
        full = nan_like((nblk, pb.B, N))
        nl.execute(dev(y), full, nblk)
        assert plan.sync_status() == 0
    ref_br = fac.coefficients(w64, w64)
    err_br = np.linalg.norm(out.cpu().numpy() - ref_br) / np.linalg.norm(w64)
    ref = O.fbst_nulled_offgrid(pb, y, dirs)
    got = full.cpu().numpy()
    err = np.linalg.norm(got - ref) / np.linalg.norm(O.fbst(pb, y))
    print(f"off-grid nulling {kind}{mx} {contraction}: bracket {err_br:.2e} of ||w||, {err:.2e} of plain, "
          f"{O.rel_l2(got, ref):.2e} of nulled")
    assert err_br < 2e-6 and err < TOL_E2E


def test_offgrid_interferer_is_removed_on_the_gpu():
    M, N, nblk = 16, 64, 4
    plan, pb = make("ula", M, 1, 2 * M, 1, N, 0.5)
    u = pb.directions[10, 0] + 1.0 / pb.B                # halfway between two grid beams
    y = interference_config("ula", M, 1, N, nblk, 0.5, [], [(u, 0.0)], 20.0, None, 4, Q=64)["y"]
    plain = nan_like((nblk, 2 * M, N))
    plan.execute(dev(y), plain, nblk)
    with _fb().Nulling(plan, directions=[[u, 0.0]]) as nl:
        nul = nan_like((nblk, 2 * M, N))
        nl.execute(dev(y), nul, nblk)
    with _fb().Nulling(plan, [10]) as nl:
        near = nan_like((nblk, 2 * M, N))
        nl.execute(dev(y), near, nblk)
    torch.cuda.synchronize()
    p = float(torch.linalg.vector_norm(plain))
    ratio, r_near = float(torch.linalg.vector_norm(nul)) / p, float(torch.linalg.vector_norm(near)) / p
    print(f"off-grid interferer left: {ratio:.3f} (nearest grid beam nulled instead: {r_near:.3f})")
    assert ratio < 0.1 and ratio < r_near / 3


def test_grid_directions_give_the_grid_nulling():
    plan, pb = make("ula", 24, 1, 24, 1, 64, 0.5, max_blocks=2)
    ints = [5, 17]
    y = scene(pb, "ula", 24, 1, 64, 0.5, ints, 2, 8)
    with _fb().Nulling(plan, ints) as a, _fb().Nulling(plan, directions=pb.directions[ints]) as b:
        oa, ob = nan_like((2, 24, 64)), nan_like((2, 24, 64))
        a.execute(dev(y), oa, 2)
        b.execute(dev(y), ob, 2)
    torch.cuda.synchronize()
    plain = O.fbst(pb, y)
    assert float(torch.linalg.vector_norm(oa - ob)) / np.linalg.norm(plain) < 1e-6
