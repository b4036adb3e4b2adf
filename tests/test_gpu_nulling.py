"""Parity of the beamspace interference nulling (Sec. VIII-B, Eq. (14)) through the C ABI with the
FP64 oracle, on seeded scenes with interferers 20 dB above the source.

Tolerances, from the arithmetic. Eq. (14) subtracts from each w_b the interferer's projected
component (Sec. VIII-B derives it from the array-space projection y - F_p (F_p^H F_p + delta I)^{-1}
F_p^H y), a correction as large as the interferer's contribution. FP32 errors are therefore set by
the size of the operands, not of the (much smaller) difference, and are measured here against the
input scale.

* The bracket of Eq. (14) (fbst_null_apply, on the oracle's w rounded to complex64): the stored
  operands are complex64 (cross Gram matrices; A_p^{-1} w_p computed in FP64, then rounded) and the
  contraction accumulates in FP32 over P*L terms of split-TF32 products (2^-21 relative each). An
  emulation of the complex64 roundings gives at most 3e-7 of |w_b| on any beam; the bound is 5e-6
  of |w_b| per beam and of ||w|| over the array.
* End to end (fbst_null_execute from y): stage 1 leaves FP32 errors in w_b and w_p that no longer
  cancel once the interferer is subtracted, so the nulled output inherits the plain transform's
  absolute error. The bar is the transform's own, 1e-5, relative to the plain transform's output
  of the same input (an emulation with stage-1-sized errors: 5e-7 of the plain output, 2e-6 of the
  nulled one, with interferers 20 dB above the source).
Outputs are poisoned with NaN first.
"""
import numpy as np
import pytest

import oracle as O
from synth import configs, interference_config

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_BRACKET = 5e-6       # of ||w||
TOL_BRACKET_BEAM = 5e-6  # of |w_b|
TOL_E2E = 1e-5           # of the plain transform's output


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
    err = np.linalg.norm(got - ref) / np.linalg.norm(w64)
    per = np.linalg.norm(got - ref, axis=(0, 2)) / np.linalg.norm(w64, axis=(0, 2))
    assert err < TOL_BRACKET, (err, O.rel_l2(got, ref))
    assert per.max() < TOL_BRACKET_BEAM, (per.max(), int(per.argmax()))


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


@pytest.mark.parametrize("stage2", ["auto", "dense_tf32x3"])
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
        assert nl.launch_count(nblk) == 2 * (5 + (1 if stage2 in ("auto", "dense_tf32x3") else 2))
    got = out.cpu().numpy()
    ref = O.fbst_nulled(pb, y, ints)
    err = np.linalg.norm(got - ref) / np.linalg.norm(O.fbst(pb, y))
    assert err < TOL_E2E, (err, O.rel_l2(got, ref))


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
    with _fb().Nulling(plan, c["interferers"]) as nl:
        out = nan_like((64, 256, 256))
        nl.execute(dev(d["y"]), out, 64)
        assert plan.sync_status() == 0
    got = out.cpu().numpy()
    assert np.isfinite(got).all()
    beams = [63, 64, 65, 96, 160, 255]
    ref = O.fbst_nulled(pb, d["y"][:2], c["interferers"], beams=beams)
    err = np.linalg.norm(got[:2, beams] - ref) / np.linalg.norm(O.fbst(pb, d["y"][:2], beams=beams))
    assert err < TOL_E2E, (err, O.rel_l2(got[:2, beams], ref))


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
