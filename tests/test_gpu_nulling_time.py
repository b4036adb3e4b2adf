"""Parity of the time-domain interference nulling (Sec. VIII-B, Eq. (15)) through the C ABI with the
FP64 oracle, on seeded scenes with interferers 20 dB above the source.

The library applies G'_{b,p} = F_u A_b^{-1} (F_b^H F_p) F_x^+ factor by factor to the interferer
beams y_p over the broader interval of 2L samples (F_x^+ built in FP64 and rounded once, the cross Gram
contraction in FP32 or split TF32, then the plan's own stage 2) and subtracts the result from the
plain beams in FP32. The interferer beams of the end-to-end path are summed in FP64 from
F_x A_p^{-1} w_p: that operator's entries are of the size of ||A_p^{-1}|| and cancel down to the
beam (an FP32 sum measured 1.7e-4 to 5.6e-3 of the plain output on these cases). The correction is the interferer's share of each beam, about ten times
what remains, so, as for Eq. (14), the bar is the transform's own, 1e-5, relative to the plain
output of the same input; the error relative to the nulled output is printed. Cases:

* fbst_null_apply_time on the oracle's own time-domain beams (plain beams over the block and
  interferer beams over the broader interval, rounded to complex64);
* fbst_null_execute of a time-domain object from y, end to end, against the oracle's Eq. (15);
* the GPU's Eq. (15) against its Eq. (14) on the same input (equal in exact arithmetic);
* the C2NT size (256-element ULA, L = 512: the broader interval must be 2L samples there, see the
  oracle's pins) on two blocks;
* argument checks: the bracket entry point refuses a time-domain object, and a plan whose N is odd
  is refused at creation.
Outputs are poisoned with NaN first.
"""
import numpy as np
import pytest

import oracle as O
from synth import interference_config

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_E2E = 1e-5   # of the plain transform's output


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
    dirs = pb.directions
    src = tuple(dirs[(ints[0] + pb.B // 2) % pb.B])
    return interference_config(kind, mx, my, N, nblk, frac_bw, [src], [tuple(dirs[p]) for p in ints],
                               20.0, 10.0, seed, Q=64)["y"]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def nan_like(shape):
    return torch.full(shape, complex(np.nan, np.nan), dtype=torch.complex64, device="cuda")


CASES = [
    ("ula", 16, 1, 16, 1, 64, 0.5, [5]),              # L = 128, one interferer
    ("ula", 40, 1, 48, 1, 96, 0.45, [3, 30]),         # L = 192, two interferers, B != M
    ("ura", 4, 4, 4, 4, 32, 0.3, [5]),                # rectangular array
]


@pytest.mark.parametrize("contraction", ["fp32", "tf32x3"])
@pytest.mark.parametrize("case", CASES)
def test_apply_time_on_oracle_beams(case, contraction):
    kind, mx, my, bx, by, N, fb_, ints = case
    plan, pb = make(kind, mx, my, bx, by, N, fb_, max_blocks=2)
    nblk = 3
    y = scene(pb, kind, mx, my, N, fb_, ints, nblk, 41)
    f = O.TimeNullingFactors(pb, ints)
    w = O.fan_coefficients(pb, y)
    plain = f.out.apply(w)                                   # (nblk, B, N)
    y_int = f.interferer_beams(w[:, ints])                   # (nblk, P, L)
    ref = f.apply(plain, y_int)
    with _fb().Nulling(plan, ints, contraction, time_domain=True) as nl:
        out = nan_like((nblk, pb.B, N))
        nl.apply_time(dev(plain.astype(np.complex64)), dev(y_int.astype(np.complex64)), out, nblk)
        assert plan.sync_status() == 0
    got = out.cpu().numpy()
    err = np.linalg.norm(got - ref) / np.linalg.norm(plain)
    print(f"apply_time {kind}{mx} {contraction}: {err:.2e} of plain, {O.rel_l2(got, ref):.2e} of nulled")
    assert np.isfinite(got).all()
    assert err < TOL_E2E


@pytest.mark.parametrize("stage2", ["auto", "dense_f16x3"])
@pytest.mark.parametrize("contraction", ["fp32", "tf32x3"])
@pytest.mark.parametrize("case", CASES)
def test_time_execute_matches_oracle(case, contraction, stage2):
    kind, mx, my, bx, by, N, fb_, ints = case
    plan, pb = make(kind, mx, my, bx, by, N, fb_, stage2=stage2, max_blocks=2)
    nblk = 3
    y = scene(pb, kind, mx, my, N, fb_, ints, nblk, 91)
    with _fb().Nulling(plan, ints, contraction, time_domain=True) as nl:
        out = nan_like((nblk, pb.B, N))
        nl.execute(dev(y), out, nblk)
        assert plan.sync_status() == 0
        s2 = lambda ready: 1 if stage2 == "auto" or (ready and kind == "ula") else 2
        assert nl.launch_count(nblk) == 2 * (2 + s2(True) + 4 + s2(False))
    got = out.cpu().numpy()
    ref = O.fbst_nulled_time(pb, y, ints)
    err = np.linalg.norm(got - ref) / np.linalg.norm(O.fbst(pb, y))
    print(f"time-domain nulled {kind}{mx} {contraction} {stage2}: {err:.2e} of plain, "
          f"{O.rel_l2(got, ref):.2e} of nulled")
    assert err < TOL_E2E


def test_time_form_equals_beamspace_form_on_gpu():
    plan, pb = make("ula", 40, 1, 48, 1, 96, 0.45, max_blocks=4)
    ints = [3, 30]
    y = scene(pb, "ula", 40, 1, 96, 0.45, ints, 4, 7)
    fb = _fb()
    a, b = nan_like((4, pb.B, 96)), nan_like((4, pb.B, 96))
    with fb.Nulling(plan, ints, "fp32", time_domain=True) as nt:
        nt.execute(dev(y), a, 4)
    with fb.Nulling(plan, ints, "fp32") as nb_:
        nb_.execute(dev(y), b, 4)
    torch.cuda.synchronize()
    plain = O.fbst(pb, y)
    d = np.linalg.norm(a.cpu().numpy() - b.cpu().numpy()) / np.linalg.norm(plain)
    print(f"Eq. (15) vs Eq. (14) on the GPU: {d:.2e} of plain")
    assert d < TOL_E2E


def test_time_form_argument_checks():
    fb = _fb()
    plan, pb = make("ula", 16, 1, 16, 1, 64, 0.5)
    with fb.Nulling(plan, [5], "fp32", time_domain=True) as nl:
        w = torch.zeros((1, pb.B, pb.L), dtype=torch.complex64, device="cuda")
        with pytest.raises(fb.FBSTError):
            nl.apply(w, w, 1)
    with fb.Nulling(plan, [5], "fp32") as nb_:
        y = torch.zeros((1, pb.B, 64), dtype=torch.complex64, device="cuda")
        yi = torch.zeros((1, 1, pb.L), dtype=torch.complex64, device="cuda")
        with pytest.raises(fb.FBSTError):
            nb_.apply_time(y, yi, y, 1)
    odd, _ = make("ula", 16, 1, 16, 1, 63, 0.5)   # N odd
    with pytest.raises(fb.FBSTError):
        fb.Nulling(odd, [5], "fp32", time_domain=True)


def test_time_form_at_the_c2_size():
    from synth import configs
    c = configs.NULLING["C2N"]
    plan, pb = make("ula", c["mx"], 1, c["bx"], 1, c["N"], c["frac_bw"], max_blocks=2)
    y = configs.nulling_data("C2N", nblk=2)["y"]
    beams = [0, 63, 64, 65, 96, 160, 255]
    with _fb().Nulling(plan, c["interferers"], "fp32", time_domain=True) as nl:
        out = nan_like((2, pb.B, pb.N))
        nl.execute(dev(y), out, 2)
        assert plan.sync_status() == 0
    got = out.cpu().numpy()[:, beams]
    ref = O.fbst_nulled_time(pb, y, c["interferers"], beams=beams)
    err = np.linalg.norm(got - ref) / np.linalg.norm(O.fbst(pb, y, beams=beams))
    print(f"C2NT size: {err:.2e} of plain, {O.rel_l2(got, ref):.2e} of nulled")
    assert err < TOL_E2E
