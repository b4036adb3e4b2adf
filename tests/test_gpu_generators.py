"""Parity of the superfast generator solver (Sec. V: x_b = A_b^{-1} e_0 in O(L log^2 L)) through the
C ABI with the FP64 oracle's dense solve of the Gram matrix it builds by direct sums (Eq. (5)).

The solver is the doubling form of the Schur algorithm with FP64 FFT polynomial products; it gives
the Levinson result up to rounding, so it is held to the Levinson test's bar (1e-9 relative to
the dense solve in FP64, for A_b of condition number about 2/delta_rel = 2e3). The shapes cover
each branch of the recursion: L - 1 <= 32 steps (the root is a leaf), a leaf of exactly 32 steps
(its degree-32 coefficient), a node whose FFT size equals its step count (the product's wrapped
coefficient), odd splits, rectangular and non-uniform arrays, the headline ULA1024 plan (sampled
beams) and the largest L = 2048 (FFT size 2048). Plans built with either solver give the same
transform, on the grid and off it.
"""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_X = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_08887_gb300.build import build
    build()


def _fb():
    import paper_2512_08887_gb300 as fb
    return fb


def make(kind, mx, my, bx, by, N, frac_bw, solver, stage2="auto", positions=None, offsets=None):
    fb = _fb()
    band = fb.make_band(frac_bw, stage2=stage2, max_blocks=4, generator_solver=solver)
    geom = fb.make_geometry(kind, mx, my, bx, by)
    plan = fb.Plan(geom, N, band, positions=positions) if positions is not None else fb.Plan(geom, N, band)
    i = plan.info
    pb = O.make_problem(kind, mx, my, bx, by, N, frac_bw=i.fb_num / i.fb_den, epsilon=i.eps_num / i.eps_den,
                        delta=i.delta, L=i.L, offsets=offsets)
    return plan, pb


def dense_x(pb, b):
    return np.linalg.solve(O.gram(pb, b), np.eye(pb.L)[:, 0])


CASES = [
    ("ula", 8, 1, 8, 1, 16, 0.5, None),      # L = 32: 31 steps, the root is a leaf
    ("ula", 8, 1, 8, 1, 17, 0.5, None),      # L = 34: 33 steps, leaves of 16 and 17
    ("ula", 16, 1, 16, 1, 32, 0.5, None),    # L = 64: a leaf of exactly 32 steps
    ("ula", 16, 1, 12, 1, 64, 0.45, None),   # L = 128: a node of 64 steps with P = 64
    ("ula", 13, 1, 10, 1, 100, 0.37, None),  # L = 200: odd splits
    ("ura", 4, 4, 4, 4, 48, 0.3, None),      # rectangular array, L = 96
]


@pytest.mark.parametrize("case", CASES)
def test_superfast_matches_dense_solve(case):
    kind, mx, my, bx, by, N, fbw, beams = case
    plan, pb = make(kind, mx, my, bx, by, N, fbw, "superfast")
    x = plan.generators()
    worst = 0.0
    for b in (range(pb.B) if beams is None else beams):
        ref = dense_x(pb, b)
        err = O.rel_l2(x[b], ref)
        worst = max(worst, err)
        assert err < TOL_X, (b, err)
    print(f"superfast {kind}{mx} L={pb.L}: worst rel err {worst:.2e} of the dense solve")


@pytest.mark.parametrize("mx,N,beams", [(1024, 512, [0, 1, 511, 512, 1000]), (16, 1024, [0, 5, 8, 15])])
def test_superfast_at_the_largest_sizes(mx, N, beams):
    # ULA1024 (L = 1024, the benchmark's plan) and L = 2048 (the library's largest, FFT size 2048):
    # both solvers on the device, sampled beams against the dense solve.
    plan, pb = make("ula", mx, 1, mx, 1, N, 0.5, "superfast")
    xs = plan.generators()
    xl = torch.empty((pb.B, pb.L), dtype=torch.complex128, device="cuda")
    plan.solve_generators("levinson", xl)
    torch.cuda.synchronize()
    xl = xl.cpu().numpy()
    assert O.rel_l2(xs, xl) < TOL_X
    for b in beams:
        ref = dense_x(pb, b)
        es, el = O.rel_l2(xs[b], ref), O.rel_l2(xl[b], ref)
        print(f"L={pb.L} beam {b}: superfast {es:.2e}, Levinson {el:.2e}")
        assert es < TOL_X and el < TOL_X


def test_superfast_on_a_nonuniform_array():
    from synth import array_positions, perturbed_geometry
    mx, N = 24, 40
    geom = perturbed_geometry("ula", mx, 1, 0.2, 3)
    plan, pb = make("ula", mx, 1, mx, 1, N, 0.5, "superfast", positions=array_positions(geom),
                    offsets=geom.offsets)
    x = plan.generators()
    for b in (0, 7, 12, 23):
        assert O.rel_l2(x[b], dense_x(pb, b)) < TOL_X


def test_solve_generators_on_a_side_stream_equals_the_plan():
    plan, pb = make("ula", 64, 1, 64, 1, 96, 0.5, "levinson")
    x = torch.full((pb.B, pb.L), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan.solve_generators("superfast", x, stream=s)
    s.synchronize()
    assert plan.sync_status() == 0
    assert O.rel_l2(x.cpu().numpy(), plan.generators()) < TOL_X
    with pytest.raises(ValueError):
        plan.solve_generators("superfast", torch.empty((pb.B, pb.L), dtype=torch.complex64, device="cuda"))
    with pytest.raises(KeyError):
        plan.solve_generators("schur", x)


@pytest.mark.parametrize("stage2", ["gs_ir1", "dense_f16x3"])
def test_plans_of_both_solvers_give_the_same_transform(stage2):
    rng = np.random.default_rng(4)
    a, pb = make("ula", 64, 1, 64, 1, 128, 0.5, "levinson", stage2=stage2)
    b, _ = make("ula", 64, 1, 64, 1, 128, 0.5, "superfast", stage2=stage2)
    y = rng.standard_normal((3, pb.M, pb.N)) + 1j * rng.standard_normal((3, pb.M, pb.N))
    yd = torch.from_numpy(y.astype(np.complex64)).cuda()
    oa = torch.empty((3, pb.B, pb.N), dtype=torch.complex64, device="cuda")
    ob = torch.empty_like(oa)
    a.execute(yd, oa, 3)
    b.execute(yd, ob, 3)
    torch.cuda.synchronize()
    ref = O.fbst(pb, y)
    ga, gb = oa.cpu().numpy(), ob.cpu().numpy()
    assert O.rel_l2(gb, ref) < 1e-5
    assert O.rel_l2(gb, ga) < 1e-6


def test_offgrid_operators_from_the_superfast_solver():
    # fbst_offgrid_create solves for the directions' generators with the plan's solver.
    fb = _fb()
    dirs = [(0.0517, 0.0), (-0.3301, 0.0), (0.77, 0.0)]
    outs = []
    rng = np.random.default_rng(8)
    y = rng.standard_normal((2, 32, 64)) + 1j * rng.standard_normal((2, 32, 64))
    for solver in ("levinson", "superfast"):
        plan, pb = make("ula", 32, 1, 32, 1, 64, 0.5, solver)
        out = torch.empty((2, len(dirs), 64), dtype=torch.complex64, device="cuda")
        with fb.OffGrid(plan, dirs) as og:
            og.execute(torch.from_numpy(y.astype(np.complex64)).cuda(), out, 2)
        torch.cuda.synchronize()
        assert plan.sync_status() == 0
        outs.append(out.cpu().numpy())
    assert O.rel_l2(outs[1], outs[0]) < 1e-6
