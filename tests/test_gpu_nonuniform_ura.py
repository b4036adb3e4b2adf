"""Parity of the FBST on rectangular arrays whose elements are off the grid in both coordinates
(Sec. IX, Eq. (16)) through the C ABI with the FP64 oracle, whose sums run over the actual element
positions (pinned for a 3 x 4 array in test_oracle_nonuniform.py).

The library computes stage 1b as a two-dimensional type-1 NUFFT (W x W spreading onto an
oversampled nf_x x nf_y grid, a 2-D FFT, the two axes' deconvolution factors; kernel error about
1e-8 per axis, below the FP32 rounding) and the Toeplitz generators by FP64 direct sums over the
positions. Bars as for the linear array: the generators to 1e-9 (FP64 Levinson), stage 1 to 2e-6,
the transform to 1e-5 (FP32), also per beam. Outputs are poisoned with NaN first.
"""
import numpy as np
import pytest

import oracle as O
from synth import array_positions, perturbed_geometry

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_08887_gb300.build import build
    build()


def make(mx, my, bx, by, N, fbw, sigma, seed=3, stage2="auto", max_blocks=8):
    import paper_2512_08887_gb300 as fb
    geom = perturbed_geometry("ura", mx, my, sigma, seed)
    plan = fb.Plan(fb.make_geometry("ura", mx, my, bx, by), N,
                   fb.make_band(fbw, stage2=stage2, max_blocks=max_blocks), positions=array_positions(geom))
    i = plan.info
    pb = O.make_problem("ura", mx, my, bx, by, N, frac_bw=i.fb_num / i.fb_den, epsilon=i.eps_num / i.eps_den,
                        delta=i.delta, L=i.L, offsets=geom.offsets)
    return plan, pb


def crandn(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


def run(plan, fn, x, shape, nblk):
    out = torch.full(shape, complex(np.nan, np.nan), dtype=torch.complex64, device="cuda")
    getattr(plan, fn)(torch.from_numpy(np.ascontiguousarray(x)).cuda(), out, nblk)
    assert plan.sync_status() == 0
    return out.cpu().numpy()


def per_beam_err(got, ref):
    e = np.linalg.norm(got - ref, axis=(0, 2))
    n = np.linalg.norm(ref, axis=(0, 2))
    return float(np.max(e / np.maximum(n, np.sqrt(np.mean(n ** 2)))))


CASES = [
    (8, 8, 8, 8, 64, 0.5, 0.2),        # 16 x 16 grid
    (6, 10, 8, 12, 48, 0.45, 0.3),     # unequal axes: 16 x 32 grid, M != B
    (16, 16, 20, 20, 32, 0.3, 0.2),    # 64 x 64 grid, B > M
]


@pytest.mark.parametrize("case", CASES)
def test_generators_and_stage1_match_oracle(rng, case):
    mx, my, bx, by, N, fbw, sigma = case
    plan, pb = make(mx, my, bx, by, N, fbw, sigma)
    assert plan.info.P_space_x >= 2 * bx and plan.info.P_space_y >= 2 * by
    x = plan.generators()
    for b in (0, pb.B // 3, pb.B - 1):
        ref = np.linalg.solve(O.gram(pb, b), np.eye(pb.L)[:, 0])
        assert O.rel_l2(x[b], ref) < 1e-9, b
    y = crandn(rng, 3, pb.M, N)
    got = run(plan, "czt", y, (3, pb.B, pb.L), 3)
    ref = O.fan_coefficients(pb, y)
    print(f"non-uniform URA stage 1 {mx}x{my} -> {bx}x{by}: {O.rel_l2(got, ref):.2e}")
    assert O.rel_l2(got, ref) < 2e-6
    assert per_beam_err(got, ref) < 2e-6


@pytest.mark.parametrize("stage2", ["gs_ir1", "dense_f16x3"])
@pytest.mark.parametrize("case", CASES[:2])
def test_execute_matches_oracle(rng, case, stage2):
    mx, my, bx, by, N, fbw, sigma = case
    plan, pb = make(mx, my, bx, by, N, fbw, sigma, stage2=stage2, max_blocks=4)
    nblk = 6                                                      # two chunks, the second ragged
    y = crandn(rng, nblk, pb.M, N)
    got = run(plan, "execute", y, (nblk, pb.B, N), nblk)
    beams = np.unique(np.r_[0, np.linspace(0, pb.B - 1, 11).astype(int), pb.B - 1])
    ref = O.fbst(pb, y, beams=beams)
    assert O.rel_l2(got[:, beams], ref) < 1e-5
    assert per_beam_err(got[:, beams], ref) < 1e-5


def test_grid_positions_give_the_uniform_transform(rng):
    # Elements exactly on the grid through the 2-D NUFFT against the rectangular chirp-z of App. B.
    import paper_2512_08887_gb300 as fb
    mx, my, N = 8, 8, 64
    pos = np.stack(np.meshgrid(np.arange(mx, dtype=float), np.arange(my, dtype=float), indexing="ij"),
                   axis=-1).reshape(-1, 2)
    geom = fb.make_geometry("ura", mx, my)
    nu = fb.Plan(geom, N, fb.make_band(0.5, max_blocks=2), positions=pos)
    un = fb.Plan(geom, N, fb.make_band(0.5, max_blocks=2))
    y = crandn(rng, 2, mx * my, N)
    a = run(nu, "execute", y, (2, mx * my, N), 2)
    b = run(un, "execute", y, (2, mx * my, N), 2)
    assert O.rel_l2(a, b) < 2e-6


def test_full_size_perturbed_32x32_array(rng):
    # The 32 x 32 rectangular array (config C3's geometry, N = 512, L = 1024) with both coordinates
    # moved by N(0, 0.2^2) half wavelengths: 8 blocks, sampled beams including the corners.
    plan, pb = make(32, 32, 32, 32, 512, 0.3, 0.2, seed=5, stage2="dense_f16x3", max_blocks=8)
    y = crandn(rng, 8, pb.M, 512)
    got = run(plan, "execute", y, (8, pb.B, 512), 8)
    beams = np.unique(np.r_[0, 31, 32 * 16 + 16, np.linspace(0, pb.B - 1, 12).astype(int), pb.B - 32, pb.B - 1])
    ref = O.fbst(pb, y[:2], beams=beams)
    print(f"perturbed 32x32 array: {O.rel_l2(got[:2, beams], ref):.2e}")
    assert O.rel_l2(got[:2, beams], ref) < 1e-5
    assert per_beam_err(got[:2, beams], ref) < 1e-5
    assert np.isfinite(got).all()
