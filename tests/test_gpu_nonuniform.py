"""Parity of the FBST on non-uniform linear arrays (Sec. IX, Eq. (16)) through the C ABI with the
FP64 oracle, whose sums run over the actual element positions (pinned in test_oracle_nonuniform.py).

The library computes stage 1b as a type-1 non-uniform FFT (kernel error about 1e-8, below the
FP32 rounding) and the Toeplitz generators by FP64 direct sums over the positions; everything else
is the plan of a uniform array. Bars, as for the uniform array: the generators from Levinson to
1e-9 (FP64), stage 1 to 2e-6, the transform to 1e-5 (FP32), per beam as in the headline tests.
Outputs are poisoned with NaN first.
"""
import numpy as np
import pytest

import oracle as O
from synth import Source, array_record, perturbed_geometry, waveform, array_positions

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_08887_gb300.build import build
    build()


def make(M, B, N, fbw, sigma, seed=3, stage2="auto", max_blocks=8):
    import paper_2512_08887_gb300 as fb
    geom = perturbed_geometry("ula", M, 1, sigma, seed)
    pos = array_positions(geom)
    plan = fb.Plan(fb.make_geometry("ula", M, 1, B, 1), N, fb.make_band(fbw, stage2=stage2, max_blocks=max_blocks),
                   positions=pos)
    i = plan.info
    pb = O.make_problem("ula", M, 1, B, 1, N, frac_bw=i.fb_num / i.fb_den, epsilon=i.eps_num / i.eps_den,
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


CASES = [(16, 16, 64, 0.5, 0.3), (40, 24, 96, 0.45, 0.2), (100, 150, 64, 0.8, 0.4), (256, 256, 128, 0.5, 0.2)]


@pytest.mark.parametrize("case", CASES)
def test_generators_and_stage1_match_oracle(rng, case):
    M, B, N, fbw, sigma = case
    plan, pb = make(M, B, N, fbw, sigma)
    assert plan.info.P_space_x >= 2 * B
    x = plan.generators()
    for b in (0, B // 3, B - 1):
        ref = np.linalg.solve(O.gram(pb, b), np.eye(pb.L)[:, 0])
        assert O.rel_l2(x[b], ref) < 1e-9, b
    y = crandn(rng, 3, M, N)
    got = run(plan, "czt", y, (3, B, pb.L), 3)
    ref = O.fan_coefficients(pb, y)
    print(f"non-uniform stage 1 M={M} B={B}: {O.rel_l2(got, ref):.2e}")
    assert O.rel_l2(got, ref) < 2e-6


@pytest.mark.parametrize("stage2", ["gs_ir1", "dense_tf32x3"])
@pytest.mark.parametrize("case", CASES)
def test_execute_matches_oracle(rng, case, stage2):
    M, B, N, fbw, sigma = case
    plan, pb = make(M, B, N, fbw, sigma, stage2=stage2, max_blocks=4)
    nblk = 6                                                      # two chunks, the second ragged
    y = crandn(rng, nblk, M, N)
    got = run(plan, "execute", y, (nblk, B, N), nblk)
    beams = np.unique(np.r_[0, np.linspace(0, B - 1, 9).astype(int), B - 1])
    ref = O.fbst(pb, y, beams=beams)
    assert O.rel_l2(got[:, beams], ref) < 1e-5
    assert per_beam_err(got[:, beams], ref) < 1e-5


def test_zero_offsets_give_the_uniform_transform(rng):
    import paper_2512_08887_gb300 as fb
    M, B, N = 48, 40, 64
    pos = np.stack([np.arange(M, dtype=float), np.zeros(M)], axis=1)
    nu = fb.Plan(fb.make_geometry("ula", M, 1, B, 1), N, fb.make_band(0.5, max_blocks=2), positions=pos)
    un = fb.Plan(fb.make_geometry("ula", M, 1, B, 1), N, fb.make_band(0.5, max_blocks=2))
    y = crandn(rng, 2, M, N)
    a = run(nu, "execute", y, (2, B, N), 2)
    b = run(un, "execute", y, (2, B, N), 2)
    assert O.rel_l2(a, b) < 2e-6


def test_plane_wave_on_a_perturbed_array_is_reproduced():
    M, N, b = 32, 64, 21
    plan, pb = make(M, M, N, 0.5, 0.3, seed=8)
    rs = np.random.default_rng(7)
    Q = 64
    src = Source(pb.directions[b, 0], 0.0, (rs.standard_normal(Q) + 1j * rs.standard_normal(Q)) * np.sqrt(0.5 / Q),
                 rs.uniform(-0.5, 0.5, Q))
    y = array_record(pb.geom, [src], 0.5, N, None, None)[None].astype(np.complex64)
    got = run(plan, "execute", y, (1, M, N), 1)
    assert O.rel_l2(got[0, b], waveform(src, np.arange(N))) < 1e-2


def test_full_size_perturbed_1024_element_array(rng):
    # The headline array with elements moved by N(0, 0.2^2) half wavelengths: 16 blocks, the
    # split-TF32 stage 2, sampled beams including both edges.
    M, N = 1024, 512
    plan, pb = make(M, M, N, 0.5, 0.2, seed=11, stage2="dense_tf32x3", max_blocks=16)
    y = crandn(rng, 16, M, N)
    got = run(plan, "execute", y, (16, M, N), 16)
    beams = np.unique(np.r_[0, 1, np.linspace(0, M - 1, 14).astype(int), M - 2, M - 1])
    ref = O.fbst(pb, y[:4], beams=beams)
    print(f"perturbed 1024-element array: {O.rel_l2(got[:4, beams], ref):.2e}")
    assert O.rel_l2(got[:4, beams], ref) < 1e-5
    assert per_beam_err(got[:4, beams], ref) < 1e-5
    assert np.isfinite(got).all()


def test_invalid_positions_are_rejected():
    import paper_2512_08887_gb300 as fb
    band = fb.make_band(0.5)
    bad = np.stack([np.arange(8, dtype=float), np.zeros(8)], axis=1)
    bad[3, 0] = np.nan
    with pytest.raises(fb.FBSTError) as e:
        fb.Plan(fb.make_geometry("ula", 8), 16, band, positions=bad)
    assert e.value.status == -1
    bad = np.stack([np.arange(8, dtype=float), np.full(8, 0.1)], axis=1)
    with pytest.raises(fb.FBSTError) as e:
        fb.Plan(fb.make_geometry("ula", 8), 16, band, positions=bad)
    assert e.value.status == -1
    with pytest.raises(fb.FBSTError) as e:   # a 256 x 256 oversampled grid: beyond the 2-D kernel
        fb.Plan(fb.make_geometry("ura", 2, 2, 128, 128), 16, band, positions=np.zeros((4, 2)))
    assert e.value.status == -4
    nu = fb.Plan(fb.make_geometry("ula", 8), 16, band, positions=np.stack([np.arange(8.0), np.zeros(8)], axis=1))
    with pytest.raises(fb.FBSTError) as e:
        fb.Nulling(nu, [2])
    assert e.value.status == -4
