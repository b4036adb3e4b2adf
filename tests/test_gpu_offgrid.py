"""Parity of the off-grid beams (Sec. VIII-A) through the C ABI with the FP64 oracle.

The library interpolates the stage-1 beam vectors of the K grid beams around each direction (a
natural cubic spline in the direction cosine, per axis) and applies the off-grid direction's own
regularised least-squares operator (Gohberg-Semencul with one refinement step, FP64 plan-time
spectra). Bars: the interpolation alone is a K-term (K^2 for a rectangular array) FP32 weighted sum
of complex64 vectors with weights of magnitude about 1, held to 2e-6 of |w*| per direction (the
stage-1 bar); the off-grid beams end to end to the transform's 1e-5. The distance of the
interpolated beam vector from the exact one is a property of the spline (the oracle's, not the
library's) and is reported, not gated. Outputs are poisoned with NaN first.
"""
import numpy as np
import pytest

import oracle as O
from synth import ArrayGeometry, Source, array_record, waveform

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_INTERP = 2e-6
TOL_E2E = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_08887_gb300.build import build
    build()


def _plan(kind, mx, my, bx, by, N, fbw, max_blocks=4):
    import paper_2512_08887_gb300 as fb
    plan = fb.Plan(fb.make_geometry(kind, mx, my, bx, by), N, fb.make_band(fbw, max_blocks=max_blocks))
    i = plan.info
    pb = O.make_problem(kind, mx, my, bx, by, N, frac_bw=i.fb_num / i.fb_den, epsilon=i.eps_num / i.eps_den,
                        delta=i.delta, L=i.L)
    return plan, pb


def _nan(shape):
    return torch.full(shape, complex(np.nan, np.nan), dtype=torch.complex64, device="cuda")


def _dirs(pb, rng, n):
    """n directions: off-grid ones at random, one exactly on a grid beam, the two grid ends."""
    if pb.geom.kind == "ula":
        u = np.r_[rng.uniform(-0.99, 0.99, n - 3), pb.directions[5, 0], -1.0, 1.0 - 1e-9]
        return np.stack([u, np.zeros_like(u)], axis=1)
    uv = rng.uniform(-0.95, 0.95, (n - 2, 2))
    return np.vstack([uv, pb.directions[7], [-1.0, 0.97]])


CASES = [("ula", 16, 1, 32, 1, 64, 0.5, 3), ("ula", 40, 1, 70, 1, 96, 0.45, 5),
         ("ura", 4, 4, 8, 8, 32, 0.3, 2), ("ula", 64, 1, 128, 1, 128, 0.5, 6)]


@pytest.mark.parametrize("case", CASES)
def test_offgrid_beams_match_oracle(rng, case):
    import paper_2512_08887_gb300 as fb
    kind, mx, my, bx, by, N, fbw, nblk = case
    plan, pb = _plan(kind, mx, my, bx, by, N, fbw, max_blocks=4)     # nblk > 4: several chunks
    dirs = _dirs(pb, rng, 9)
    y = (rng.standard_normal((nblk, pb.M, N)) + 1j * rng.standard_normal((nblk, pb.M, N))).astype(np.complex64)
    fac = O.OffGridFactors(pb, dirs)
    w64 = O.fan_coefficients(pb, y)
    with fb.OffGrid(plan, dirs) as og:
        # Interpolation alone, on the oracle's w rounded to complex64.
        w32 = w64.astype(np.complex64)
        ws = _nan((nblk, len(dirs), pb.L))
        og.interpolate(torch.from_numpy(w32).cuda(), ws, nblk)
        ref_ws = fac.interpolate(w32.astype(np.complex128))
        per = np.linalg.norm(ws.cpu().numpy() - ref_ws, axis=(0, 2)) / np.linalg.norm(ref_ws, axis=(0, 2))
        assert per.max() < TOL_INTERP, per
        # End to end from y.
        out = _nan((nblk, len(dirs), N))
        og.execute(torch.from_numpy(y).cuda(), out, nblk)
        assert plan.sync_status() == 0
    got = out.cpu().numpy()
    ref = fac.apply(fac.interpolate(w64))
    per = np.linalg.norm(got - ref, axis=(0, 2)) / np.linalg.norm(ref, axis=(0, 2))
    print(f"{kind} {mx}x{my} beams {bx}x{by}: rel L2 {O.rel_l2(got, ref):.2e}, per direction max {per.max():.2e}")
    assert O.rel_l2(got, ref) < TOL_E2E and per.max() < TOL_E2E


def test_grid_direction_gives_the_plain_beam(rng):
    import paper_2512_08887_gb300 as fb
    plan, pb = _plan("ula", 24, 1, 48, 1, 64, 0.5)
    y = (rng.standard_normal((2, 24, 64)) + 1j * rng.standard_normal((2, 24, 64))).astype(np.complex64)
    yd = torch.from_numpy(y).cuda()
    plain = _nan((2, 48, 64))
    plan.execute(yd, plain, 2)
    with fb.OffGrid(plan, [pb.directions[17], pb.directions[30]]) as og:
        out = _nan((2, 2, 64))
        og.execute(yd, out, 2)
    torch.cuda.synchronize()
    ref = plain.cpu().numpy()[:, [17, 30]]
    assert O.rel_l2(out.cpu().numpy(), ref) < TOL_E2E


def test_offgrid_source_is_recovered_on_the_gpu():
    # Physics (Sec. VIII-A): a plane wave from halfway between two beams of a 2x oversampled grid is
    # tracked by the interpolated off-grid beam far better than by the nearest grid beam.
    import paper_2512_08887_gb300 as fb
    M, N = 32, 64
    plan, pb = _plan("ula", M, 1, 2 * M, 1, N, 0.5, max_blocks=1)
    rs = np.random.default_rng(5)
    u = pb.directions[45, 0] + 1.0 / pb.B
    Q = 64
    src = Source(u, 0.0, (rs.standard_normal(Q) + 1j * rs.standard_normal(Q)) * np.sqrt(0.5 / Q),
                 rs.uniform(-0.5, 0.5, Q))
    y = array_record(ArrayGeometry("ula", M), [src], 0.5, N, None, None)[None].astype(np.complex64)
    yd = torch.from_numpy(y).cuda()
    grid = _nan((1, pb.B, N))
    plan.execute(yd, grid, 1)
    with fb.OffGrid(plan, [[u, 0.0]]) as og:
        off = _nan((1, 1, N))
        og.execute(yd, off, 1)
    torch.cuda.synchronize()
    s = waveform(src, np.arange(N))
    e_off, e_grid = O.rel_l2(off.cpu().numpy()[0, 0], s), O.rel_l2(grid.cpu().numpy()[0, 45], s)
    print(f"off-grid source: interpolated beam {e_off:.3f}, nearest grid beam {e_grid:.3f}")
    assert e_off < 0.5 * e_grid


def test_offgrid_invalid_arguments():
    import paper_2512_08887_gb300 as fb
    plan, pb = _plan("ula", 16, 1, 16, 1, 64, 0.5)
    for dirs, K in (([[1.5, 0.0]], 8), ([[0.1, 0.2]], 8), ([[float("nan"), 0.0]], 8), ([[0.1, 0.0]], 1),
                    ([[0.1, 0.0]], 17)):
        with pytest.raises(fb.FBSTError) as e:
            fb.OffGrid(plan, dirs, K=K)
        assert e.value.status == -1
    with fb.OffGrid(plan, [[0.1, 0.0]]) as og:
        out = torch.zeros((1, 1, 64), dtype=torch.complex64, device="cuda")
        with pytest.raises(fb.FBSTError):
            og.execute(0, out, 1)
        og.execute(0, 0, 0)                          # an empty call is a no-op
    assert plan.sync_status() == 0
