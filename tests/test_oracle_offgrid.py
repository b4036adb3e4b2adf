"""Pins of the oracle's off-grid beams (Sec. VIII-A): interpolation of beam vectors over the 8
nearest grid beams by a natural cubic spline, then the regularised least-squares beam of the
off-grid direction (Eq. (5)-(7) with that direction's F).

Each pin checks the oracle against something other than itself: an independent library spline,
the explicit Eq. (6) matrix of an off-grid direction, the special case of a grid direction (which
must reduce to the pinned plain transform), and the physics the paper describes (an interpolated
beam recovers an off-grid source better than the nearest grid beam).
"""
import numpy as np
import pytest
import scipy.interpolate

import oracle as O
from synth import ArrayGeometry, Source, array_record, waveform


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_spline_weights_match_an_independent_natural_spline(rng):
    for n in (2, 3, 5, 8):
        x = np.sort(rng.uniform(-1, 1, n))
        x[1:] += np.arange(1, n) * 1e-3            # strictly increasing
        f = rng.standard_normal(n)
        ref = scipy.interpolate.CubicSpline(x, f, bc_type="natural")
        for xq in np.r_[x, rng.uniform(x[0], x[-1], 7)]:
            assert O.natural_spline_weights(x, xq) @ f == pytest.approx(float(ref(xq)), abs=1e-12)


def test_spline_weights_interpolate_knots_and_reproduce_lines(rng):
    x = -1.0 + 2.0 * np.arange(8) / 16
    for i, xi in enumerate(x):
        np.testing.assert_allclose(O.natural_spline_weights(x, xi), np.eye(8)[i], atol=1e-14)
    for xq in rng.uniform(x[0], x[-1], 10):
        c = O.natural_spline_weights(x, xq)
        assert c.sum() == pytest.approx(1.0, abs=1e-13)
        assert c @ (3.0 * x - 0.5) == pytest.approx(3.0 * xq - 0.5, abs=1e-13)


def test_window_is_centred_and_clamped():
    assert O.interp_window(64, 20.3) == 17            # indices 17..24 around [20, 21]
    assert O.interp_window(64, 0.2) == 0              # clamped at the start
    assert O.interp_window(64, 63.5) == 56            # and at the end
    assert O.interp_window(5, 2.5) == 0               # fewer grid beams than the window


@pytest.mark.parametrize("kind,mx,my,bx,by", [("ula", 12, 1, 24, 1), ("ura", 4, 3, 8, 6)])
def test_grid_direction_reduces_to_the_plain_transform(rng, kind, mx, my, bx, by):
    pb = O.make_problem(kind, mx, my, bx, by, N=16, frac_bw=0.5, delta_rel=1e-3)
    b = 9
    terms = O.offgrid_terms(pb, pb.directions[b])
    assert dict((k, w) for k, w in terms if abs(w) > 1e-13) == pytest.approx({b: 1.0}, abs=1e-13)
    y = _crandn(rng, 2, pb.M, pb.N)
    np.testing.assert_allclose(O.fbst_offgrid(pb, y, [pb.directions[b]]), O.fbst(pb, y, beams=[b]), atol=1e-11)


def test_offgrid_gram_and_coefficients_follow_eq6(rng):
    # An off-grid direction: its A from the explicit Eq. (6) matrix F^H F + delta I, its exact
    # coefficient vector F^H y, both against the oracle's direct sums.
    for kind, mx, my in (("ula", 7, 1), ("ura", 3, 4)):
        pb = O.make_problem(kind, mx, my, mx, my, N=12, frac_bw=0.45, delta_rel=1e-3)
        d = np.array([0.3173, -0.2219 if kind == "ura" else 0.0])
        F = O.F_theta(pb, 0, direction=d)
        A = O.gram_direction(pb, d)
        np.testing.assert_allclose(A, F.conj().T @ F + pb.delta * np.eye(pb.L), atol=1e-10)
        np.testing.assert_allclose(A, A.conj().T, atol=1e-12)
        assert np.allclose(A[1:, 1:], A[:-1, :-1], atol=1e-10)        # Toeplitz
        y = _crandn(rng, pb.M, pb.N)
        w = O.fan_coefficients(pb, y[None], directions=[d])[0, 0]
        np.testing.assert_allclose(w, F.conj().T @ y.ravel(), atol=1e-10)


def test_interpolated_beam_recovers_an_offgrid_source_better_than_the_grid():
    # Physics of Sec. VIII-A: a noise-free plane wave from halfway between two grid beams of a
    # 2x oversampled grid (B = 2M). The beam formed at its direction from 8 interpolated beam
    # vectors tracks the waveform more closely than the nearest grid beam, and its interpolated
    # beam vector is near the exact one.
    M, N, fb = 32, 64, 0.5
    pb = O.make_problem("ula", M, 1, 2 * M, 1, N=N, frac_bw=fb, delta_rel=1e-3)
    rs = np.random.default_rng(5)
    u = pb.directions[45, 0] + 1.0 / pb.B           # halfway between beams 45 and 46
    Q = 64
    src = Source(u, 0.0, (rs.standard_normal(Q) + 1j * rs.standard_normal(Q)) * np.sqrt(0.5 / Q),
                 rs.uniform(-0.5, 0.5, Q))
    y = array_record(ArrayGeometry("ula", M), [src], fb, N, None, None)[None]
    s = waveform(src, np.arange(N))
    off = O.fbst_offgrid(pb, y, [[u, 0.0]])[0, 0]
    grid = O.fbst(pb, y, beams=[45])[0, 0]
    e_off, e_grid = O.rel_l2(off, s), O.rel_l2(grid, s)
    assert e_off < 0.5 * e_grid, (e_off, e_grid)
    fac = O.OffGridFactors(pb, [[u, 0.0]])
    w = O.fan_coefficients(pb, y)
    w_exact = O.fan_coefficients(pb, y, directions=[[u, 0.0]])
    assert O.rel_l2(fac.interpolate(w), w_exact) < 0.1
