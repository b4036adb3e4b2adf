"""Pins of the oracle's beamspace interference nulling (Sec. VIII-B, Eq. (14)); no GPU needed.

Eq. (14) is derived in the paper from an array-space projection: nulling in beamspace equals the
plain FBST of the measurements after the (regularised) projection of each interferer's Fourier
extension out of them. That gives a route to the same numbers that shares nothing with the
oracle's cross Gram matrices or its normal-equation solves:

* the cross Gram matrix F_b^H F_p against the explicit Eq. (6) matrices (signs, carriers, indices);
* its diagonal special case F_b^H F_b + delta I = A_b;
* Eq. (14) against the FBST of y - sum_p F_p x_p, x_p by QR least squares on the augmented system
  (one and two interferers, linear and rectangular arrays);
* the nulled interferer beam in closed form: F_p^H F_p = A_p - delta I gives
  bhat_p = delta F_u A_p^{-2} w_p for a single interferer;
* no interferers: the plain FBST;
* physics: an interferer on a grid beam is removed from every beam, and a source far from it
  passes almost unchanged (the interference bias of Sec. VIII-B is small when the two are apart).
"""
import numpy as np
import pytest

import oracle as O
from synth import ArrayGeometry, Source, array_record
from synth import configs, interference_config


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


PROBLEMS = [("ula", 12, 1, 12, 1, 32), ("ura", 4, 3, 4, 3, 24)]


@pytest.mark.parametrize("kind,mx,my,bx,by,N", PROBLEMS)
def test_cross_gram_is_the_product_of_the_explicit_matrices(kind, mx, my, bx, by, N):
    pb = O.make_problem(kind, mx, my, bx, by, N, frac_bw=0.5, delta_rel=1e-3)
    for b, p in [(1, 5), (7, 2), (0, pb.B - 1), (3, 3)]:
        C = O.cross_gram(pb, b, p)
        Ce = O.F_theta(pb, b).conj().T @ O.F_theta(pb, p)
        assert np.abs(C - Ce).max() <= 1e-12 * np.abs(Ce).max()
    # Diagonal case: the Gram matrix of Eq. (5) without the regulariser.
    A = O.gram(pb, 2)
    assert np.abs(O.cross_gram(pb, 2, 2) + pb.delta * np.eye(pb.L) - A).max() <= 1e-13 * np.abs(A).max()
    # Off the diagonal the element sum is not Toeplitz: the matrix must not be constant along diagonals.
    C = O.cross_gram(pb, 1, 5)
    assert np.abs(np.diag(C, 1) - np.diag(C, 1)[0]).max() > 1e-3 * np.abs(C).max()


@pytest.mark.parametrize("kind,mx,my,bx,by,N", PROBLEMS)
@pytest.mark.parametrize("interferers", [[3], [3, 7]])
def test_eq14_equals_fbst_of_the_projected_measurements(kind, mx, my, bx, by, N, interferers, rng):
    pb = O.make_problem(kind, mx, my, bx, by, N, frac_bw=0.5, delta_rel=1e-3)
    y = _crandn(rng, 2, pb.M, N)
    got = O.fbst_nulled(pb, y, interferers)
    yt = y.reshape(2, -1).copy()
    for p in interferers:
        F = O.F_theta(pb, p)
        for k in range(2):
            yt[k] -= F @ O.lstsq_augmented(F, y.reshape(2, -1)[k], pb.delta)
    ref = O.fbst(pb, yt.reshape(y.shape))
    assert O.rel_l2(got, ref) < 1e-11


def test_nulled_interferer_beam_closed_form(rng):
    pb = O.make_problem("ula", 10, 1, 10, 1, 24, frac_bw=0.4, delta_rel=1e-2)
    y = _crandn(rng, 1, pb.M, pb.N)
    p = 6
    got = O.fbst_nulled(pb, y, [p], beams=[p])[0, 0]
    A = O.gram(pb, p)
    w = O.fan_coefficients(pb, y, [p])[0, 0]
    ref = pb.delta * (O.F_u(pb) @ np.linalg.solve(A, np.linalg.solve(A, w)))
    assert O.rel_l2(got, ref) < 1e-9


def test_no_interferers_is_the_plain_transform(rng):
    pb = O.make_problem("ula", 8, 1, 8, 1, 16, frac_bw=0.5, delta_rel=1e-3)
    y = _crandn(rng, 2, pb.M, pb.N)
    assert O.rel_l2(O.fbst_nulled(pb, y, []), O.fbst(pb, y)) < 1e-14


def _wave(rng, u, power, Q=64):
    amp = (rng.standard_normal(Q) + 1j * rng.standard_normal(Q)) * np.sqrt(0.5 * power / Q)
    return Source(u, 0.0, amp, rng.uniform(-0.5, 0.5, Q))


def test_interferer_removed_and_distant_source_kept():
    M, N, nblk = 16, 64, 4
    pb = O.make_problem("ula", M, 1, M, 1, N, frac_bw=0.5, delta_rel=1e-3)
    rng = np.random.default_rng(5)
    ui, us = pb.directions[4, 0], pb.directions[11, 0]
    g = ArrayGeometry("ula", M)
    fac = O.NullingFactors(pb, [4])

    def run(sources):
        y = array_record(g, sources, 0.5, nblk * N, None, None).reshape(M, nblk, N).transpose(1, 0, 2)
        return O.fbst(pb, y), O.fbst_nulled(pb, y, [4], factors=fac)

    plain, nul = run([_wave(rng, ui, 100.0)])
    assert np.linalg.norm(nul) < 2e-2 * np.linalg.norm(plain)          # measured 4.5e-3
    plain, nul = run([_wave(rng, us, 1.0)])
    assert O.rel_l2(nul[:, 11], plain[:, 11]) < 2e-2                     # measured 4.9e-3


def test_nulling_workload_recipe():
    d = configs.nulling_data("C2N", nblk=1, Q=8)
    assert d["y"].shape == (1, 256, 256) and d["y"].dtype == np.complex64
    assert d["interferers"] == [64, 96] and d["source_beams"] == [160]
    # Same seed, same data.
    assert np.array_equal(d["y"], configs.nulling_data("C2N", nblk=1, Q=8)["y"])


def test_offgrid_interferers_reduce_to_grid_interferers():
    # Interferers placed exactly on grid beams: the interpolation returns those beams' vectors and
    # F_p is the grid beam's, so the off-grid form equals Eq. (14) with grid interferers.
    rng = np.random.default_rng(31)
    for kind, mx, my, bx, by, ints in (("ula", 12, 1, 16, 1, [3, 9]), ("ura", 3, 3, 4, 4, [5])):
        pb = O.make_problem(kind, mx, my, bx, by, N=16, frac_bw=0.5, delta_rel=1e-3)
        y = rng.standard_normal((2, pb.M, pb.N)) + 1j * rng.standard_normal((2, pb.M, pb.N))
        a = O.fbst_nulled(pb, y, ints)
        b = O.fbst_nulled_offgrid(pb, y, pb.directions[ints])
        np.testing.assert_allclose(b, a, atol=1e-10 * np.abs(a).max())


def test_cross_gram_to_an_offgrid_direction_follows_eq6():
    pb = O.make_problem("ula", 7, 1, 9, 1, N=10, frac_bw=0.45, delta_rel=1e-3)
    d = np.array([0.2713, 0.0])
    C = O.cross_gram_direction(pb, 4, d)
    np.testing.assert_allclose(C, O.F_theta(pb, 4).conj().T @ O.F_theta(pb, 0, direction=d), atol=1e-10)


def test_offgrid_interferer_is_suppressed():
    # Physics of Sec. VIII-B with an off-grid interferer (halfway between two beams of a 2x
    # oversampled grid): its interpolated vector is about 5% off, so it is not removed to the grid
    # case's 0.45%, but less than 10% of the interferer's plain output is left (6.6%), against a
    # third (34%) when the nearest grid beam is nulled instead.
    M, N = 16, 64
    pb = O.make_problem("ula", M, 1, 2 * M, 1, N=N, frac_bw=0.5, delta_rel=1e-3)
    u = pb.directions[10, 0] + 1.0 / pb.B
    y = interference_config("ula", M, 1, N, 2, 0.5, [], [(u, 0.0)], 20.0, None, 4, Q=64)["y"]
    plain = O.fbst(pb, y)
    nulled = O.fbst_nulled_offgrid(pb, y, [[u, 0.0]])
    ratio = np.linalg.norm(nulled) / np.linalg.norm(plain)
    assert ratio < 0.1, ratio
    # Nulling the nearest grid beam instead leaves several times more of it.
    nearest = np.linalg.norm(O.fbst_nulled(pb, y, [10])) / np.linalg.norm(plain)
    assert ratio < nearest / 3, (ratio, nearest)
