"""Pins of the oracle's time-domain interference nulling (Sec. VIII-B, Eq. (15)); no GPU needed.

Eq. (15) rewrites the beamspace nulling of Eq. (14) on time-domain beams: the interferer's beam
y_p = F_x beta_p over a reconstruction interval broad enough for F_x to have full column rank is
mapped by G'_{b,p} = F_u H_{b,p} F_x^+ and subtracted from the plain beam y_b. The oracle forms
every matrix literally (pseudo-inverse, dense solve), independently of the Eq. (14) oracle's
bracket, which is itself pinned against the array-space projection (test_oracle_nulling.py).
Pins:

* on the broader interval (2L samples centred on the block) F_x^+ F_x = I, and Eq. (15) gives the
  Eq. (14) result for one and two interferers, linear and rectangular arrays;
* why 2L: an interval of only L samples makes F_x square but ill conditioned as L grows (the
  stretched frequencies interleave near half a cycle per sample), while 2L keeps it near 1;
* the defining identity of G': G'_{b,p} F_x beta = F_u H_{b,p} beta for any beta;
* on the block's own N samples (the Nyquist interval, N < L) F_x is fat, F_x^+ F_x != I, and the
  time-domain form no longer equals Eq. (14): the broader interval is what makes it exact;
* no interferers: the plain FBST.
"""
import numpy as np
import pytest

import oracle as O


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


PROBLEMS = [("ula", 12, 1, 12, 1, 32, [5]), ("ula", 16, 1, 20, 1, 24, [3, 14]), ("ura", 4, 3, 4, 3, 24, [7])]


def _problem(kind, mx, my, bx, by, N):
    return O.make_problem(kind, mx, my, bx, by, N, frac_bw=0.5, epsilon=1.01, delta_rel=1e-3)


@pytest.mark.parametrize("kind,mx,my,bx,by,N,ints", PROBLEMS)
def test_broader_interval_makes_time_domain_nulling_equal_eq14(kind, mx, my, bx, by, N, ints):
    pb = _problem(kind, mx, my, bx, by, N)
    n0, Nu = O.time_interval(pb)
    assert Nu == 2 * pb.L and n0 == -((2 * pb.L - pb.N) // 2)
    Fx = O.F_u_interval(pb, n0, Nu)
    assert np.abs(np.linalg.pinv(Fx) @ Fx - np.eye(pb.L)).max() < 1e-10
    # The block's own samples are rows -n0 .. -n0 + N - 1 of the broader interval.
    assert np.abs(Fx[-n0:-n0 + pb.N] - O.F_u(pb)).max() < 1e-12
    rng = np.random.default_rng(3)
    y = _crandn(rng, 2, pb.M, pb.N)
    got = O.fbst_nulled_time(pb, y, ints)
    ref = O.fbst_nulled(pb, y, ints)
    assert O.rel_l2(got, ref) < 1e-10


def test_g_prime_maps_interferer_beams_like_h():
    pb = _problem("ula", 12, 1, 12, 1, 32)
    f = O.TimeNullingFactors(pb, [4], beams=[0, 6, 11])
    rng = np.random.default_rng(5)
    beta = _crandn(rng, pb.L)
    for i, b in enumerate([0, 6, 11]):
        H = np.linalg.solve(O.gram(pb, b), O.cross_gram(pb, b, 4))
        lhs = f.Gp[i][0] @ (f.Fx @ beta)
        rhs = O.F_u(pb) @ (H @ beta)
        assert np.linalg.norm(lhs - rhs) <= 1e-10 * np.linalg.norm(rhs)


def test_nyquist_interval_is_not_enough():
    pb = _problem("ula", 16, 1, 16, 1, 32)
    Fn = O.F_u_interval(pb, 0, pb.N)
    assert np.linalg.matrix_rank(Fn) == pb.N < pb.L
    assert np.abs(np.linalg.pinv(Fn) @ Fn - np.eye(pb.L)).max() > 0.1
    rng = np.random.default_rng(9)
    y = _crandn(rng, 2, pb.M, pb.N)
    f = O.TimeNullingFactors(pb, [5], n0=0, Nu=pb.N)
    w = O.fan_coefficients(pb, y, f.out.beams)
    got = f.apply(f.out.apply(w), f.interferer_beams(O.fan_coefficients(pb, y, [5])))
    assert O.rel_l2(got, O.fbst_nulled(pb, y, [5])) > 1e-2


def test_no_interferers_is_the_plain_transform():
    pb = _problem("ula", 12, 1, 12, 1, 32)
    rng = np.random.default_rng(2)
    y = _crandn(rng, 1, pb.M, pb.N)
    f = O.TimeNullingFactors(pb, [])
    w = O.fan_coefficients(pb, y, f.out.beams)
    plain = f.out.apply(w)
    assert np.array_equal(f.apply(plain, np.zeros((1, 0, pb.L))), plain)


def test_interval_of_2l_samples_is_well_conditioned():
    conds = []
    for N in (64, 256):
        pb = _problem("ula", 12, 1, 12, 1, N)
        n0, Nu = O.time_interval(pb)
        square = O.F_u_interval(pb, -((pb.L - pb.N) // 2), pb.L)
        conds.append((np.linalg.cond(O.F_u_interval(pb, n0, Nu)), np.linalg.cond(square)))
    assert all(c2 < 20 for c2, _ in conds)
    assert conds[1][1] > 1e6          # L = 512 samples only: numerically singular
