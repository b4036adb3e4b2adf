"""Pins of the oracle on non-uniform arrays (Sec. IX, Eq. (16)); no GPU needed.

Off the grid only the element sum of the fan changes (it becomes the non-uniform sum of Eq. (16));
the temporal sum, the Toeplitz structure of A_b and stage 2 stay as they are. The oracle's sums
run over the actual positions, so the pins check that claim and the oracle on perturbed arrays:

* the fan and the Gram matrix against the explicit Eq. (6) matrices built from the positions;
* A_b stays Hermitian positive definite Toeplitz, with the generator
  a_b(d) = D_N(2 pi eps d / L) sum_m exp(-2 pi i eps d tau_{b,m} / L) + delta [d = 0];
* the normal-equation solve against QR least squares on the augmented system;
* zero offsets give the uniform array exactly; non-zero offsets do change the fan;
* physics: a plane wave from a grid direction is reproduced on a perturbed array.

Each test draws from its own seeded generator, so adding these tests leaves the draws of the
session-wide generator that the other oracle tests share unchanged.
"""
import numpy as np
import pytest

import oracle as O
from synth import Source, array_positions, array_record, perturbed_geometry, waveform


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _problem(kind, mx, my, bx, by, N, sigma, seed=3, **kw):
    g = perturbed_geometry(kind, mx, my, sigma, seed)
    return O.make_problem(kind, mx, my, bx, by, N, offsets=g.offsets, **kw)


ARRAYS = [("ula", 7, 1, 9, 1), ("ura", 3, 4, 4, 3)]


@pytest.mark.parametrize("kind,mx,my,bx,by", ARRAYS)
def test_fan_and_gram_match_explicit_eq6_matrix_off_grid(kind, mx, my, bx, by):
    rng = np.random.default_rng(901)
    pb = _problem(kind, mx, my, bx, by, 6, 0.3, frac_bw=0.45, delta_rel=1e-3)
    y = _crandn(rng, pb.M, pb.N)
    w = O.fan_coefficients(pb, y)
    for b in range(pb.B):
        F = O.F_theta(pb, b)
        np.testing.assert_allclose(w[b], F.conj().T @ y.reshape(-1), rtol=0, atol=1e-12 * np.abs(w).max())
        G = F.conj().T @ F + pb.delta * np.eye(pb.L)
        np.testing.assert_allclose(O.gram(pb, b), G, rtol=0, atol=1e-12 * np.abs(G).max())


@pytest.mark.parametrize("kind,mx,my,bx,by", ARRAYS)
def test_gram_stays_toeplitz_with_the_off_grid_generator(kind, mx, my, bx, by):
    pb = _problem(kind, mx, my, bx, by, 12, 0.4, frac_bw=0.5, delta_rel=1e-3)
    d = np.arange(pb.L)
    n = np.arange(pb.N)
    for b in range(pb.B):
        A = O.gram(pb, b)
        np.testing.assert_allclose(A, A.conj().T, atol=1e-12 * np.abs(A).max())
        for off in range(-pb.L + 1, pb.L):
            diag = np.diagonal(A, offset=off)
            assert np.abs(diag - diag[0]).max() <= 1e-11 * np.abs(A).max()
        assert np.linalg.eigvalsh(A).min() > 0.5 * pb.delta
        tau = pb.tau([b])[0]
        a = (np.exp(2j * np.pi * pb.epsilon * np.outer(d, n) / pb.L).sum(axis=1)
             * np.exp(-2j * np.pi * pb.epsilon * np.outer(d, tau) / pb.L).sum(axis=1))
        a[0] += pb.delta
        np.testing.assert_allclose(A[0], a, rtol=0, atol=1e-11 * np.abs(a).max())


def test_solve_matches_augmented_least_squares_off_grid():
    rng = np.random.default_rng(902)
    pb = _problem("ula", 6, 1, 6, 1, 10, 0.25, frac_bw=0.5, delta_rel=1e-3)
    y = _crandn(rng, pb.M, pb.N)
    beta = O.Stage2Factors(pb).coefficients(O.fan_coefficients(pb, y[None]))
    for b in range(pb.B):
        ref = O.lstsq_augmented(O.F_theta(pb, b), y.reshape(-1), pb.delta)
        np.testing.assert_allclose(beta[0, b], ref, rtol=0, atol=1e-9 * np.abs(ref).max())


def test_zero_offsets_are_the_uniform_array_and_offsets_matter():
    rng = np.random.default_rng(903)
    kw = dict(frac_bw=0.5, delta_rel=1e-3)
    uni = O.make_problem("ula", 8, 1, 8, 1, 16, **kw)
    zero = _problem("ula", 8, 1, 8, 1, 16, 0.0, **kw)
    pert = _problem("ula", 8, 1, 8, 1, 16, 0.2, **kw)
    np.testing.assert_array_equal(zero.positions, uni.positions)
    y = _crandn(rng, 2, 8, 16)
    np.testing.assert_array_equal(O.fbst(zero, y), O.fbst(uni, y))
    w_u, w_p = O.fan_coefficients(uni, y), O.fan_coefficients(pert, y)
    assert O.rel_l2(w_p, w_u) > 1e-2
    assert pert.positions[0].tolist() == [0.0, 0.0]         # the phase reference stays at the origin


@pytest.mark.parametrize("kind,mx,my,bx,by,b", [("ula", 16, 1, 16, 1, 11), ("ura", 4, 4, 4, 4, 9)])
def test_plane_wave_from_grid_angle_is_reproduced_off_grid(kind, mx, my, bx, by, b):
    rng = np.random.default_rng(904)
    # The same sanity bound as on the uniform grid (the bias itself is parity unpinned).
    g = perturbed_geometry(kind, mx, my, 0.2, 11)
    pb = O.make_problem(kind, mx, my, bx, by, 64, frac_bw=0.5, delta_rel=1e-3, offsets=g.offsets)
    u, v = pb.directions[b]
    amp = _crandn(rng, 64) * np.sqrt(0.5 / 64)
    src = Source(u, v, amp, rng.uniform(-0.5, 0.5, 64))
    np.testing.assert_array_equal(array_positions(g), pb.positions)
    y = array_record(g, [src], pb.frac_bw, pb.N, None, None)
    bh = O.fbst(pb, y[None])[0]
    s = waveform(src, np.arange(pb.N))
    assert O.rel_l2(bh[b], s) < 5e-3
