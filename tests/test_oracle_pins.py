"""Pins of the FP64 oracle against facts the paper and the mathematics fix (no GPU needed).

Each test names what it pins. Together they are chosen so that a dropped term, a wrong sign or
index, or a transposed operand anywhere in the oracle fails at least one of them:

* explicit Eq. (6) matrix vs the separable sums (index/sign of every exponent, both arrays);
* library reductions: the time sum at eps=1, L=2N is a zero-padded FFT; the frequency bin
  ell'=L/2 at eps=1 is a spatial inverse FFT; fb -> 0 turns every bin into the narrowband FFT;
* time-origin invariance (the paper counts n = 1..N, the oracle n = 0..N-1);
* structure: A_b is Hermitian, positive definite and Toeplitz (Sec. V);
* the solve vs QR least squares on the augmented system, and the dense operator vs the solve;
* closed forms: a hand-derived tiny case (tests/golden) and the single-sensor limit;
* physics: an on-grid plane wave is reproduced, noise variance matches the Monte Carlo and tends
  to sigma^2/M as N grows (Sec. VII), and the beam tracks exact-sinc delay-and-sum;
* linearity.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from synth import ArrayGeometry, Source, array_positions, array_record, waveform

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _toy_source(rng, u, v=0.0, Q=64):
    amp = _crandn(rng, Q) * np.sqrt(0.5 / Q)
    return Source(u, v, amp, rng.uniform(-0.5, 0.5, Q))


@pytest.mark.parametrize("kind,mx,my,bx,by", [("ula", 5, 1, 7, 1), ("ura", 3, 4, 4, 3)])
def test_fan_matches_explicit_eq6_matrix(rng, kind, mx, my, bx, by):
    pb = O.make_problem(kind, mx, my, bx, by, N=6, frac_bw=0.37, epsilon=1.01, delta_rel=1e-3)
    y = _crandn(rng, pb.M, pb.N)
    w = O.fan_coefficients(pb, y)
    for b in range(pb.B):
        F = O.F_theta(pb, b)
        np.testing.assert_allclose(w[b], F.conj().T @ y.reshape(-1), rtol=0, atol=1e-12 * np.abs(w).max())
        G = F.conj().T @ F + pb.delta * np.eye(pb.L)
        np.testing.assert_allclose(O.gram(pb, b), G, rtol=0, atol=1e-12 * np.abs(G).max())


def test_time_sum_is_zero_padded_fft_at_eps_one(rng):
    pb = O.make_problem("ula", 4, 1, 4, 1, N=16, frac_bw=0.5, epsilon=1.0, gamma=2, delta_rel=1e-3)
    y = _crandn(rng, pb.M, pb.N)
    yhat = O.stage1_time(pb, y)
    ref = np.fft.fft(y, 2 * pb.N, axis=1)[:, (pb.lprime.astype(int)) % (2 * pb.N)]
    np.testing.assert_allclose(yhat, ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def test_top_frequency_bin_is_spatial_ifft_ula(rng):
    # eps = 1 and ell' = L/2 give (1/fb + 1/2)*rho = 1/2, so the steering is exp(j*pi*u_b*m):
    # with u_b = -1 + 2b/B and B = M the sum is B*ifft((-1)^m yhat[m]).
    pb = O.make_problem("ula", 16, 1, 16, 1, N=8, frac_bw=0.7, epsilon=1.0, delta_rel=1e-3)
    yhat = _crandn(rng, pb.M, pb.L)
    w = O.stage1_space(pb, yhat)
    col = pb.L - 1
    assert pb.lprime[col] == pb.L / 2
    sign = (-1.0) ** np.arange(pb.M)
    np.testing.assert_allclose(w[:, col], pb.B * np.fft.ifft(sign * yhat[:, col]), atol=1e-10)


def test_top_frequency_bin_is_2d_spatial_ifft_ura(rng):
    pb = O.make_problem("ura", 4, 4, 4, 4, N=8, frac_bw=0.3, epsilon=1.0, delta_rel=1e-3)
    yhat = _crandn(rng, pb.M, pb.L)
    w = O.stage1_space(pb, yhat)
    col = pb.L - 1
    k = np.arange(4)
    sign = np.multiply.outer((-1.0) ** k, (-1.0) ** k).ravel()
    ref = 16 * np.fft.ifft2((sign * yhat[:, col]).reshape(4, 4)).ravel()
    np.testing.assert_allclose(w[:, col], ref, atol=1e-10)


def test_narrowband_limit_every_bin_is_spatial_fft(rng):
    # As fb -> 0, rho -> 0 and rho/fb -> 1/2: the steering of every frequency bin tends to
    # exp(j*pi*u_b*m), the narrowband spatial DFT. The deviation is O(rho*eps*M).
    fb = 1e-6
    pb = O.make_problem("ula", 8, 1, 8, 1, N=8, frac_bw=fb, delta_rel=1e-3)
    yhat = _crandn(rng, pb.M, pb.L)
    w = O.stage1_space(pb, yhat)
    sign = (-1.0) ** np.arange(pb.M)
    ref = pb.B * np.fft.ifft(sign[:, None] * yhat, axis=0)
    assert np.abs(w - ref).max() <= 10 * fb * pb.M * np.abs(yhat).sum(axis=0).max()


def test_time_origin_does_not_change_the_beam(rng):
    # The paper counts snapshots n = 1..N; the oracle uses 0..N-1. Shifting t_n by one sample
    # multiplies F and F_u by the same unitary diagonal, so bhat must not change.
    pb = O.make_problem("ula", 5, 1, 5, 1, N=8, frac_bw=0.5, delta_rel=1e-3)
    y = _crandn(rng, pb.M, pb.N)
    b = 3
    tau = pb.tau([b])[0]
    n1 = np.arange(1, pb.N + 1, dtype=np.float64)
    t_minus_tau = n1[None, :] - tau[:, None]
    F1 = (np.exp(-2j * np.pi * tau / pb.frac_bw)[:, None, None]
          * np.exp(2j * np.pi * pb.epsilon * np.multiply.outer(t_minus_tau, pb.lprime) / pb.L)).reshape(-1, pb.L)
    Fu1 = np.exp(2j * np.pi * pb.epsilon * np.multiply.outer(n1, pb.lprime) / pb.L)
    beta1 = np.linalg.solve(F1.conj().T @ F1 + pb.delta * np.eye(pb.L), F1.conj().T @ y.reshape(-1))
    np.testing.assert_allclose(O.fbst(pb, y[None], beams=[b])[0, 0], Fu1 @ beta1, atol=1e-9)


def test_gram_is_hermitian_positive_definite_toeplitz():
    pb = O.make_problem("ula", 12, 1, 12, 1, N=16, frac_bw=0.5, delta_rel=1e-3)
    for b in (0, 5, 11):
        A = O.gram(pb, b)
        np.testing.assert_allclose(A, A.conj().T, atol=1e-12 * np.abs(A).max())
        for d in range(-pb.L + 1, pb.L):
            diag = np.diagonal(A, offset=d)
            assert np.abs(diag - diag[0]).max() <= 1e-11 * np.abs(A).max()
        assert np.linalg.eigvalsh(A).min() > 0.5 * pb.delta


def test_solve_matches_augmented_least_squares(rng):
    pb = O.make_problem("ula", 6, 1, 6, 1, N=10, frac_bw=0.5, delta_rel=1e-3)
    y = _crandn(rng, pb.M, pb.N)
    fac = O.Stage2Factors(pb)
    beta = fac.coefficients(O.fan_coefficients(pb, y[None]))
    for b in range(pb.B):
        ref = O.lstsq_augmented(O.F_theta(pb, b), y.reshape(-1), pb.delta)
        np.testing.assert_allclose(beta[0, b], ref, rtol=0, atol=1e-9 * np.abs(ref).max())


def test_dense_operator_equals_solve_then_reconstruct(rng):
    pb = O.make_problem("ura", 3, 3, 3, 3, N=8, frac_bw=0.4, delta_rel=1e-3)
    y = _crandn(rng, 2, pb.M, pb.N)
    bh = O.fbst(pb, y)
    w = O.fan_coefficients(pb, y)
    for b in range(pb.B):
        G = O.dense_operator(pb, b)
        np.testing.assert_allclose(w[:, b] @ G.T, bh[:, b], atol=1e-9 * np.abs(bh).max())


def test_golden_tiny_closed_form():
    with open(os.path.join(GOLDEN, "tiny_closed_form.json")) as f:
        g = json.load(f)
    for c in g["cases"]:
        pb = O.make_problem("ula", 1, 1, 1, 1, N=1, frac_bw=c["frac_bw"], epsilon=c["epsilon"],
                            delta=c["delta"], L=2)
        y = np.array([[[c["y"][0] + 1j * c["y"][1]]]])
        out = O.fbst(pb, y)[0, 0, 0]
        assert abs(out - (c["bhat"][0] + 1j * c["bhat"][1])) < 1e-13


def test_golden_paper_parameters_and_snapshot_bound():
    with open(os.path.join(GOLDEN, "paper_parameters.json")) as f:
        g = json.load(f)
    fb = 2 * g["omega_ghz"] / g["f_c_ghz"]
    assert fb == g["expected"]["frac_bw"]
    pb = O.make_problem("ula", g["ula_elements"], 1, 4, 1, N=g["N"], frac_bw=fb, delta_rel=1e-3)
    assert abs(pb.rho - g["expected"]["rho"]) < 1e-15
    assert abs(g["f_c_ghz"] / (2 * g["omega_ghz"]) - g["expected"]["fc_Ts"]) < 1e-15
    # Eq. (8): N must exceed the largest aperture delay in samples (endfire, |u| = 1).
    ula_bound = pb.rho * (g["ula_elements"] - 1)
    side = g["upa_side"] - 1
    upa_bound = pb.rho * side * np.sqrt(2.0)  # max over the unit disk of |u*px + v*py| spans
    assert g["N"] > 2 * ula_bound and g["N"] > 2 * upa_bound


def test_single_sensor_limit_returns_the_samples(rng):
    # M = 1 and tau = 0: F = F_u, and F_u (N x L, L = 2N) has full row rank, so as delta -> 0
    # the regularised fit interpolates the data exactly: bhat = y.
    for N in (16, 64):
        pb = O.make_problem("ula", 1, 1, 1, 1, N=N, frac_bw=0.5, delta=1e-9)
        y = _crandn(rng, 1, 1, N)
        assert O.rel_l2(O.fbst(pb, y)[0, 0], y[0, 0]) < 1e-8


def test_plane_wave_from_grid_angle_is_reproduced(rng):
    # Noise-free plane wave from beam b's own direction: the beam is an estimate of s(t_n)
    # referenced to element 0. The paper gives no number for the bias (its formula needs Slepian
    # operators), so this is a sanity bound only -- the bias value itself is parity unpinned.
    for kind, mx, my, bx, by, b in (("ula", 16, 1, 16, 1, 11), ("ura", 4, 4, 4, 4, 9)):
        pb = O.make_problem(kind, mx, my, bx, by, N=64, frac_bw=0.5, delta_rel=1e-3)
        u, v = pb.directions[b]
        src = _toy_source(rng, u, v)
        y = array_record(pb.geom, [src], pb.frac_bw, pb.N, None, None)
        bh = O.fbst(pb, y[None])[0]
        s = waveform(src, np.arange(pb.N))
        assert O.rel_l2(bh[b], s) < 5e-3
        # A beam on the far side of the grid must not pass the wave.
        far = (b + pb.B // 2) % pb.B
        assert np.linalg.norm(bh[far]) < 0.3 * np.linalg.norm(s)


def test_noise_variance_matches_monte_carlo(rng):
    pb = O.make_problem("ula", 4, 1, 4, 1, N=16, frac_bw=0.5, delta_rel=1e-3)
    b, trials, sigma2 = 1, 400, 0.3
    fac = O.Stage2Factors(pb, [b])
    noise = _crandn(rng, trials, pb.M, pb.N) * np.sqrt(sigma2 / 2)
    bh = O.fbst(pb, noise, factors=fac)[:, 0]
    mc = np.mean(np.sum(np.abs(bh) ** 2, axis=1))
    pred = sigma2 * O.noise_power_trace(pb, b)
    assert abs(mc / pred - 1) < 3 * np.sqrt(2 / trials)


def test_noise_variance_tends_to_array_gain():
    # Sec. VII: the per-sample variance approaches sigma^2/M as N grows.
    M = 8
    ratios = []
    for N in (8, 16, 32, 64, 128):
        pb = O.make_problem("ula", M, 1, M, 1, N=N, frac_bw=0.5, delta_rel=1e-3)
        ratios.append(O.noise_power_trace(pb, 5) / N * M)
    assert all(r1 > r2 for r1, r2 in zip(ratios, ratios[1:]))
    assert 1.0 < ratios[-1] < 1.15


def test_tracks_exact_sinc_delay_and_sum(rng):
    # Brute-force broadband beamforming with exact (full-record) sinc delays on a tiny array at
    # 40 dB: both estimate s(t_n); the least-squares beam must be at least as good (+1e-3 slack).
    M, N, fb, b = 8, 64, 0.5, 5
    pb = O.make_problem("ula", M, 1, M, 1, N=N, frac_bw=fb, delta_rel=1e-3)
    u = pb.directions[b, 0]
    src = _toy_source(rng, u)
    total, t0 = 4096, 2000
    rec = array_record(ArrayGeometry("ula", M), [src], fb, total, 40.0, rng)
    bh = O.fbst(pb, rec[None, :, t0:t0 + N], beams=[b])[0, 0]
    s = waveform(src, np.arange(t0, t0 + N))
    ds = O.delay_and_sum_exact(rec, array_positions(ArrayGeometry("ula", M)), u, 0.0, fb,
                               np.arange(t0, t0 + N))
    assert O.rel_l2(bh, s) <= O.rel_l2(ds, s) + 1e-3
    assert O.rel_l2(bh, s) < 2e-2


def test_linearity(rng):
    pb = O.make_problem("ula", 6, 1, 5, 1, N=12, frac_bw=0.45, delta_rel=1e-3)
    y1, y2 = _crandn(rng, 2, pb.M, pb.N), _crandn(rng, 2, pb.M, pb.N)
    fac = O.Stage2Factors(pb)
    np.testing.assert_allclose(O.fbst(pb, y1 + 2 * y2, factors=fac),
                               O.fbst(pb, y1, factors=fac) + 2 * O.fbst(pb, y2, factors=fac), atol=1e-10)


def test_long_record_delay_and_sum_equals_the_direct_sinc_sum(rng):
    # The convolution form must be the same finite sinc series as the direct sum (brute force),
    # on a linear and a rectangular array, at output times near both record ends and inside.
    for kind, mx, my, u, v in (("ula", 6, 1, 0.37, 0.0), ("ura", 3, 3, -0.2, 0.55)):
        geom = ArrayGeometry(kind, mx, my)
        rec = _crandn(rng, geom.M, 300).astype(np.complex128)
        pos = array_positions(geom)
        n_out = np.array([0, 1, 17, 150, 298, 299])
        direct = O.delay_and_sum_exact(rec, pos, u, v, 0.4, n_out)
        conv = O.delay_and_sum_exact_record(rec, pos, u, v, 0.4, n_out)
        np.testing.assert_allclose(conv, direct, rtol=0, atol=1e-12 * np.abs(direct).max())


def test_stream_of_overlapping_blocks_tracks_a_plane_wave_better():
    # Sec. III-A's streaming remark: blocks every `hop` samples, each contributing its central hop
    # output samples. A noise-free plane wave from a grid beam pins the stream's time indexing (sample
    # j is the beam at record time c + j: one sample off would cost about the whole signal) and the
    # reason to overlap: dropping the block edges, where the Fourier extension fits worst, halves the
    # bias relative to non-overlapping blocks (hop = N).
    M, N, fb, b = 16, 64, 0.5, 5
    pb = O.make_problem("ula", M, 1, M, 1, N=N, frac_bw=fb, delta_rel=1e-3)
    rs = np.random.default_rng(4)
    Q = 64
    src = Source(pb.directions[b, 0], 0.0, (rs.standard_normal(Q) + 1j * rs.standard_normal(Q)) * np.sqrt(0.5 / Q),
                 rs.uniform(-0.5, 0.5, Q))
    T = 64 * 12
    rec = array_record(ArrayGeometry("ula", M), [src], fb, T, None, None)
    err = {}
    for hop in (64, 32):
        nblk = (T - N) // hop + 1
        out = O.fbst_stream(pb, rec, hop, nblk, beams=[b])[0]
        c = (N - hop) // 2
        err[hop] = O.rel_l2(out, waveform(src, np.arange(c, c + nblk * hop)))
        shifted = O.rel_l2(out, waveform(src, np.arange(c + 1, c + 1 + nblk * hop)))
        assert shifted > 0.1 > err[hop]
    assert err[32] < 0.5 * err[64]
    with pytest.raises(ValueError):
        O.fbst_stream(pb, rec, 33, 3)                 # N - hop must be even
