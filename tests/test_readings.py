"""numpy checks of the readings of the paper that the CUDA kernels implement (no GPU).

These restate, in plain numpy, the algebra the kernels rely on and compare it with library
routines, so that a misreading shows up on the CPU:
* Sec. V Gohberg-Semencul: A^{-1} = (1/x_0)[L(x)L(x)^H - L(ZJ conj x)L(ZJ conj x)^H] for Hermitian
  positive-definite Toeplitz A, applied through circulants of size >= 2L-1 (gs.cuh);
* the Levinson recursion for x = A^{-1} e_0 (plan.cu);
* Sec. IV / Eq. (7) chirp-z sums evaluated by Bluestein with the output (or input) split into
  halves that share one transform (stage1.cu, stage2.cu), with the same index maps.
"""
import numpy as np
import pytest
import scipy.linalg


def _hpd_toeplitz(rng, L):
    # Toeplitz Gram matrix of random exponentials plus a ridge: Hermitian positive definite.
    f = rng.uniform(-0.5, 0.5, 3 * L)
    a = np.array([np.sum(np.exp(2j * np.pi * f * d)) for d in range(L)])
    a[0] += 0.1 * L
    col = np.conj(a)                  # A[l, 0] = a(-l) = conj(a(l))
    return scipy.linalg.toeplitz(col, a), a


def _levinson(a):
    c = np.conj(a)
    f = np.zeros(len(a), complex)
    f[0] = 1 / c[0].real
    for k in range(1, len(a)):
        ef = np.sum(c[k:0:-1] * f[:k])
        fk = f[:k + 1].copy()
        f[:k + 1] = (fk - ef * np.conj(fk[::-1])) / (1 - abs(ef) ** 2)
    return f


def _L(c):
    return scipy.linalg.toeplitz(c, np.zeros(len(c)))


@pytest.mark.parametrize("L", [1, 2, 3, 8, 33, 64])
def test_levinson_and_gohberg_semencul_identity(rng, L):
    A, a = _hpd_toeplitz(rng, L)
    x = _levinson(a)
    np.testing.assert_allclose(x, np.linalg.solve(A, np.eye(L)[:, 0]), rtol=0, atol=1e-10 * np.abs(x).max())
    v = np.zeros(L, complex)
    v[1:] = np.conj(x[::-1][:-1])     # Z J conj(x)
    inv = (_L(x) @ _L(x).conj().T - _L(v) @ _L(v).conj().T) / x[0].real
    np.testing.assert_allclose(inv, np.linalg.inv(A), rtol=0, atol=1e-10 * np.abs(inv).max())


@pytest.mark.parametrize("L", [8, 24, 64])
def test_gs_apply_through_circulants(rng, L):
    A, a = _hpd_toeplitz(rng, L)
    x = _levinson(a)
    P = 1 << int(np.ceil(np.log2(2 * L - 1)))
    v = np.zeros(L, complex)
    v[1:] = np.conj(x[::-1][:-1])
    X = np.fft.fft(np.r_[x, np.zeros(P - L)] / np.sqrt(x[0].real)) / P
    V = np.fft.fft(np.r_[v, np.zeros(P - L)] / np.sqrt(x[0].real)) / P
    w = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    W = np.fft.fft(np.r_[w, np.zeros(P - L)])
    u1 = np.fft.ifft(W * np.conj(X)) * P
    u2 = np.fft.ifft(W * np.conj(V)) * P
    u1[L:] = 0
    u2[L:] = 0
    beta = (np.fft.ifft(X * np.fft.fft(u1) - V * np.fft.fft(u2)) * P)[:L]
    np.testing.assert_allclose(beta, np.linalg.solve(A, w), rtol=0, atol=1e-10 * np.abs(beta).max())


def _circ(g, dmin, dmax, P):
    out = np.zeros(P, complex)
    for d in range(dmin, dmax + 1):
        out[d % P] = g(d)
    return out


@pytest.mark.parametrize("N,L,eps,S", [(8, 16, 1.01, 2), (8, 16, 1.01, 1), (12, 30, 1.0, 2), (5, 10, 1.3, 1)])
def test_temporal_chirpz_split_bluestein(rng, N, L, eps, S):
    y = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    lp = np.arange(1, L + 1) - L / 2
    ref = np.exp(-2j * np.pi * eps * np.outer(lp, np.arange(N)) / L) @ y
    Lh = L // S
    P = 1 << int(np.ceil(np.log2(N + Lh - 1)))
    n = np.arange(N)
    Y = np.fft.fft(np.r_[y * np.exp(-1j * np.pi * eps * n ** 2 / L), np.zeros(P - N)])
    out = np.zeros(L, complex)
    for h in range(S):
        ch = h * Lh + 1 - L / 2
        G = np.fft.fft(_circ(lambda d: np.exp(1j * np.pi * eps * (d * d + 2 * ch * d) / L), -(N - 1), Lh - 1, P))
        r = np.fft.ifft(Y * G)[:Lh]
        i = np.arange(Lh)
        out[h * Lh:(h + 1) * Lh] = r * np.exp(-1j * np.pi * eps * (i * i + 2 * ch * i) / L)
    np.testing.assert_allclose(out, ref, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("N,L,eps,S", [(8, 16, 1.01, 2), (8, 16, 1.01, 1), (6, 20, 1.2, 2)])
def test_reconstruction_chirpz_split_bluestein(rng, N, L, eps, S):
    beta = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    lp = np.arange(1, L + 1) - L / 2
    ref = np.exp(2j * np.pi * eps * np.outer(np.arange(N), lp) / L) @ beta
    Lr = L // S
    P = 1 << int(np.ceil(np.log2(Lr + N - 1)))
    acc = np.zeros(P, complex)
    i = np.arange(Lr)
    for h in range(S):
        ch = h * Lr + 1 - L / 2
        x = beta[h * Lr:(h + 1) * Lr] * np.exp(1j * np.pi * eps * (i * i + 2 * ch * i) / L)
        Q = np.fft.fft(_circ(lambda d: np.exp(-1j * np.pi * eps * (d * d - 2 * ch * d) / L), -(Lr - 1), N - 1, P))
        acc += np.fft.fft(np.r_[x, np.zeros(P - Lr)]) * Q
    n = np.arange(N)
    out = np.fft.ifft(acc)[:N] * np.exp(1j * np.pi * eps * n ** 2 / L)
    np.testing.assert_allclose(out, ref, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("Ma,Ba,kappa", [(16, 16, 0.4), (13, 10, 0.37), (8, 20, 1.7)])
def test_spatial_chirpz_bluestein(rng, Ma, Ba, kappa):
    # w[b] = sum_m x[m] exp(2*pi*i*kappa*u_b*m), u_b = (2b - Ba)/Ba.
    x = rng.standard_normal(Ma) + 1j * rng.standard_normal(Ma)
    u = (2 * np.arange(Ba) - Ba) / Ba
    ref = np.exp(2j * np.pi * kappa * np.outer(u, np.arange(Ma))) @ x
    P = 1 << int(np.ceil(np.log2(Ma + Ba - 1)))
    m, b = np.arange(Ma), np.arange(Ba)
    pre = np.exp(2j * np.pi * kappa * (m * m - Ba * m) / Ba)
    K = np.fft.fft(_circ(lambda d: np.exp(-2j * np.pi * kappa * d * d / Ba), -(Ma - 1), Ba - 1, P))
    r = np.fft.ifft(np.fft.fft(np.r_[x * pre, np.zeros(P - Ma)]) * K)[:Ba]
    out = r * np.exp(2j * np.pi * kappa * b * b / Ba)
    np.testing.assert_allclose(out, ref, atol=1e-10 * np.abs(ref).max())
