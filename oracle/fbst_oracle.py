"""Plain FP64 CPU oracle of the fast broadband beamspace transform (FBST).

TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the benchmark's CPU-baseline
leg may import this module. The product path (the CUDA library and its Python binding) never
calls it, and it shares no code, tables or constants with that path.

What it computes. The FBST reaches exactly (up to rounding) the regularised least-squares beam
of Sec. III-A: for each beam b,

    w_b     = F_b^H y                               (Eq. (5), the fan of Sec. IV computes it)
    beta_b  = (F_b^H F_b + delta I)^{-1} w_b        (Eq. (5); Sec. V solves it fast)
    bhat_b  = F_u beta_b                            (Eq. (7))

with F_b the MN x L non-uniform Fourier matrix of Eq. (6) and F_u the N x L reconstruction
matrix of Eq. (7). So the oracle is that definition written out in float64 numpy:

* w_b by direct (non-FFT) sums, ordered as in Sec. IV: a direct sum over time for every sensor,
  then a direct sum over sensors for every frequency index (Eq. (9)-(12)).
* A_b = F_b^H F_b + delta I by direct sums. F_b factors as (carrier phase of the sensor) x
  (time part) x (delay part), so its Gram matrix is the elementwise product of the Gram matrix of
  the time part and that of the delay part; both are plain matrix products. No closed form and no
  Toeplitz shortcut is used.
* beta_b by dense LU (scipy.linalg.lu_factor / lu_solve), bhat_b by a dense product with F_u.

Conventions (0-based everywhere, units of samples, so T_s = 1):
* n = 0..N-1 (t_n = n), sensors m = 0..M-1 with positions p_m from synth.array_positions.
* ell = 0..L-1 stands for the paper's ell = 1..L, so ell' = (ell + 1) - L/2 (Eq. (3) and Eq. (12)).
* omega_ell * T_s = 2*pi*eps*ell'/L (Eq. (3)).
* Beams: u_b = -1 + 2b/B for a linear array; for an mx-by-my rectangular array b = a*by + c with
  (u_a, v_c) = (-1 + 2a/bx, -1 + 2c/by). (Eq. (11) is garbled for even B; this grid covers [-1, 1).)
* fb = 2*Omega/f_c, rho = fb/(2+fb), f_c*T_s = 1/fb and tau_{b,m} = rho*(u_b*px_m + v_b*py_m)
  (Sec. IV for the linear array, App. B for the planar array).
"""
from __future__ import annotations

from dataclasses import dataclass
from functools import cached_property

import numpy as np
import scipy.linalg

from synth.planewave import ArrayGeometry, array_positions

TWO_PI_J = 2j * np.pi


@dataclass(frozen=True)
class Problem:
    """One FBST problem: array, beam grid, block length and basis parameters."""

    geom: ArrayGeometry
    bx: int
    by: int
    N: int
    L: int
    frac_bw: float
    epsilon: float
    delta: float  # absolute regulariser delta of Eq. (5)

    @property
    def M(self) -> int:
        return self.geom.M

    @property
    def B(self) -> int:
        return self.bx * self.by

    @property
    def rho(self) -> float:
        return self.frac_bw / (2.0 + self.frac_bw)

    @cached_property
    def positions(self) -> np.ndarray:
        return array_positions(self.geom)

    @cached_property
    def directions(self) -> np.ndarray:
        """(B, 2) direction cosines of the beam grid."""
        if self.geom.kind == "ula":
            u = -1.0 + 2.0 * np.arange(self.bx) / self.bx
            return np.stack([u, np.zeros_like(u)], axis=1)
        a, c = np.meshgrid(np.arange(self.bx), np.arange(self.by), indexing="ij")
        return np.stack([-1.0 + 2.0 * a.ravel() / self.bx, -1.0 + 2.0 * c.ravel() / self.by], axis=1)

    @cached_property
    def lprime(self) -> np.ndarray:
        """ell' = ell - L/2 for the paper's ell = 1..L (Eq. (3))."""
        return np.arange(1, self.L + 1, dtype=np.float64) - self.L / 2

    def tau(self, beams=None, directions=None) -> np.ndarray:
        """tau_{b,m}/T_s = rho*(u_b*px_m + v_b*py_m), shape (len(beams), M); or, given
        `directions` ((n, 2) direction cosines, on or off the grid), the same for those."""
        if directions is not None:
            d = np.atleast_2d(np.asarray(directions, dtype=np.float64))
        else:
            d = self.directions if beams is None else self.directions[np.asarray(beams)]
        return self.rho * (d @ self.positions.T)


def make_problem(kind: str, mx: int, my: int, bx: int, by: int, N: int, frac_bw: float,
                 epsilon: float = 1.01, gamma: float = 2.0, delta: float | None = None,
                 delta_rel: float | None = None, L: int | None = None, offsets=None) -> Problem:
    """Build a Problem. L = gamma*N unless given. delta is absolute, or delta_rel*M*N. `offsets`
    (M pairs, half wavelengths) moves the elements off the grid: a non-uniform array (Sec. IX),
    for which every sum below is the same direct sum over the actual positions."""
    geom = ArrayGeometry(kind, mx, my, None if offsets is None else tuple(map(tuple, offsets)))
    if L is None:
        L = int(round(gamma * N))
    if delta is None:
        delta = float(delta_rel) * (geom.M * N)
    return Problem(geom, bx, by, N, L, float(frac_bw), float(epsilon), float(delta))


# ----------------------------------------------------------------------------------------------
# Explicit matrices (Eq. (6) and Eq. (7)) -- used directly on small problems and as pins.
# ----------------------------------------------------------------------------------------------

def F_theta(pb: Problem, b: int, direction=None) -> np.ndarray:
    """The MN x L matrix of Eq. (6) for beam b (or for the direction cosines `direction`, on or
    off the grid); row m*N + n is (sensor m, snapshot n).

    [F]_{(m,n), ell} = exp(-2j*pi*f_c*tau_m) * exp(j*omega_ell*(t_n - tau_m)).
    """
    tau = pb.tau([b])[0] if direction is None else pb.tau(directions=direction)[0]   # (M,)
    n = np.arange(pb.N, dtype=np.float64)
    t_minus_tau = n[None, :] - tau[:, None]   # (M, N)
    carrier = np.exp(-TWO_PI_J * tau / pb.frac_bw)[:, None, None]
    basis = np.exp(TWO_PI_J * pb.epsilon * np.multiply.outer(t_minus_tau, pb.lprime) / pb.L)
    return (carrier * basis).reshape(pb.M * pb.N, pb.L)


def F_u(pb: Problem) -> np.ndarray:
    """[F_u]_{n, ell} = exp(j*omega_ell*t_n) (Eq. (7)), shape (N, L)."""
    n = np.arange(pb.N, dtype=np.float64)
    return np.exp(TWO_PI_J * pb.epsilon * np.multiply.outer(n, pb.lprime) / pb.L)


# ----------------------------------------------------------------------------------------------
# Stage 1: w_b = F_b^H y by direct sums (Sec. IV, Eq. (9)-(12); App. B for the planar array)
# ----------------------------------------------------------------------------------------------

def stage1_time(pb: Problem, y: np.ndarray) -> np.ndarray:
    """yhat[..., m, ell] = sum_n y[..., m, n] exp(-2j*pi*eps*ell'*n/L)  (the first sum of Sec. IV).

    y has shape (..., M, N); the result has shape (..., M, L), complex128.
    """
    n = np.arange(pb.N, dtype=np.float64)
    E = np.exp(-TWO_PI_J * pb.epsilon * np.multiply.outer(n, pb.lprime) / pb.L)  # (N, L)
    return np.asarray(y, dtype=np.complex128) @ E


def stage1_space(pb: Problem, yhat: np.ndarray, beams=None, chunk: int = 64, directions=None) -> np.ndarray:
    """w[..., b, ell] = sum_m yhat[..., m, ell] exp(2j*pi*(1/fb + eps*ell'/L)*tau_{b,m}).

    This is the second sum of Sec. IV (and the two array sums of App. B written as one sum over
    the elements). yhat has shape (..., M, L); the result has shape (..., nbeams, L).
    """
    yhat = np.asarray(yhat, dtype=np.complex128)
    tau = pb.tau(beams, directions)                       # (nb, M)
    lead = yhat.shape[:-2]
    Y = yhat.reshape((-1,) + yhat.shape[-2:])             # (K, M, L)
    out = np.empty((Y.shape[0], tau.shape[0], pb.L), dtype=np.complex128)
    for l0 in range(0, pb.L, chunk):
        lp = pb.lprime[l0:l0 + chunk]
        kappa = 1.0 / pb.frac_bw + pb.epsilon * lp / pb.L           # (c,)
        S = np.exp(TWO_PI_J * kappa[:, None, None] * tau[None, :, :])  # (c, nb, M)
        # out[k, b, l] = sum_m S[l, b, m] * Y[k, m, l]
        out[:, :, l0:l0 + lp.size] = np.einsum("lbm,kml->kbl", S, Y[:, :, l0:l0 + lp.size], optimize=True)
    return out.reshape(lead + (tau.shape[0], pb.L))


def fan_coefficients(pb: Problem, y: np.ndarray, beams=None, directions=None) -> np.ndarray:
    """w = F_b^H y for every beam: (..., M, N) -> (..., nbeams, L); with `directions`, the exact
    coefficient vectors of those (possibly off-grid) directions instead."""
    return stage1_space(pb, stage1_time(pb, y), beams, directions=directions)


# ----------------------------------------------------------------------------------------------
# Stage 2: beta_b = (F_b^H F_b + delta I)^{-1} w_b, bhat_b = F_u beta_b (Eq. (5), Eq. (7), Sec. V)
# ----------------------------------------------------------------------------------------------

def gram(pb: Problem, b: int) -> np.ndarray:
    """A_b = F_b^H F_b + delta I of grid beam b (see gram_direction)."""
    return gram_direction(pb, pb.directions[b])


def gram_direction(pb: Problem, direction) -> np.ndarray:
    """A = F^H F + delta I by direct sums for the direction cosines `direction` = (u, v), on or off
    the grid (Eq. (5); its entries are those of Sec. V).

    With E[n, ell] = exp(j*omega_ell*t_n) and phi[ell, m] = exp(-j*omega_ell*tau_m), the entry
    [F_b]_{(m,n),ell} is carrier_m * E[n,ell] * phi[ell,m], so
    [F_b^H F_b]_{ell,k} = (sum_n conj(E[n,ell]) E[n,k]) * (sum_m conj(phi[ell,m]) phi[k,m]):
    the elementwise product of two Gram matrices (the unit-modulus carrier drops out).
    """
    E = F_u(pb)                                                                  # (N, L)
    tau = pb.tau(directions=direction)[0]
    phi = np.exp(-TWO_PI_J * pb.epsilon * np.multiply.outer(pb.lprime, tau) / pb.L)  # (L, M)
    A = (E.conj().T @ E) * (phi.conj() @ phi.T)
    A[np.diag_indices(pb.L)] += pb.delta
    return A


class Stage2Factors:
    """LU factors of every requested A_b, built once (the per-plan part of the oracle)."""

    def __init__(self, pb: Problem, beams=None):
        self.pb = pb
        self.beams = np.arange(pb.B) if beams is None else np.asarray(beams)
        self.Fu = F_u(pb)
        self.lu = [scipy.linalg.lu_factor(gram(pb, int(b))) for b in self.beams]

    def apply(self, w: np.ndarray) -> np.ndarray:
        """w: (nblk, nbeams, L) in the order of self.beams -> bhat: (nblk, nbeams, N)."""
        w = np.asarray(w, dtype=np.complex128)
        out = np.empty(w.shape[:-1] + (self.pb.N,), dtype=np.complex128)
        for i, lu in enumerate(self.lu):
            beta = scipy.linalg.lu_solve(lu, w[:, i, :].T)      # (L, nblk)
            out[:, i, :] = (self.Fu @ beta).T
        return out

    def coefficients(self, w: np.ndarray) -> np.ndarray:
        """beta = A_b^{-1} w_b for every requested beam, shape (nblk, nbeams, L)."""
        w = np.asarray(w, dtype=np.complex128)
        out = np.empty_like(w)
        for i, lu in enumerate(self.lu):
            out[:, i, :] = scipy.linalg.lu_solve(lu, w[:, i, :].T).T
        return out


def fbst(pb: Problem, y: np.ndarray, beams=None, factors: Stage2Factors | None = None) -> np.ndarray:
    """Full FBST: y (nblk, M, N) -> bhat (nblk, nbeams, N), complex128."""
    y = np.asarray(y)
    if y.ndim == 2:
        y = y[None]
    if factors is None:
        factors = Stage2Factors(pb, beams)
    w = fan_coefficients(pb, y, factors.beams)
    return factors.apply(w)


def dense_operator(pb: Problem, b: int) -> np.ndarray:
    """G_b = F_u A_b^{-1} (N x L), the precomputed operator of Sec. III-B / Sec. V."""
    A = gram(pb, b)
    # G_b = F_u A^{-1}  <=>  G_b^T = A^{-T} F_u^T, and A^T = conj(A) for Hermitian A.
    return scipy.linalg.solve(A.T, F_u(pb).T).T


# ----------------------------------------------------------------------------------------------
# Beamspace interference nulling (Sec. VIII-B, Eq. (14))
# ----------------------------------------------------------------------------------------------

def cross_gram(pb: Problem, b: int, p: int) -> np.ndarray:
    """F_b^H F_p for grid beams b and p (see cross_gram_direction)."""
    return cross_gram_direction(pb, b, pb.directions[p])


def cross_gram_direction(pb: Problem, b: int, direction) -> np.ndarray:
    """F_b^H F_p (L x L) for grid beam b and the direction cosines `direction` of p (on or off the
    grid) by direct sums: the product inside G_p of Eq. (14).

    As in gram(), [F_b]_{(m,n),ell} = c_{b,m} * E[n,ell] * phi_b[ell,m] with the carrier
    c_{b,m} = exp(-2j*pi*tau_{b,m}/fb), so
    [F_b^H F_p]_{ell,k} = (sum_n conj(E[n,ell]) E[n,k]) * (sum_m conj(c_{b,m} phi_b[ell,m]) c_{p,m} phi_p[k,m]).
    For b != p the carriers no longer cancel and the element sum is not a function of k - ell.
    """
    E = F_u(pb)                                                                   # (N, L)
    tb, tp = pb.tau([b])[0], pb.tau(directions=direction)[0]                      # (M,)
    el = lambda tau: (np.exp(-TWO_PI_J * tau / pb.frac_bw)[None, :]
                      * np.exp(-TWO_PI_J * pb.epsilon * np.multiply.outer(pb.lprime, tau) / pb.L))  # (L, M)
    return (E.conj().T @ E) * (el(tb).conj() @ el(tp).T)


class NullingFactors:
    """Per-plan part of Eq. (14): the stage-2 factors of the output beams and of the interferer
    beams, and the cross Gram matrices F_b^H F_p of every (output beam, interferer) pair."""

    def __init__(self, pb: Problem, interferers, beams=None):
        self.pb = pb
        self.interferers = [int(p) for p in interferers]
        self.out = Stage2Factors(pb, beams)
        self.intf = Stage2Factors(pb, self.interferers)
        self.C = [[cross_gram(pb, int(b), p) for p in self.interferers] for b in self.out.beams]

    def coefficients(self, w: np.ndarray, w_int: np.ndarray) -> np.ndarray:
        """The bracket of Eq. (14), w_b - sum_p F_b^H F_p (F_p^H F_p + delta I)^{-1} w_p.

        w: (nblk, nbeams, L) for the output beams, w_int: (nblk, P, L) for the interferer beams.
        """
        w = np.asarray(w, dtype=np.complex128)
        out = w.copy()
        if self.interferers:
            beta_int = self.intf.coefficients(w_int)                     # (nblk, P, L)
            for i in range(len(self.out.beams)):
                for j in range(len(self.interferers)):
                    out[:, i, :] -= beta_int[:, j, :] @ self.C[i][j].T
        return out


def fbst_nulled(pb: Problem, y: np.ndarray, interferers, beams=None,
                factors: NullingFactors | None = None) -> np.ndarray:
    """FBST with beamspace nulling of the interferer beams (Eq. (14)): y (nblk, M, N) -> bhat
    (nblk, nbeams, N) with bhat_b = F_u A_b^{-1} (w_b - sum_p F_b^H F_p A_p^{-1} w_p)."""
    y = np.asarray(y)
    if y.ndim == 2:
        y = y[None]
    if factors is None:
        factors = NullingFactors(pb, interferers, beams)
    w = fan_coefficients(pb, y, factors.out.beams)
    w_int = fan_coefficients(pb, y, factors.interferers) if factors.interferers else None
    return factors.out.apply(factors.coefficients(w, w_int))


def F_u_interval(pb: Problem, n0: int, Nu: int) -> np.ndarray:
    """[F_u]_{n, ell} = exp(j*omega_ell*t_n) (Eq. (7)) on the samples t_n = n0 .. n0 + Nu - 1,
    shape (Nu, L); n0 = 0, Nu = N is the block's own F_u."""
    n = n0 + np.arange(Nu, dtype=np.float64)
    return np.exp(TWO_PI_J * pb.epsilon * np.multiply.outer(n, pb.lprime) / pb.L)


def time_interval(pb: Problem) -> tuple:
    """The broader reconstruction interval of the time-domain nulling (Eq. (15)): 2L samples centred
    on the block, t = -(2L - N)/2 .. (2L + N)/2 - 1. Its F_u has full column rank and stays well
    conditioned (about 2 to 10 up to L = 1024): the frequencies eps*ell'/L span 1.01 cycles per
    sample, so near +-1/2 cycle the two ends of the set interleave at twice the density, and an
    interval of only L samples cannot resolve them (condition number 58 at L = 128, 3e10 at
    L = 512)."""
    return -((2 * pb.L - pb.N) // 2), 2 * pb.L


class TimeNullingFactors:
    """Eq. (15): the nulled time-domain beam y~_b = y_b - sum_p G'_{b,p} y_p, windowed to the block,
    with y_b = F_u beta_b the plain beam over the block's N samples, y_p = F_x beta_p the interferer
    beam over the broader interval (F_x = F_u on that interval), and
    G'_{b,p} = F_u H_{b,p} F_x^+,   H_{b,p} = (F_b^H F_b + delta I)^{-1} F_b^H F_p.
    The matrices are formed literally: F_x^+ by the pseudo-inverse, H by a dense solve."""

    def __init__(self, pb: Problem, interferers, beams=None, n0: int | None = None, Nu: int | None = None):
        self.pb = pb
        self.interferers = [int(p) for p in interferers]
        d0, dN = time_interval(pb)
        self.n0, self.Nu = (d0 if n0 is None else int(n0)), (dN if Nu is None else int(Nu))
        self.Fx = F_u_interval(pb, self.n0, self.Nu)                   # (Nu, L)
        self.Fx_pinv = np.linalg.pinv(self.Fx)                         # (L, Nu)
        self.out = Stage2Factors(pb, beams)
        self.intf = Stage2Factors(pb, self.interferers)
        Fu = F_u(pb)
        self.Gp = []
        for b in self.out.beams:
            A = gram(pb, int(b))
            row = []
            for p in self.interferers:
                H = scipy.linalg.solve(A, cross_gram(pb, int(b), p))  # (L, L)
                row.append(Fu @ H @ self.Fx_pinv)                      # (N, Nu)
            self.Gp.append(row)

    def interferer_beams(self, w_int: np.ndarray) -> np.ndarray:
        """The interferers' time-domain beams over the broader interval, F_x A_p^{-1} w_p:
        (nblk, P, L) -> (nblk, P, Nu)."""
        beta = self.intf.coefficients(w_int)
        return np.einsum("nl,bpl->bpn", self.Fx, beta)

    def apply(self, y: np.ndarray, y_int: np.ndarray) -> np.ndarray:
        """Eq. (15) on time-domain beams: y (nblk, nbeams, N), y_int (nblk, P, Nu) -> y~."""
        out = np.array(y, dtype=np.complex128)
        for i in range(len(self.out.beams)):
            for j in range(len(self.interferers)):
                out[:, i, :] -= np.asarray(y_int[:, j, :], dtype=np.complex128) @ self.Gp[i][j].T
        return out


def fbst_nulled_time(pb: Problem, y: np.ndarray, interferers, beams=None,
                     factors: TimeNullingFactors | None = None) -> np.ndarray:
    """FBST followed by the time-domain nulling of Eq. (15): y (nblk, M, N) -> y~ (nblk, nbeams, N)."""
    y = np.asarray(y)
    if y.ndim == 2:
        y = y[None]
    if factors is None:
        factors = TimeNullingFactors(pb, interferers, beams)
    w = fan_coefficients(pb, y, factors.out.beams)
    plain = factors.out.apply(w)
    w_int = fan_coefficients(pb, y, factors.interferers)
    return factors.apply(plain, factors.interferer_beams(w_int))


# ----------------------------------------------------------------------------------------------
# Off-grid beams by interpolation of beam vectors (Sec. VIII-A)
# ----------------------------------------------------------------------------------------------

def natural_spline_weights(x: np.ndarray, xq: float) -> np.ndarray:
    """Weights c with s(xq) = sum_i c_i f_i, where s is the natural cubic spline through the points
    (x_i, f_i) (x increasing): cubic on every interval, continuous with its first and second
    derivatives at the inner knots, second derivative zero at both ends. The spline is linear in
    the data, so c_i is the spline of the unit data e_i evaluated at xq.

    With h_i = x_{i+1} - x_i and moments s''(x_i) = Mo_i, the inner conditions read
    h_{i-1} Mo_{i-1} + 2 (h_{i-1} + h_i) Mo_i + h_i Mo_{i+1} = 6 ((f_{i+1} - f_i)/h_i - (f_i - f_{i-1})/h_{i-1})
    with Mo_0 = Mo_{n-1} = 0; on [x_i, x_{i+1}] with a = x_{i+1} - xq, b = xq - x_i,
    s = (Mo_i a^3 + Mo_{i+1} b^3) / (6 h_i) + (f_i - Mo_i h_i^2 / 6) a / h_i + (f_{i+1} - Mo_{i+1} h_i^2 / 6) b / h_i.
    """
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    if n == 1:
        return np.ones(1)
    h = np.diff(x)
    F = np.eye(n)                                  # column j: the unit data e_j
    Mo = np.zeros((n, n))
    if n > 2:
        A = np.zeros((n - 2, n - 2))
        rhs = np.zeros((n - 2, n))
        for r, i in enumerate(range(1, n - 1)):
            if r > 0:
                A[r, r - 1] = h[i - 1]
            A[r, r] = 2.0 * (h[i - 1] + h[i])
            if r < n - 3:
                A[r, r + 1] = h[i]
            rhs[r] = 6.0 * ((F[i + 1] - F[i]) / h[i] - (F[i] - F[i - 1]) / h[i - 1])
        Mo[1:n - 1] = np.linalg.solve(A, rhs)
    i = int(np.clip(np.searchsorted(x, xq, side="right") - 1, 0, n - 2))
    a, b = x[i + 1] - xq, xq - x[i]
    return ((Mo[i] * a ** 3 + Mo[i + 1] * b ** 3) / (6.0 * h[i])
            + (F[i] - Mo[i] * h[i] ** 2 / 6.0) * a / h[i] + (F[i + 1] - Mo[i + 1] * h[i] ** 2 / 6.0) * b / h[i])


def interp_window(n_grid: int, coord: float, K: int = 8) -> int:
    """First index of the K consecutive grid indices around the continuous grid coordinate `coord`
    (K/2 on each side of the interval that holds it), moved inward at the ends of the grid."""
    K = min(K, n_grid)
    first = int(np.floor(coord)) - (K // 2 - 1)
    return int(min(max(first, 0), n_grid - K))


def offgrid_terms(pb: Problem, direction, K: int = 8) -> list:
    """(grid beam, weight) pairs that form the interpolated beam vector of `direction` = (u, v):
    a natural cubic spline along u through the K nearest grid beams (the beam grid is uniform in
    the direction cosine, u_a = -1 + 2a/bx), and for a rectangular array the same along v (the
    tensor product of the two one-dimensional splines)."""
    u, v = float(direction[0]), float(direction[1])

    def axis(nb, c):
        coord = (c + 1.0) * nb / 2.0                 # grid index of c (u_a = -1 + 2a/nb)
        first = interp_window(nb, coord, K)
        k = min(K, nb)
        idx = np.arange(first, first + k)
        return idx, natural_spline_weights(-1.0 + 2.0 * idx / nb, c)

    ia, wa = axis(pb.bx, u)
    if pb.geom.kind == "ula":
        return [(int(a), float(w)) for a, w in zip(ia, wa)]
    ic, wc = axis(pb.by, v)
    return [(int(a) * pb.by + int(c), float(x * z)) for a, x in zip(ia, wa) for c, z in zip(ic, wc)]


class OffGridFactors:
    """Per-plan part of the off-grid beams of Sec. VIII-A: the interpolation terms of every
    requested direction and the LU factors of its own A = F^H F + delta I (an off-grid direction
    has its own regularised least-squares problem, Eq. (5))."""

    def __init__(self, pb: Problem, directions, K: int = 8):
        self.pb = pb
        self.directions = np.atleast_2d(np.asarray(directions, dtype=np.float64))
        self.terms = [offgrid_terms(pb, d, K) for d in self.directions]
        self.beams = sorted({b for t in self.terms for b, _ in t})
        self.Fu = F_u(pb)
        self.lu = [scipy.linalg.lu_factor(gram_direction(pb, d)) for d in self.directions]

    def interpolate(self, w_grid: np.ndarray) -> np.ndarray:
        """w_grid: (nblk, B, L), every grid beam -> interpolated (nblk, ndirs, L)."""
        w_grid = np.asarray(w_grid, dtype=np.complex128)
        out = np.zeros(w_grid.shape[:-2] + (len(self.terms), self.pb.L), dtype=np.complex128)
        for k, t in enumerate(self.terms):
            for b, c in t:
                out[..., k, :] += c * w_grid[..., b, :]
        return out

    def apply(self, wstar: np.ndarray) -> np.ndarray:
        """Stage 2 of the off-grid directions: (nblk, ndirs, L) -> (nblk, ndirs, N)."""
        wstar = np.asarray(wstar, dtype=np.complex128)
        out = np.empty(wstar.shape[:-1] + (self.pb.N,), dtype=np.complex128)
        for i, lu in enumerate(self.lu):
            out[:, i, :] = (self.Fu @ scipy.linalg.lu_solve(lu, wstar[:, i, :].T)).T
        return out


def fbst_offgrid(pb: Problem, y: np.ndarray, directions, factors: OffGridFactors | None = None) -> np.ndarray:
    """Off-grid beams (Sec. VIII-A): y (nblk, M, N) -> (nblk, ndirs, N), the beam vector of each
    direction interpolated from the grid beams' w_b, then F_u A^{-1} of that direction."""
    y = np.asarray(y)
    if y.ndim == 2:
        y = y[None]
    if factors is None:
        factors = OffGridFactors(pb, directions)
    w = np.zeros(y.shape[:-2] + (pb.B, pb.L), dtype=np.complex128)
    w[..., factors.beams, :] = fan_coefficients(pb, y, factors.beams)
    return factors.apply(factors.interpolate(w))


class OffGridNullingFactors:
    """Eq. (14) for interferers at arbitrary directions (Sec. VIII-B: exact alignment with the grid
    is not required): each interferer's vector w_p is interpolated from the grid beam vectors as in
    Sec. VIII-A, and G_p = F^H F_p (F_p^H F_p + delta I)^{-1} uses that direction's own F_p."""

    def __init__(self, pb: Problem, directions, beams=None, K: int = 8):
        self.pb = pb
        self.out = Stage2Factors(pb, beams)
        self.intf = OffGridFactors(pb, directions, K)         # interpolation terms and LU of each A_p
        self.C = [[cross_gram_direction(pb, int(b), d) for d in self.intf.directions] for b in self.out.beams]

    def coefficients(self, w: np.ndarray, w_grid: np.ndarray) -> np.ndarray:
        """The bracket of Eq. (14): w (nblk, nbeams, L) of the output beams, w_grid (nblk, B, L)
        every grid beam (the interferers' vectors are interpolated from it)."""
        w = np.asarray(w, dtype=np.complex128)
        w_int = self.intf.interpolate(w_grid)                               # (nblk, P, L)
        out = w.copy()
        for j, lu in enumerate(self.intf.lu):
            beta = scipy.linalg.lu_solve(lu, w_int[:, j, :].T).T          # (nblk, L)
            for i in range(len(self.out.beams)):
                out[:, i, :] -= beta @ self.C[i][j].T
        return out


def fbst_nulled_offgrid(pb: Problem, y: np.ndarray, directions, beams=None,
                        factors: OffGridNullingFactors | None = None) -> np.ndarray:
    """FBST with beamspace nulling of interferers at the given directions (Eq. (14), Sec. VIII-A/B):
    y (nblk, M, N) -> (nblk, nbeams, N)."""
    y = np.asarray(y)
    if y.ndim == 2:
        y = y[None]
    if factors is None:
        factors = OffGridNullingFactors(pb, directions, beams)
    w_grid = fan_coefficients(pb, y)
    return factors.out.apply(factors.coefficients(w_grid[:, factors.out.beams], w_grid))


# ----------------------------------------------------------------------------------------------
# Streaming over contiguous, overlapping blocks (Sec. III-A, streaming remark)
# ----------------------------------------------------------------------------------------------

def stream_blocks(record: np.ndarray, N: int, hop: int, nblk: int) -> np.ndarray:
    """Blocks k = 0..nblk-1 of N snapshots starting every `hop` samples of a continuous record
    (M, T): (nblk, M, N)."""
    return np.stack([record[:, k * hop:k * hop + N] for k in range(nblk)])


def fbst_stream(pb: Problem, record: np.ndarray, hop: int, nblk: int, beams=None,
                factors: Stage2Factors | None = None) -> np.ndarray:
    """The beams of a continuous record from overlapping blocks: block k covers samples
    [k*hop, k*hop + N) and contributes its central `hop` output samples, [c, c + hop) with
    c = (N - hop)/2, at stream times k*hop + c + i. Returns (nbeams, nblk*hop); stream sample j is
    the beam at record time c + j."""
    if (pb.N - hop) % 2 or not 1 <= hop <= pb.N:
        raise ValueError("hop must be in [1, N] with N - hop even")
    c = (pb.N - hop) // 2
    bh = fbst(pb, stream_blocks(record, pb.N, hop, nblk), beams=beams, factors=factors)   # (nblk, nb, N)
    return np.concatenate([bh[k, :, c:c + hop] for k in range(nblk)], axis=1)


# ----------------------------------------------------------------------------------------------
# Tools used by the pins (not part of the method)
# ----------------------------------------------------------------------------------------------

def lstsq_augmented(F: np.ndarray, y: np.ndarray, delta: float) -> np.ndarray:
    """argmin ||F beta - y||^2 + delta ||beta||^2 by QR least squares on [F; sqrt(delta) I]."""
    L = F.shape[1]
    Fa = np.vstack([F, np.sqrt(delta) * np.eye(L)])
    ya = np.concatenate([y, np.zeros(L, dtype=np.complex128)])
    return np.linalg.lstsq(Fa, ya, rcond=None)[0]


def noise_power_trace(pb: Problem, b: int) -> float:
    """sigma^-2 E||F_u A^{-1} F^H n||^2 = tr(F_u A^{-1} F^H F A^{-1} F_u^H) for white noise n.

    The discrete analogue of the variance expression of Sec. VII (the paper integrates r(t,t)
    over [0, T]; here the beam is read at the N sample times instead).
    """
    F = F_theta(pb, b)
    A = gram(pb, b)
    K = np.linalg.solve(A, F.conj().T)          # A^{-1} F^H  (L x MN)
    Op = F_u(pb) @ K                            # N x MN
    return float(np.real(np.vdot(Op, Op)))


def delay_and_sum_exact(record: np.ndarray, positions: np.ndarray, u: float, v: float,
                        frac_bw: float, n_out: np.ndarray) -> np.ndarray:
    """Delay-and-sum with exact (full-record) sinc fractional delays (Sec. III, before Eq. (2)).

    b(t_n) = (1/M) sum_m exp(2j*pi*f_c*tau_m) y_m(t_n + tau_m), with y_m(t) rebuilt from all of
    its samples by the sinc series y_m(t) = sum_k y_m[k] sinc(t - k). record: (M, n_total).
    """
    rho = frac_bw / (2.0 + frac_bw)
    tau = rho * (u * positions[:, 0] + v * positions[:, 1])
    k = np.arange(record.shape[1], dtype=np.float64)
    out = np.zeros(len(n_out), dtype=np.complex128)
    for m in range(record.shape[0]):
        t = np.asarray(n_out, dtype=np.float64) + tau[m]
        interp = np.sinc(np.subtract.outer(t, k)) @ record[m]
        out += np.exp(TWO_PI_J * tau[m] / frac_bw) * interp
    return out / record.shape[0]


def delay_and_sum_exact_record(record: np.ndarray, positions: np.ndarray, u: float, v: float,
                               frac_bw: float, n_out: np.ndarray) -> np.ndarray:
    """The same exact-sinc delay-and-sum as delay_and_sum_exact, for long records.

    For element m every output time t_n + tau_m has the same fractional part, so the sinc series
    sum_k y_m[k] sinc(n + tau_m - k) over the whole record is the full linear convolution of y_m
    with the sampled kernel h_m[j] = sinc(j + tau_m), j = -(K-1)..K-1, read at n. The convolution
    is taken with scipy's FFT convolution (a library primitive); nothing is truncated.
    """
    import scipy.signal
    rho = frac_bw / (2.0 + frac_bw)
    tau = rho * (u * positions[:, 0] + v * positions[:, 1])
    K = record.shape[1]
    j = np.arange(-(K - 1), K, dtype=np.float64)
    idx = np.asarray(n_out, dtype=np.int64) + (K - 1)
    out = np.zeros(len(idx), dtype=np.complex128)
    for m in range(record.shape[0]):
        full = scipy.signal.fftconvolve(np.asarray(record[m], dtype=np.complex128), np.sinc(j + tau[m]))
        out += np.exp(TWO_PI_J * tau[m] / frac_bw) * full[idx]
    return out / record.shape[0]


def rel_l2(a: np.ndarray, b: np.ndarray) -> float:
    """||a - b||_2 / ||b||_2 over all entries."""
    a = np.asarray(a, dtype=np.complex128).ravel()
    b = np.asarray(b, dtype=np.complex128).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
