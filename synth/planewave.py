"""Plane-wave array data from the paper's signal model (Sec. III, Eq. (1)).

Units: time is measured in samples (T_s = 1) and frequency in cycles per sample. The
experiments sample critically, f_s = 2*Omega (Sec. VI), so the baseband band [-Omega, Omega]
is [-1/2, 1/2] cycles per sample. The fractional bandwidth is fb = 2*Omega/f_c, which gives
f_c*T_s = 1/fb. Element positions are integer multiples of the half wavelength at the top of
the band, f_c + Omega (Sec. IV for the linear array, App. B for the planar array). A plane
wave with direction cosines (u, v) then reaches element p = (px, py) with delay

    tau_p / T_s = rho * (u*px + v*py),    rho = Omega / (f_c + Omega) = fb / (2 + fb),

and, after demodulation, the element records y_p[n] = exp(-2j*pi*f_c*tau_p) s(n - tau_p)
(Eq. (1)) plus white noise.

The waveform s(t) is a sum of Q complex sinusoids with frequencies drawn uniformly over the
band and independent CN(0, 1/Q) weights (the "sum of sinusoids" model of Sec. VI). It is
conditionally Gaussian, fills the band, has unit power, and its delayed values are known
exactly, which gives the tests an exact truth. Noise at a nominal SNR of S dB is CN(0, 10^(-S/10))
per sensor and sample, so each source has unit power against that noise.

Everything is generated in float64 from numpy's PCG64 and cast to complex64 at the end, so
both the oracle and the CUDA path see the same complex64 array.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class ArrayGeometry:
    """A linear array ("ula", mx elements) or an mx-by-my rectangular array on the half-wavelength
    grid, optionally moved off it by per-element offsets (a non-uniform array, Sec. IX)."""

    kind: str
    mx: int
    my: int = 1
    offsets: tuple | None = None  # M pairs (dx, dy), half wavelengths, added to the grid positions

    @property
    def M(self) -> int:
        return self.mx * self.my


def array_positions(geom: ArrayGeometry) -> np.ndarray:
    """Element positions in half wavelengths at f_c + Omega, shape (M, 2).

    Linear array: element m sits at (m, 0), m = 0..M-1. Rectangular array: element
    s = kx*my + ky sits at (kx, ky). Element 0 is the phase reference (zero delay).
    """
    if geom.kind == "ula":
        if geom.my != 1:
            raise ValueError("a linear array has my == 1")
        pos = np.stack([np.arange(geom.mx, dtype=np.float64), np.zeros(geom.mx)], axis=1)
    elif geom.kind == "ura":
        kx, ky = np.meshgrid(np.arange(geom.mx), np.arange(geom.my), indexing="ij")
        pos = np.stack([kx.ravel(), ky.ravel()], axis=1).astype(np.float64)
    else:
        raise ValueError(f"unknown array kind {geom.kind!r}")
    if geom.offsets is not None:
        pos = pos + np.asarray(geom.offsets, dtype=np.float64).reshape(geom.M, 2)
    return pos


def perturbed_geometry(kind: str, mx: int, my: int, sigma: float, seed: int) -> ArrayGeometry:
    """Grid positions moved by independent N(0, sigma^2) offsets in half wavelengths (along x only for
    a linear array), element 0 kept at the origin as the phase reference: non-uniform spacing
    emulated from a uniform array, as the experiments of Sec. IX do."""
    rng = np.random.Generator(np.random.PCG64(seed))
    off = rng.normal(0.0, sigma, (mx * my, 2))
    if kind == "ula":
        off[:, 1] = 0.0
    off[0] = 0.0
    return ArrayGeometry(kind, mx, my, tuple(map(tuple, off.tolist())))


@dataclass
class Source:
    """One plane wave: direction cosines (u, v) and its sum-of-sinusoids waveform."""

    u: float
    v: float
    amp: np.ndarray   # (Q,) complex weights
    freq: np.ndarray  # (Q,) frequencies in cycles per sample, inside [-1/2, 1/2]


def draw_sources(rng: np.random.Generator, K: int, kind: str, Q: int = 256) -> list[Source]:
    """K sources at random directions with independent band-filling waveforms.

    Linear array: theta ~ U(-pi/2, pi/2) and u = sin(theta). Rectangular array: (u, v) uniform
    over the unit disk (only physical directions).
    """
    out = []
    for _ in range(K):
        if kind == "ula":
            u, v = float(np.sin(rng.uniform(-np.pi / 2, np.pi / 2))), 0.0
        else:
            r, ph = np.sqrt(rng.uniform()), rng.uniform(0, 2 * np.pi)
            u, v = float(r * np.cos(ph)), float(r * np.sin(ph))
        amp = (rng.standard_normal(Q) + 1j * rng.standard_normal(Q)) * np.sqrt(0.5 / Q)
        freq = rng.uniform(-0.5, 0.5, Q)
        out.append(Source(u, v, amp, freq))
    return out


def waveform(src: Source, t: np.ndarray) -> np.ndarray:
    """s(t) = sum_q a_q exp(2j*pi*f_q*t) at the (real, possibly fractional) times t."""
    t = np.asarray(t, dtype=np.float64)
    return np.exp(2j * np.pi * np.multiply.outer(t, src.freq)) @ src.amp


def array_record(geom: ArrayGeometry, sources: list[Source], frac_bw: float, n_total: int,
                 snr_db: float | None, rng: np.random.Generator | None,
                 t0: int = 0) -> np.ndarray:
    """Demodulated array samples y[p, n] for n = t0..t0+n_total-1, complex128, shape (M, n_total).

    y_p[n] = sum_sources exp(-2j*pi*(1/fb)*tau_p) s(n - tau_p) + noise, with
    tau_p = rho*(u*px + v*py) samples. With snr_db=None no noise is added.
    """
    rho = frac_bw / (2.0 + frac_bw)
    pos = array_positions(geom)
    M = geom.M
    y = np.zeros((M, n_total), dtype=np.complex128)
    if sources:
        # Stack the sinusoids of all sources: y = coef (M x KQ) @ phase (KQ x n_total), where
        # coef[p, q] = a_q exp(-2j*pi*(1/fb + f_q)*tau_p) and phase[q, n] = exp(2j*pi*f_q*n).
        coef = []
        freqs = []
        for s in sources:
            tau = rho * (s.u * pos[:, 0] + s.v * pos[:, 1])
            coef.append(np.exp(-2j * np.pi * np.multiply.outer(tau, 1.0 / frac_bw + s.freq)) * s.amp)
            freqs.append(s.freq)
        coef = np.concatenate(coef, axis=1)
        freqs = np.concatenate(freqs)
        chunk = 4096
        for c0 in range(0, n_total, chunk):
            n = np.arange(t0 + c0, t0 + min(n_total, c0 + chunk), dtype=np.float64)
            y[:, c0:c0 + n.size] = coef @ np.exp(2j * np.pi * np.multiply.outer(freqs, n))
    if snr_db is not None:
        sigma2 = 10.0 ** (-snr_db / 10.0)
        y += (rng.standard_normal((M, n_total)) + 1j * rng.standard_normal((M, n_total))) * np.sqrt(sigma2 / 2)
    return y


def _blocks(record: np.ndarray, N: int, nblk: int) -> np.ndarray:
    """Cut an (M, nblk*N) record into contiguous blocks, layout [nblk][M][N], complex64."""
    M = record.shape[0]
    return np.ascontiguousarray(record[:, : nblk * N].reshape(M, nblk, N).transpose(1, 0, 2)).astype(np.complex64)


def ula_config(M: int, N: int, nblk: int, frac_bw: float, K: int, snr_db: float | None,
               seed: int, Q: int = 256, first_block: int = 0, geom: ArrayGeometry | None = None) -> dict:
    """One continuous record of K plane waves on an M-element linear array, cut into nblk blocks.
    With first_block > 0 the record starts first_block*N samples later in the same signal (same
    sources; the noise of that segment comes from its own child seed)."""
    ss = np.random.SeedSequence(seed)
    rs, rn = (np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(2))
    if first_block:
        rn = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, first_block])))
    geom = ArrayGeometry("ula", M) if geom is None else geom     # `geom` may move the elements (Sec. IX)
    src = draw_sources(rs, K, "ula", Q)
    rec = array_record(geom, src, frac_bw, nblk * N, snr_db, rn, t0=first_block * N)
    return {"geom": geom, "sources": src, "frac_bw": frac_bw, "N": N, "nblk": nblk,
            "y": _blocks(rec, N, nblk)}


def ura_config(mx: int, my: int, N: int, nblk: int, frac_bw: float, K: int, snr_db: float | None,
               seed: int, Q: int = 256, geom: ArrayGeometry | None = None) -> dict:
    """Same as ula_config for an mx-by-my rectangular array, sources uniform over the unit disk;
    `geom` may move the elements off the grid (the same sources, delays at the actual positions)."""
    ss = np.random.SeedSequence(seed)
    rs, rn = (np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(2))
    geom = geom if geom is not None else ArrayGeometry("ura", mx, my)
    src = draw_sources(rs, K, "ura", Q)
    rec = array_record(geom, src, frac_bw, nblk * N, snr_db, rn)
    return {"geom": geom, "sources": src, "frac_bw": frac_bw, "N": N, "nblk": nblk,
            "y": _blocks(rec, N, nblk)}


def interference_config(kind: str, mx: int, my: int, N: int, nblk: int, frac_bw: float,
                        source_dirs, interferer_dirs, inr_db: float, snr_db: float | None,
                        seed: int, Q: int = 256) -> dict:
    """Unit-power sources at source_dirs and interferers of power 10^(inr_db/10) at
    interferer_dirs (lists of direction cosines (u, v)), one record cut into nblk blocks."""
    ss = np.random.SeedSequence(seed)
    rs, rn = (np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(2))
    geom = ArrayGeometry(kind, mx, my)
    src = []
    for (u, v), power in [(d, 1.0) for d in source_dirs] + [(d, 10.0 ** (inr_db / 10.0)) for d in interferer_dirs]:
        amp = (rs.standard_normal(Q) + 1j * rs.standard_normal(Q)) * np.sqrt(0.5 * power / Q)
        src.append(Source(float(u), float(v), amp, rs.uniform(-0.5, 0.5, Q)))
    rec = array_record(geom, src, frac_bw, nblk * N, snr_db, rn)
    return {"geom": geom, "sources": src, "frac_bw": frac_bw, "N": N, "nblk": nblk,
            "y": _blocks(rec, N, nblk)}


def uneven_ula_instances(seed: int, count: int = 64, K: int = 4, snr_db: float = 15.0,
                         m_exponents=(5, 10), n_choices=(128, 256, 512, 1024),
                         fb_range=(0.2, 0.6), Q: int = 64, with_data: bool = True) -> list[dict]:
    """Independent linear arrays with M = 2^U{5..10}, N from n_choices, fb ~ U[0.2, 0.6] rounded
    to 1e-3, one block each, K sources and snr_db of noise, each drawn from its own child seed."""
    out = []
    for child in np.random.SeedSequence(seed).spawn(count):
        rp, rs, rn = (np.random.Generator(np.random.PCG64(s)) for s in child.spawn(3))
        M = 2 ** int(rp.integers(m_exponents[0], m_exponents[1] + 1))
        N = int(rp.choice(n_choices))
        fb = round(float(rp.uniform(*fb_range)), 3)
        inst = {"M": M, "N": N, "B": M, "frac_bw": fb}
        if with_data:
            geom = ArrayGeometry("ula", M)
            src = draw_sources(rs, K, "ula", Q)
            rec = array_record(geom, src, fb, N, snr_db, rn)
            inst["y"] = _blocks(rec, N, 1)
            inst["sources"] = src
        out.append(inst)
    return out
