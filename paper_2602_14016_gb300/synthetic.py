"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
comparisons.

This module holds no part of the assimilation arithmetic (no time stepping,
no adjoint, no preconditioner): it only draws seeded random fields with the
statistics of the paper's workloads.  Both the CUDA path and the CPU oracle
are fed the arrays it returns.

Conventions: physical fields are float64 arrays [iy, ix] on the n x n grid
x_j = 2 pi j / n; half spectra are numpy ``rfft2`` layouts [q, p] (ky index
q, kx = p), unnormalised forward transform.
"""
from __future__ import annotations

import numpy as np


def wavenumbers(n: int):
    """Signed integer wavenumbers (kx over the half spectrum, ky full)."""
    kx = np.arange(n // 2 + 1)
    ky = np.fft.fftfreq(n, 1.0 / n).astype(np.int64)
    return np.meshgrid(kx, ky)


def retained_mask(n: int) -> np.ndarray:
    """Square 2/3-rule truncation |kx|, |ky| <= floor((n-1)/3)."""
    KX, KY = wavenumbers(n)
    K = (n - 1) // 3
    return (np.abs(KX) <= K) & (np.abs(KY) <= K)


def energy_spectrum_shape(k: np.ndarray, k0: float = 4.0) -> np.ndarray:
    """E(k) proportional to k^4 exp(-2 (k/k0)^2), peaking at k = k0."""
    return k**4 * np.exp(-2.0 * (k / k0) ** 2)


def random_vorticity_hat(n: int, seed: int, k0: float = 4.0, energy: float = 1.0) -> np.ndarray:
    """Random-phase vorticity half spectrum on the retained set.

    Per-mode amplitude |w_hat(k)|^2 proportional to |k| E(|k|) (a shell of
    radius k holds about 2 pi k modes, and |w_hat|^2 = k^2 |u_hat|^2), phases
    from the DFT of seeded white noise (so the field is real), zero mean,
    scaled so that 1/2 <u^2 + v^2> over the grid equals ``energy``.
    """
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((n, n))
    h = np.fft.rfft2(noise)
    KX, KY = wavenumbers(n)
    k = np.sqrt(KX**2 + KY**2)
    amp = np.sqrt(k * energy_spectrum_shape(k, k0))
    mag = np.abs(h)
    h = np.where(mag > 0, h / np.where(mag > 0, mag, 1.0), 0.0) * amp
    h = np.where(retained_mask(n), h, 0.0)
    h[0, 0] = 0.0
    # enforce exact Hermitian symmetry of the kx = 0 column
    col = h[:, 0].copy()
    h[:, 0] = 0.5 * (col + np.conj(col[(-np.arange(n)) % n]))
    # kinetic energy 1/2 mean(u^2+v^2) = 1/(2 n^4) sum_full |w_hat|^2 / k^2
    wgt = np.where(KX == 0, 1.0, 2.0)
    k2 = np.where(k > 0, k * k, 1.0)
    e = 0.5 / n**4 * np.sum(wgt * np.abs(h) ** 2 / k2)
    return h * np.sqrt(energy / e)


def random_vorticity(n: int, seed: int, k0: float = 4.0, energy: float = 1.0) -> np.ndarray:
    """Physical counterpart of :func:`random_vorticity_hat`."""
    return np.fft.irfft2(random_vorticity_hat(n, seed, k0, energy), s=(n, n))


def random_field(n: int, seed: int) -> np.ndarray:
    """Seeded standard-normal grid field (directions for derivative checks)."""
    return np.random.default_rng(seed).standard_normal((n, n))


def random_retained_hat(n: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """DFT of a seeded white-noise field, restricted to the retained set."""
    h = np.fft.rfft2(np.random.default_rng(seed).standard_normal((n, n))) * scale
    return np.where(retained_mask(n), h, 0.0)


def unit_norm_terminal_hat(n: int, seed: int) -> np.ndarray:
    """White noise on the retained set, unit Euclidean norm over the grid."""
    h = random_retained_hat(n, seed)
    f = np.fft.irfft2(h, s=(n, n))
    return h / np.sqrt(np.sum(f * f))


def gaussian_draws(shape, seed: int) -> np.ndarray:
    """Seeded standard-normal draws (observation noise before scaling)."""
    return np.random.default_rng(seed).standard_normal(shape)
