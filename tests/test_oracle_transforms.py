"""Pins of the oracle's transforms against the definition of the DFT.

The oracle's FFT is a radix-2 algorithm; these checks compare it with the
O(m^2) definition on tiny sizes, with numpy's FFT (a separate library
implementation, run, not copied), and with Parseval and round-trip identities.
"""
import numpy as np
import pytest

from conftest import rel


def brute_dft(x, sign=-1):
    m = len(x)
    j = np.arange(m)
    return np.array([np.sum(x * np.exp(sign * 2j * np.pi * j * k / m)) for k in range(m)])


def brute_dft2_half(f):
    n = f.shape[0]
    out = np.zeros((n, n // 2 + 1), complex)
    iy, ix = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    for q in range(n):
        for p in range(n // 2 + 1):
            out[q, p] = np.sum(f * np.exp(-2j * np.pi * (p * ix + q * iy) / n))
    return out


@pytest.mark.parametrize("m", [2, 4, 8, 16, 64])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft1d_matches_brute_force(orc, m, sign):
    rng = np.random.default_rng(m)
    x = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    # the O(m^2) sum itself carries about m * eps of rounding
    assert rel(orc.fft1d(x, sign), brute_dft(x, sign)) < max(1e-14, 4e-16 * m)


@pytest.mark.parametrize("n", [8, 16])
def test_r2c_matches_brute_force_2d(orc, n):
    f = np.random.default_rng(n).standard_normal((n, n))
    assert rel(orc.r2c(f), brute_dft2_half(f)) < 1e-14


@pytest.mark.parametrize("n", [8, 32, 64])
def test_r2c_c2r_against_numpy_and_roundtrip(orc, n):
    f = np.random.default_rng(100 + n).standard_normal((n, n))
    h = orc.r2c(f)
    assert rel(h, np.fft.rfft2(f)) < 1e-14
    assert rel(orc.c2r(h), f) < 1e-14
    # Parseval: sum f^2 = 1/n^2 sum_full |h|^2 (kx = 0 and n/2 columns once, others twice)
    w = np.full(h.shape, 2.0)
    w[:, 0] = 1.0
    w[:, -1] = 1.0
    assert abs(np.sum(f * f) - np.sum(w * np.abs(h) ** 2) / n**2) < 1e-12 * np.sum(f * f)


def test_single_mode_transform(orc):
    n = 16
    y, x = np.meshgrid(2 * np.pi * np.arange(n) / n, 2 * np.pi * np.arange(n) / n, indexing="ij")
    f = np.cos(3 * x - 2 * y)
    h = orc.r2c(f)
    expect = np.zeros_like(h)
    expect[(-2) % n, 3] = n * n / 2  # exp(i(3x - 2y)) component: kx = 3, ky = -2
    assert np.abs(h - expect).max() < 1e-12
