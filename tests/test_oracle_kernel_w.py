"""Pins of the oracle's control multiplier m(k) = |k| W(k)^{1/2} (Eq. 18-19)
for every kernel family of Sec. III.B and the task's exp(-a|k|).

The multiplier is read off single Fourier modes: s = cos(kx x + ky y) has a
known DFT (numpy), so w0_hat / DFT(s) at that mode is m(k).  Two kinds of
pins, neither a retyping of the oracle's formula:

- exact values that special parameters fix: with a = ln 4 the exponential
  kernel gives m = |k| 2^{-|k|} (1/2 at |k| = 1 and 2, 5/32 at |k| = 5);
  |k|^{-2 alpha} gives integer or half-integer powers of 5 at mode (3, 4);
  the heat kernel with nu beta = ln 2 gives |k| 2^{-k^2/2}; a table of
  4^{-|kx|} 9^{-|ky|} gives |k| 2^{-|kx|} 3^{-|ky|} (not symmetric in kx,
  ky, so a transposed table index fails);
- identities of the families over every retained mode at the sweep's own
  parameters: m_a m_b = |k| m_{a+b} (exponential semigroups), m_alpha
  m_{2-alpha} = 1 (fractional powers), exp(-nu beta k^2) depends on nu and
  beta only through nu beta (so nu cannot be dropped), m = 0 at k = 0 and
  outside the 2/3-rule set.
"""
import math

import numpy as np
import pytest

from paper_2602_14016_gb300 import synthetic

N = 16  # K = 5: modes up to |kx|, |ky| <= 5 are retained


def _grid(n):
    return np.meshgrid(2 * np.pi * np.arange(n) / n, 2 * np.pi * np.arange(n) / n, indexing="ij")


def problem(orc, kernel, kp, nu=1e-2, table=None, n=N):
    return orc.Problem(n=n, nsteps=1, dt=1e-3, nu=nu, px=4, every=1, kernel=kernel, kparam=kp, ktable=table)


def mode_multiplier(orc, P, kx, ky):
    """w0_hat / DFT(s) at (ky, kx) for s = cos(kx x + ky y)."""
    n = P.n
    y, x = _grid(n)
    s = np.cos(kx * x + ky * y)
    S = np.fft.rfft2(s)
    w0 = orc.omega_from_control(P, s)
    q = ky % n
    m = w0[q, kx] / S[q, kx]
    assert abs(m.imag) <= 1e-14 * max(abs(m.real), 1.0)
    return m.real


def all_multipliers(orc, P):
    """m(k) on every half-spectrum mode, from one random field."""
    n = P.n
    s = synthetic.random_field(n, 5)
    S = np.fft.rfft2(s)
    w0 = orc.omega_from_control(P, s)
    return w0 / S


def lattice_k(n):
    KX, KY = synthetic.wavenumbers(n)
    return np.sqrt(KX**2 + KY**2), KX, KY


EXACT = [
    # (kernel, param, nu, [(kx, ky, exact m)])
    ("identity", 0.0, 1e-2, [(3, 4, 5.0), (1, 0, 1.0), (0, 5, 5.0)]),
    ("exp_abs", math.log(4.0), 1e-2, [(1, 0, 0.5), (0, 2, 0.5), (3, 4, 5 / 32), (4, -3, 5 / 32), (5, 0, 5 / 32)]),
    ("frac", 0.0, 1e-2, [(3, 4, 5.0), (0, 2, 2.0)]),
    ("frac", 0.5, 1e-2, [(0, 4, 2.0), (3, 4, math.sqrt(5.0))]),
    ("frac", 1.0, 1e-2, [(3, 4, 1.0), (1, 1, 1.0), (0, 5, 1.0)]),
    ("frac", 1.5, 1e-2, [(0, 4, 0.5), (3, -4, 1 / math.sqrt(5.0))]),
    ("frac", -1.0, 1e-2, [(3, 4, 25.0), (1, 1, 2.0)]),
    ("exp_sq", 100 * math.log(2.0), 1e-2, [(1, 1, math.sqrt(2.0) / 2), (0, 2, 0.5), (2, -2, math.sqrt(2.0) / 8)]),
    ("exp_sq", math.log(2.0), 1.0, [(1, 1, math.sqrt(2.0) / 2), (0, 2, 0.5)]),
]


@pytest.mark.parametrize("kernel,kp,nu,cases", EXACT, ids=[f"{e[0]}:{e[1]:.3g}:nu{e[2]:g}" for e in EXACT])
def test_multiplier_exact_values(orc, kernel, kp, nu, cases):
    P = problem(orc, kernel, kp, nu)
    for kx, ky, m in cases:
        got = mode_multiplier(orc, P, kx, ky)
        assert abs(got - m) <= 4e-15 * m, (kernel, kp, kx, ky, got, m)


def test_table_kernel_exact_values(orc):
    """W from a table [q][p] laid out as the half spectrum."""
    n = N
    KX, KY = synthetic.wavenumbers(n)
    table = 4.0 ** (-np.abs(KX)) * 9.0 ** (-np.abs(KY))
    P = problem(orc, "table", 0.0, table=table)
    for kx, ky, m in [(1, 0, 0.5), (0, 1, 1 / 3), (3, 4, 5 / 648), (4, -3, 5 / 432), (2, 5, math.sqrt(29) / (4 * 243))]:
        got = mode_multiplier(orc, P, kx, ky)
        assert abs(got - m) <= 4e-15 * m, (kx, ky, got, m)


@pytest.mark.parametrize("a,b", [(0.1, 0.3), (0.3, 0.7), (0.5, 0.5)])
def test_exponential_semigroup(orc, a, b):
    """exp(-a|k|) exp(-b|k|) = exp(-(a+b)|k|): m_a m_b = |k| m_{a+b} on R."""
    k, _, _ = lattice_k(N)
    R = synthetic.retained_mask(N) & (k > 0)
    ma = all_multipliers(orc, problem(orc, "exp_abs", a)).real
    mb = all_multipliers(orc, problem(orc, "exp_abs", b)).real
    mab = all_multipliers(orc, problem(orc, "exp_abs", a + b)).real
    assert np.allclose(ma[R] * mb[R], k[R] * mab[R], rtol=1e-14, atol=0)


@pytest.mark.parametrize("alpha", [0.0, 0.5, 1.5, -1.0])
def test_fractional_powers_are_reciprocal(orc, alpha):
    """|k|^{1-alpha} |k|^{1-(2-alpha)} = 1 on every retained mode but k = 0."""
    k, _, _ = lattice_k(N)
    R = synthetic.retained_mask(N) & (k > 0)
    m1 = all_multipliers(orc, problem(orc, "frac", alpha)).real
    m2 = all_multipliers(orc, problem(orc, "frac", 2.0 - alpha)).real
    assert np.allclose(m1[R] * m2[R], 1.0, rtol=1e-14, atol=0)


def test_heat_kernel_depends_on_nu_beta_only(orc):
    """G_e = exp(-nu beta k^2): (nu, beta) and (2 nu, beta/2) give the same W,
    (nu, beta) and (nu, 2 beta) do not, and the semigroup holds in beta."""
    k, _, _ = lattice_k(N)
    R = synthetic.retained_mask(N) & (k > 0)
    m1 = all_multipliers(orc, problem(orc, "exp_sq", 0.7, nu=1e-2)).real
    m2 = all_multipliers(orc, problem(orc, "exp_sq", 0.35, nu=2e-2)).real
    m3 = all_multipliers(orc, problem(orc, "exp_sq", 1.4, nu=1e-2)).real
    assert np.allclose(m1[R], m2[R], rtol=1e-14, atol=0)
    assert np.allclose(m1[R] * m1[R], k[R] * m3[R], rtol=1e-14, atol=0)
    assert not np.allclose(m1[R], m3[R], rtol=1e-6)


@pytest.mark.parametrize("kernel,kp", [("identity", 0.0), ("exp_abs", 1.0), ("frac", -0.5), ("exp_sq", 0.7)])
def test_multiplier_vanishes_at_mean_and_outside_retained_set(orc, kernel, kp):
    n = 32
    P = problem(orc, kernel, kp, n=n)
    s = synthetic.random_field(n, 9) + 3.0  # non-zero mean
    w0 = orc.omega_from_control(P, s)
    assert w0[0, 0] == 0
    assert np.all(w0[~synthetic.retained_mask(n)] == 0)
    k, _, _ = lattice_k(n)
    R = synthetic.retained_mask(n) & (k > 0)
    assert np.all(np.abs(w0[R]) > 0)
