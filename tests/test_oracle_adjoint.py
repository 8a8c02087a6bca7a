"""Pins of the oracle's discrete adjoint and gradient (Eq. 11-12, 19).

Tangent models are pinned against central differences of the nonlinear
forward; transposes against the tangents by dot-product tests; the full
gradient against finite differences of the cost, including a brute-force
full finite-difference gradient on a tiny grid."""
import numpy as np
import pytest

from conftest import dot, phys, rel
from paper_2602_14016_gb300 import synthetic


def small(orc, n=16, **kw):
    base = dict(n=n, nsteps=6, dt=2e-2, nu=5e-3, px=4, every=2, kernel="exp_abs", kparam=0.3)
    base.update(kw)
    return orc.Problem(**base)


@pytest.mark.parametrize("forcing", ["none", "kolmogorov"])
def test_rhs_tangent_matches_central_difference(orc, forcing):
    P = small(orc, 32, forcing=forcing, nf=3)
    y = synthetic.random_vorticity_hat(32, 1) * 3
    d = synthetic.random_retained_hat(32, 2, 1e-1)
    # F is quadratic plus affine, so (F(y+d) - F(y-d))/2 = J_F(y) d exactly
    fd = (orc.rhs(P, y + d) - orc.rhs(P, y - d)) / 2
    assert rel(fd, orc.rhs_tlm(P, y, d)) < 1e-13


def test_rhs_transpose_dot_product(orc):
    n = 32
    P = small(orc, n)
    y = synthetic.random_vorticity_hat(n, 3) * 2
    d = synthetic.random_retained_hat(n, 4)
    mu = synthetic.random_retained_hat(n, 5)
    a = dot(orc.rhs_tlm(P, y, d), mu)
    b = dot(d, orc.rhs_adj(P, y, mu))
    assert abs(a - b) < 1e-13 * max(abs(a), 1e-300) * 10


def test_step_tangent_and_transpose(orc):
    n = 16
    P = small(orc, n)
    w = synthetic.random_vorticity_hat(n, 6) * 3
    d = synthetic.random_retained_hat(n, 7)
    w2, dw = orc.step_tlm(P, w, d)
    assert rel(w2, orc.step(P, w)) == 0.0
    errs = []
    for eps in (1e-1, 1e-2, 1e-3):
        fd = (orc.step(P, w + eps * d) - orc.step(P, w - eps * d)) / (2 * eps)
        errs.append(rel(fd, dw))
    # the central difference converges at second order towards the tangent
    assert errs[1] < errs[0] / 50 and errs[2] < errs[1] / 50 and errs[2] < 1e-9, errs
    lam = synthetic.random_retained_hat(n, 8)
    a = dot(dw, lam)
    b = dot(d, orc.step_adj(P, w, lam))
    assert abs(a - b) < 1e-12 * abs(a)


def test_observation_transpose(orc):
    n = 16
    P = small(orc, n, px=8)
    d = synthetic.random_retained_hat(n, 9)
    r = synthetic.gaussian_draws((64, 2), 10)
    a = float(np.sum(orc.observe(P, d) * r))
    b = dot(d, orc.observe_adj(P, r))
    assert abs(a - b) < 1e-13 * abs(a)


@pytest.mark.parametrize("kernel,kp", [("identity", 0.0), ("exp_abs", 0.5), ("frac", 0.5), ("frac", -0.5), ("exp_sq", 0.7)])
def test_control_and_gradient_map_are_transposes(orc, kernel, kp):
    n = 16
    P = small(orc, n, kernel=kernel, kparam=kp)
    s = synthetic.random_field(n, 11)
    lam = synthetic.random_retained_hat(n, 12)
    a = dot(orc.omega_from_control(P, s), lam)
    b = float(np.sum(s * orc.gradient_map(P, lam)))
    assert abs(a - b) < 1e-13 * max(abs(a), 1.0)


def test_vorticity_control_identity(orc):
    """W = |k|^-2 (fractional kernel with exponent 1) makes s the vorticity
    itself: the control-variable equivalence of Sec. III.A and App. B."""
    n = 16
    P = small(orc, n, kernel="frac", kparam=1.0)
    s = synthetic.random_field(n, 13)
    expect = np.where(synthetic.retained_mask(n), np.fft.rfft2(s), 0)
    expect[0, 0] = 0
    assert rel(orc.omega_from_control(P, s), expect) < 1e-14


def test_identity_kernel_is_velocity_isometry(orc):
    """W = 1: the Euclidean norm of s equals that of the initial velocity (u, v)."""
    n = 16
    P = small(orc, n, kernel="identity", px=n)
    h = synthetic.random_retained_hat(n, 14)
    h[0, 0] = 0
    s = phys(h)
    uv = orc.observe(P, orc.omega_from_control(P, s))
    assert abs(np.sum(uv**2) - np.sum(s**2)) < 1e-13 * np.sum(s**2)


def test_control_roundtrip(orc):
    n = 16
    P = small(orc, n, kernel="exp_abs", kparam=1.0)
    w0 = synthetic.random_vorticity_hat(n, 15)
    s = orc.control_from_omega(P, w0)
    assert rel(orc.omega_from_control(P, s), w0) < 1e-13


def test_window_dot_product_in_control_space(orc):
    """<L ds, a_T> = <ds, L* a_T> over the whole window, L = d w_T / d s."""
    n = 16
    P = small(orc, n, nsteps=8, kernel="exp_abs", kparam=0.5, forcing="kolmogorov", nf=2, nu=1e-2)
    s = orc.control_from_omega(P, synthetic.random_vorticity_hat(n, 16) * 2)
    ds = synthetic.random_field(n, 17)
    aT = synthetic.random_retained_hat(n, 18)
    a = dot(orc.forward_tlm(P, s, ds), aT)
    _, g = orc.adjoint_terminal(P, s, aT)
    b = float(np.sum(ds * g))
    assert abs(a - b) < 1e-12 * abs(a)


def _problem_with_data(orc, n, **kw):
    P = small(orc, n, **kw)
    truth = orc.control_from_omega(P, synthetic.random_vorticity_hat(n, 20) * 2)
    _, m = orc.forward(P, truth)
    guess = orc.control_from_omega(P, synthetic.random_vorticity_hat(n, 21) * 2)
    return P, guess, m


@pytest.mark.parametrize("kernel,kp", [("identity", 0.0), ("exp_abs", 0.5), ("frac", 0.5)])
def test_gradient_against_central_differences(orc, kernel, kp):
    n = 16
    P, s, m = _problem_with_data(orc, n, kernel=kernel, kparam=kp)
    J, g, _ = orc.cost_grad(P, s, m)
    assert J > 0
    for seed in range(3):
        d = synthetic.random_field(n, 30 + seed)
        gd = float(np.sum(g * d))
        errs = []
        for eps in (1e-2, 1e-3, 1e-4):
            fd = (orc.cost(P, s + eps * d, m) - orc.cost(P, s - eps * d, m)) / (2 * eps)
            errs.append(abs(fd - gd) / abs(gd))
        # second-order convergence of the central difference, then agreement
        assert errs[1] < errs[0] / 30 or errs[1] < 1e-9
        assert errs[2] < 1e-7, errs


def test_brute_force_full_gradient(orc):
    """Every component of grad_s J by central differences on an 8x8 grid."""
    n = 8
    P = orc.Problem(n=n, nsteps=10, dt=2e-2, nu=1e-2, px=4, every=5, include_t0=True, kernel="exp_abs", kparam=0.2)
    truth = orc.control_from_omega(P, synthetic.random_vorticity_hat(n, 40) * 2)
    _, m = orc.forward(P, truth)
    s = orc.control_from_omega(P, synthetic.random_vorticity_hat(n, 41) * 2)
    _, g, _ = orc.cost_grad(P, s, m)
    fd = np.zeros_like(g)
    eps = 1e-5
    for i in range(n):
        for j in range(n):
            e = np.zeros((n, n))
            e[i, j] = eps
            fd[i, j] = (orc.cost(P, s + e, m) - orc.cost(P, s - e, m)) / (2 * eps)
    assert rel(fd, g) < 1e-8


def test_linear_limit_closed_form(orc):
    """For a tiny field the advection is negligible: each mode decays by the
    RK4 factor R(-nu k^2 dt) per step, so lambda0 = sum_j R^{n_j} H^T r_j."""
    n = 16
    P = orc.Problem(n=n, nsteps=6, dt=5e-2, nu=2e-2, px=4, every=3, include_t0=True)
    s = synthetic.random_field(n, 50) * 1e-9
    m = synthetic.gaussian_draws((P.nt, 16, 2), 51)
    _, obs = orc.forward(P, s)
    r = obs - m
    _, _, lam0 = orc.cost_grad(P, s, m)
    KX, KY = synthetic.wavenumbers(n)
    z = -P.nu * (KX**2 + KY**2) * P.dt
    R = 1 + z + z**2 / 2 + z**3 / 6 + z**4 / 24
    expect = np.zeros_like(lam0)
    for j, step in enumerate([0, 3, 6]):
        expect += R**step * orc.observe_adj(P, r[j])
    assert rel(lam0, expect) < 1e-7


def test_sobolev_term_single_mode(orc):
    """Eq. (4) term for w0 = cos(ax + by): |grad u0|^2 = cos^2(ax + by), so
    lambda/2 sum_grid |grad u0|^2 = lambda n^2 / 4."""
    n = 16
    y, x = np.meshgrid(2 * np.pi * np.arange(n) / n, 2 * np.pi * np.arange(n) / n, indexing="ij")
    P = orc.Problem(n=n, nsteps=1, dt=1e-3, nu=0.0, px=4, every=1, sobolev=0.3)
    w0 = np.fft.rfft2(np.cos(3 * x - 2 * y))
    assert abs(orc.sobolev_term(P, w0) - 0.3 * n * n / 4) < 1e-12


def test_sobolev_term_is_enstrophy_of_initial_field(orc):
    """For a divergence-free periodic field sum |grad u|^2 = sum w^2 (grid sums)."""
    n = 32
    P = orc.Problem(n=n, nsteps=1, dt=1e-3, nu=0.0, px=4, every=1, sobolev=2.0)
    w0 = synthetic.random_vorticity_hat(n, 3)
    assert abs(orc.sobolev_term(P, w0) - np.sum(phys(w0) ** 2)) < 1e-12 * np.sum(phys(w0) ** 2)


def test_regularised_gradient_against_central_differences(orc):
    n = 16
    P = orc.Problem(n=n, nsteps=6, dt=2e-2, nu=5e-3, px=4, every=2, kernel="exp_abs", kparam=0.3, sobolev=1e-2)
    truth = orc.control_from_omega(P, synthetic.random_vorticity_hat(n, 20) * 2)
    _, m = orc.forward(P, truth)
    s = orc.control_from_omega(P, synthetic.random_vorticity_hat(n, 21) * 2)
    J, g, _ = orc.cost_grad(P, s, m)
    J0, g0, _ = orc.cost_grad(orc.Problem(**{**P.__dict__, "sobolev": 0.0}), s, m)
    assert J > J0
    for seed in range(3):
        d = synthetic.random_field(n, 130 + seed)
        eps = 1e-4
        fd = (orc.cost(P, s + eps * d, m) - orc.cost(P, s - eps * d, m)) / (2 * eps)
        assert abs(fd - np.sum(g * d)) < 1e-7 * abs(fd)
