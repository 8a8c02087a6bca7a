"""Pins of the oracle's forward model (vorticity form of Eq. 1 and Eq. 24)
against closed forms and invariants that the mathematics fixes."""
import numpy as np
import pytest

from conftest import dot, phys, rel
from paper_2602_14016_gb300 import synthetic


def grid(n):
    return np.meshgrid(2 * np.pi * np.arange(n) / n, 2 * np.pi * np.arange(n) / n, indexing="ij")  # (y, x)


def prob(orc, n, **kw):
    base = dict(n=n, nsteps=1, dt=1e-3, nu=0.0, px=n, every=1)
    base.update(kw)
    return orc.Problem(**base)


def test_biot_savart_single_mode(orc):
    """w = cos(a x + b y): psi = w/k^2, u = dpsi/dy, v = -dpsi/dx at every node."""
    n = 16
    y, x = grid(n)
    a, b = 2, -3
    w = np.cos(a * x + b * y)
    P = prob(orc, n)
    obs = orc.observe(P, np.fft.rfft2(w)).reshape(n, n, 2)
    k2 = a * a + b * b
    u = -b * np.sin(a * x + b * y) / k2
    v = a * np.sin(a * x + b * y) / k2
    assert np.abs(obs[..., 0] - u).max() < 1e-14
    assert np.abs(obs[..., 1] - v).max() < 1e-14
    # incompressibility of the sampled velocity (spectral divergence)
    du = np.fft.rfft2(obs[..., 0])
    dv = np.fft.rfft2(obs[..., 1])
    KX, KY = synthetic.wavenumbers(n)
    assert np.abs(1j * KX * du + 1j * KY * dv).max() < 1e-12


def test_nonlinear_term_closed_form(orc):
    """w = cos x + cos 2y: u.grad w = -1.5 sin x sin 2y, so F = 1.5 sin x sin 2y (nu = 0)."""
    n = 16
    y, x = grid(n)
    w = np.cos(x) + np.cos(2 * y)
    F = phys(orc.rhs(prob(orc, n), np.fft.rfft2(w)))
    assert np.abs(F - 1.5 * np.sin(x) * np.sin(2 * y)).max() < 1e-13


def test_single_shell_has_no_advection(orc):
    """A field on one shell |k| = 5 satisfies u.grad w = 0, so F = -nu k^2 w."""
    n = 32
    y, x = grid(n)
    w = np.cos(3 * x + 4 * y) + 0.7 * np.sin(5 * y) - 0.2 * np.cos(4 * x - 3 * y) + 0.5 * np.sin(5 * x)
    nu = 0.01
    F = phys(orc.rhs(prob(orc, n, nu=nu), np.fft.rfft2(w)))
    assert np.abs(F + nu * 25 * w).max() < 1e-13


def test_dealias_projection(orc):
    """The output of F lies in the retained set; a product that would alias is cut."""
    n = 16
    h = synthetic.random_retained_hat(n, 3)
    F = orc.rhs(prob(orc, n, nu=0.1), h)
    assert np.all(F[~synthetic.retained_mask(n)] == 0)


@pytest.mark.parametrize("seed", [0, 1])
def test_inviscid_conservation_of_energy_and_enstrophy(orc, seed):
    """nu = 0, no forcing: sum w F(w) = 0 and sum psi F(w) = 0 (Galerkin truncation)."""
    n = 32
    h = synthetic.random_vorticity_hat(n, seed)
    F = orc.rhs(prob(orc, n), h)
    KX, KY = synthetic.wavenumbers(n)
    k2 = (KX**2 + KY**2).astype(float)
    psi = np.where(k2 > 0, h / np.where(k2 > 0, k2, 1), 0)
    scale = np.sqrt(dot(F, F) * dot(h, h))
    assert abs(dot(h, F)) < 1e-13 * scale
    assert abs(dot(psi, F)) < 1e-13 * np.sqrt(dot(F, F) * dot(psi, psi))


def test_taylor_green_decay_is_rk4_amplification(orc):
    """w0 = cos x cos y: w_n = R(z)^n w0, z = -2 nu dt, R the RK4 polynomial."""
    n = 16
    y, x = grid(n)
    nu, dt, steps = 0.05, 0.01, 20
    P = prob(orc, n, nu=nu, dt=dt, nsteps=steps, px=n, every=steps)
    w0 = np.cos(x) * np.cos(y)
    w = np.fft.rfft2(w0)
    for _ in range(steps):
        w = orc.step(P, w)
    z = -2 * nu * dt
    R = 1 + z + z**2 / 2 + z**3 / 6 + z**4 / 24
    assert np.abs(phys(w) - R**steps * w0).max() < 1e-14
    # and the exact viscous decay to O(dt^4)
    assert abs(R**steps - np.exp(-2 * nu * dt * steps)) < 1e-11


def test_laminar_kolmogorov_fixed_point(orc):
    """w = -(A/(nu nf)) cos(nf y) is a steady state of Eq. (24): F = 0, step = identity."""
    n = 32
    y, x = grid(n)
    A, nf, nu = 1.0, 4, 0.05
    P = prob(orc, n, nu=nu, forcing="kolmogorov", amp=A, nf=nf, dt=0.01)
    w = np.fft.rfft2(-(A / (nu * nf)) * np.cos(nf * y))
    F = orc.rhs(P, w)
    assert np.abs(F).max() < 1e-12 * np.abs(w).max() * nu * nf * nf
    assert rel(orc.step(P, w), w) < 1e-15


def test_kolmogorov_forcing_sign(orc):
    """From rest the forcing alone gives dw/dt = curl f = -A nf cos(nf y)."""
    n = 16
    y, x = grid(n)
    P = prob(orc, n, nu=0.01, forcing="kolmogorov", amp=0.5, nf=3)
    F = phys(orc.rhs(P, np.zeros((n, n // 2 + 1), complex)))
    assert np.abs(F - (-0.5 * 3 * np.cos(3 * y))).max() < 1e-13


def test_inviscid_drift_scales_as_dt4(orc):
    """Energy and enstrophy drift of RK4 over a fixed time falls at least 2^4-fold
    when dt halves.  RK4 is fourth order; for a quadratic invariant of nearly
    rotational dynamics its leading drift is one order higher (|R(i t)|^2 =
    1 - t^6/72 + ...), so ratios between 16 and 32 are expected."""
    n = 32
    h = synthetic.random_vorticity_hat(n, 5)
    KX, KY = synthetic.wavenumbers(n)
    k2 = (KX**2 + KY**2).astype(float)

    def EZ(w):
        psi = np.where(k2 > 0, w / np.where(k2 > 0, k2, 1), 0)
        return 0.5 * dot(psi, w), 0.5 * dot(w, w)

    T = 0.4
    drifts = []
    for dt in (0.04, 0.02):
        P = prob(orc, n, dt=dt)
        w = h.copy()
        for _ in range(int(round(T / dt))):
            w = orc.step(P, w)
        (E0, Z0), (E1, Z1) = EZ(h), EZ(w)
        drifts.append((abs(E1 - E0) / E0, abs(Z1 - Z0) / Z0))
    rE = drifts[0][0] / drifts[1][0]
    rZ = drifts[0][1] / drifts[1][1]
    assert 12 < rE < 40 and 12 < rZ < 40, (drifts, rE, rZ)


def test_observations_and_cost_of_a_known_residual(orc):
    """J = 1/2 sum of squared offsets when m = model observations - offsets."""
    n = 16
    P = orc.Problem(n=n, nsteps=4, dt=1e-3, nu=1e-2, px=4, every=2, include_t0=True)
    s = synthetic.random_field(n, 1)
    _, obs = orc.forward(P, s)
    assert obs.shape == (3, 16, 2)
    off = synthetic.gaussian_draws(obs.shape, 2)
    J = orc.cost(P, s, obs - off)
    assert abs(J - 0.5 * np.sum(off**2)) < 1e-12 * J
    J2, g, _ = orc.cost_grad(P, s, obs - off)
    assert abs(J2 - J) < 1e-13 * J


def test_probe_lattice_positions(orc):
    """Probe r*px+q samples node (r n/px, q n/px) of the velocity field."""
    n, px = 16, 4
    P = prob(orc, n, px=px)
    h = synthetic.random_vorticity_hat(n, 9)
    full = orc.observe(prob(orc, n, px=n), h).reshape(n, n, 2)
    sub = orc.observe(P, h).reshape(px, px, 2)
    st = n // px
    assert np.array_equal(sub, full[::st, ::st])
