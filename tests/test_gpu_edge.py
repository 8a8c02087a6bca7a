"""Degenerate and edge cases of the CUDA path: states and data that are zero,
the laminar Kolmogorov flow whose discrete RK4 trajectory has a closed form,
the shortest windows, a probe at every grid point, and checkpoints of one
step."""
from fractions import Fraction

import numpy as np
import pytest

from cases import make_pair, noisy_observations, truth_and_guess
from conftest import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a GPU")
    from paper_2602_14016_gb300 import api as A, build

    build.build()
    return A


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_zero_state_and_zero_data_give_zero_cost_and_gradient(api):
    """Without forcing, w = 0 stays 0 (every product vanishes), so with zero
    data the residuals, the cost and the gradient are exactly zero."""
    cfg = api.Config(n=64, nsteps=20, dt=5e-3, nu=1e-3, px=8, every=5,
                     kernels=[api.KernelSpec("frac", 0.5), api.KernelSpec("exp_abs", 1.0)])
    ctx = api.Context(cfg)
    ctx.set_observations(torch.zeros((2, cfg.nt, 64, 2), dtype=torch.float64, device="cuda"))
    J, g = ctx.cost_grad(torch.zeros((2, 64, 64), dtype=torch.float64, device="cuda"))
    assert torch.count_nonzero(J) == 0 and torch.count_nonzero(g) == 0


@pytest.mark.parametrize("n,steps,dt,nu,amp,nf", [(64, 50, 1e-2, 0.05, 1.0, 4), (256, 40, 2e-3, 1e-2, 0.7, 4),
                                                  (128, 30, 4e-3, 2e-2, 1.3, 1)])
def test_laminar_kolmogorov_flow_from_rest_matches_the_rk4_closed_form(api, n, steps, dt, nu, amp, nf):
    """From rest, the forced flow is u = U(t) sin(nf y), w = -U nf cos(nf y):
    its advection term vanishes and U' = amp - nu nf^2 U.  Classical RK4 on
    this linear equation gives exactly U_k = U* (1 - R(z)^k) with
    U* = amp/(nu nf^2), z = -nu nf^2 dt, R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24
    (Eq. (24) forcing; the RK4 stability polynomial)."""
    every = steps // 5
    cfg = api.Config(n=n, nsteps=steps, dt=dt, nu=nu, forcing="kolmogorov", amp=amp, nf=nf, px=8, every=every,
                     store=False)
    ctx = api.Context(cfg)
    wT, obs = ctx.forward(torch.zeros((1, n, n), dtype=torch.float64, device="cuda"))
    # evaluated in exact rational arithmetic: 1 - R^k cancels (R^k is near 1),
    # so double precision would leave the reference itself at ~1e-12
    z = -Fraction(nu) * nf * nf * Fraction(dt)
    R = 1 + z + z * z / 2 + z**3 / 6 + z**4 / 24
    Ustar_q = Fraction(amp) / (Fraction(nu) * nf * nf)
    Ustar = float(Ustar_q)

    def U(k):
        return float(Ustar_q * (1 - R**k))

    w = wT.cpu().numpy()[0]
    ref = -U(steps) * nf * n * n / 2  # DFT of -U nf cos(nf y) at (kx, ky) = (0, +-nf)
    assert abs(w[nf, 0] - ref) <= 1e-13 * abs(ref)
    assert abs(w[n - nf, 0] - ref) <= 1e-13 * abs(ref)
    w[nf, 0] = w[n - nf, 0] = 0
    assert np.abs(w).max() <= 1e-13 * abs(ref)
    # probes on the px x px lattice: u = U_k sin(nf y), v = 0
    o = obs.cpu().numpy()[0]
    st = n // 8
    y = (np.arange(8) * st * 2 * np.pi / n).repeat(8)
    for t in range(cfg.nt):
        k = (t + 1) * every
        assert np.allclose(o[t, :, 0], U(k) * np.sin(nf * y), rtol=0, atol=1e-13 * Ustar)
        assert np.abs(o[t, :, 1]).max() <= 1e-13 * Ustar


@pytest.mark.parametrize("ckpt", [0, 1])
def test_single_step_window_observed_at_its_end(orc, api, ckpt):
    probs, cfg = make_pair(orc, 32, 1, 1e-2, 1e-2, kernels=[("exp_abs", 0.5)], px=4, every=1)
    cfg.ckpt_every = ckpt
    P = probs[0]
    truth, guess = truth_and_guess(orc, P, 21, 22)
    _, m = orc.forward(P, truth)
    J, g, _ = orc.cost_grad(P, guess, m)
    ctx = api.Context(cfg)
    ctx.set_observations(cu(m[None]))
    Jg, gg = ctx.cost_grad(cu(guess[None]))
    assert abs(Jg.item() - J) <= 1e-12 * J
    assert rel(gg.cpu().numpy()[0], g) < 1e-8


def test_every_grid_point_observed_with_one_step_checkpoints(orc, api):
    """px = n (the observation operator is the whole velocity field) and a
    checkpoint every step, over an uneven number of steps."""
    probs, cfg = make_pair(orc, 32, 7, 1e-2, 5e-3, kernels=[("frac", 1.0)], forcing="kolmogorov", nf=2, px=32,
                           every=1, include_t0=True)
    cfg.ckpt_every = 1
    P = probs[0]
    truth, guess = truth_and_guess(orc, P, 23, 24, scale=2.0)
    _, m = orc.forward(P, truth)
    m = noisy_observations(m, 25)
    J, g, _ = orc.cost_grad(P, guess, m)
    ctx = api.Context(cfg)
    ctx.set_observations(cu(m[None]))
    Jg, gg = ctx.cost_grad(cu(guess[None]))
    assert abs(Jg.item() - J) <= 1e-12 * J
    assert rel(gg.cpu().numpy()[0], g) < 1e-8


def test_single_probe_observed_only_at_t0(orc, api):
    """One probe, one observation time (t = 0 only): the gradient is the
    control map's transpose of H^T r alone, with no adjoint integration."""
    probs, cfg = make_pair(orc, 16, 4, 1e-2, 1e-2, kernels=[("identity", 0.0)], px=1, every=4, include_t0=True)
    P = probs[0]
    truth, guess = truth_and_guess(orc, P, 26, 27)
    _, m = orc.forward(P, truth)
    obs_guess = orc.forward(P, guess)[1]
    m[1:] = obs_guess[1:]  # the last time contributes nothing
    J, g, _ = orc.cost_grad(P, guess, m)
    ctx = api.Context(cfg)
    ctx.set_observations(cu(m[None]))
    Jg, gg = ctx.cost_grad(cu(guess[None]))
    assert abs(Jg.item() - J) <= 1e-12 * J
    assert rel(gg.cpu().numpy()[0], g) < 1e-8


@pytest.mark.parametrize("n,kx,ky", [(64, 1, 2), (128, 3, -2), (256, 5, 0)])
def test_single_taylor_green_mode_decays_by_the_rk4_factor(api, n, kx, ky):
    """w = cos(kx x + ky y) is a steady Euler solution (u . grad w = 0, the
    advection term of a single |k| shell vanishes), so RK4 multiplies its
    coefficient by R(z) per step, z = -nu |k|^2 dt, and no other mode is
    excited.  In the divergence form the two products cancel only in
    (d_xx - d_yy)(u v) + d_xy (v^2 - u^2): this checks that cancellation."""
    steps, dt, nu = 60, 1e-2, 2e-2
    cfg = api.Config(n=n, nsteps=steps, dt=dt, nu=nu, px=8, every=steps, store=False)
    ctx = api.Context(cfg)
    w0 = np.zeros((n, n // 2 + 1), complex)
    if kx == 0:
        w0[ky % n, 0] = w0[-ky % n, 0] = n * n / 2
    else:
        w0[ky % n, kx] = n * n / 2
    s = ctx.control_from_omega(cu(w0[None]))
    wT, _ = ctx.forward(s)
    z = -Fraction(nu) * (kx * kx + ky * ky) * Fraction(dt)
    R = 1 + z + z * z / 2 + z**3 / 6 + z**4 / 24
    amp = float(Fraction(n * n, 2) * R**steps)
    w = wT.cpu().numpy()[0]
    assert abs(w[ky % n, kx] - amp) <= 1e-13 * amp
    w[ky % n, kx] = 0
    if kx == 0:
        assert abs(w[-ky % n, 0] - amp) <= 1e-13 * amp
        w[-ky % n, 0] = 0
    assert np.abs(w).max() <= 1e-13 * amp
