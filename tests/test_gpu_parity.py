"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: 1e-12 relative per step and on the cost, 1e-8 relative L2 on
the gradient over the full window (the stated targets); most cases land
far below them."""
import numpy as np
import pytest

from cases import make_pair, noisy_observations, truth_and_guess
from conftest import rel
from paper_2602_14016_gb300 import synthetic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

STEP_TOL = 1e-12
COST_TOL = 1e-12
GRAD_TOL = 1e-8


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a GPU")
    from paper_2602_14016_gb300 import api as A, build

    build.build()
    return A


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def stack(arrs):
    return cu(np.stack(arrs))


KERNELS = [("identity", 0.0), ("exp_abs", 0.5), ("frac", 0.5), ("frac", 1.0), ("exp_sq", 0.7), ("frac", -0.5)]


@pytest.mark.parametrize("n", [16, 64, 256])
def test_control_map(orc, api, n):
    probs, cfg = make_pair(orc, n, 2, 1e-3, 1e-3, kernels=KERNELS, px=8 if n >= 16 else 4, every=1)
    ctx = api.Context(cfg)
    s = [synthetic.random_field(n, 10 + i) for i in range(len(KERNELS))]
    w = ctx.omega_from_control(stack(s)).cpu().numpy()
    for b, P in enumerate(probs):
        assert rel(w[b], orc.omega_from_control(P, s[b])) < 1e-13
    # right inverse on the retained set
    s2 = ctx.control_from_omega(cu(w)).cpu().numpy()
    for b, P in enumerate(probs):
        assert rel(s2[b], orc.control_from_omega(P, w[b])) < 1e-12


@pytest.mark.parametrize("n", [16, 32, 64, 128, 256, 512])
@pytest.mark.parametrize("forcing", ["none", "kolmogorov"])
def test_one_step(orc, api, n, forcing):
    probs, cfg = make_pair(orc, n, 1, 2e-3, 1e-2, forcing=forcing, nf=min(4, (n - 1) // 3), px=8, every=1)
    P = probs[0]
    ctx = api.Context(cfg)
    w0 = synthetic.random_vorticity_hat(n, 3) * 3
    s = orc.control_from_omega(P, w0)
    wT, obs = ctx.forward(cu(s[None]))
    ref = orc.step(P, orc.omega_from_control(P, s))
    assert rel(wT.cpu().numpy()[0], ref) < STEP_TOL
    _, robs = orc.forward(P, s)
    assert rel(obs.cpu().numpy()[0], robs) < STEP_TOL


def test_one_step_largest_grid(orc, api):
    n = 1024
    probs, cfg = make_pair(orc, n, 1, 5e-4, 1e-3, px=32, every=1)
    P = probs[0]
    ctx = api.Context(cfg)
    s = orc.control_from_omega(P, synthetic.random_vorticity_hat(n, 4) * 3)
    wT, _ = ctx.forward(cu(s[None]))
    assert rel(wT.cpu().numpy()[0], orc.step(P, orc.omega_from_control(P, s))) < STEP_TOL


@pytest.mark.parametrize("forcing", ["none", "kolmogorov"])
def test_forward_window(orc, api, forcing):
    n = 64
    probs, cfg = make_pair(orc, n, 40, 5e-3, 1e-3, forcing=forcing, px=8, every=10, include_t0=True)
    P = probs[0]
    ctx = api.Context(cfg)
    s, _ = truth_and_guess(orc, P, 0, 1)
    wT, obs = ctx.forward(cu(s[None]))
    rw, robs = orc.forward(P, s)
    assert rel(wT.cpu().numpy()[0], rw) < 1e-11
    assert rel(obs.cpu().numpy()[0], robs) < 1e-11


CG_CASES = [
    dict(n=32, nsteps=20, dt=5e-3, nu=1e-3, kernels=[("exp_abs", 0.5)], px=8, every=5),
    dict(n=32, nsteps=12, dt=1e-2, nu=1e-2, kernels=[("frac", 0.5)], forcing="kolmogorov", nf=4, px=4, every=4,
         include_t0=True),
    dict(n=64, nsteps=30, dt=5e-3, nu=1e-3, kernels=[("identity", 0.0)], px=8, every=10),
    dict(n=64, nsteps=16, dt=5e-3, nu=1e-3, kernels=[("exp_sq", 0.7)], px=64, every=16),
    dict(n=16, nsteps=6, dt=1e-2, nu=1e-2, kernels=[("frac", 1.0)], px=1, every=3, include_t0=True),
    dict(n=128, nsteps=8, dt=4e-3, nu=5e-4, kernels=[("exp_abs", 0.3)], px=16, every=4),
    dict(n=256, nsteps=4, dt=2e-3, nu=1e-2, kernels=[("frac", 1.5)], forcing="kolmogorov", nf=4, px=16, every=2),
]


@pytest.mark.parametrize("case", CG_CASES, ids=[f"n{c['n']}-{c['kernels'][0][0]}" for c in CG_CASES])
def test_cost_and_gradient(orc, api, case):
    case = dict(case)
    probs, cfg = make_pair(orc, **case)
    P = probs[0]
    ctx = api.Context(cfg)
    truth, guess = truth_and_guess(orc, P, 5, 6, scale=2.0)
    _, m = orc.forward(P, truth)
    m = noisy_observations(m, 7)
    J, g, lam0 = orc.cost_grad(P, guess, m)
    ctx.set_observations(cu(m[None]))
    Jg, gg = ctx.cost_grad(cu(guess[None]))
    assert abs(Jg.item() - J) <= COST_TOL * J
    assert rel(gg.cpu().numpy()[0], g) < GRAD_TOL
    l0, filt = ctx.last_adjoint()
    assert rel(l0.cpu().numpy()[0], lam0) < GRAD_TOL


def test_batch_members_match_single_runs(orc, api):
    n = 32
    kernels = [("identity", 0.0), ("exp_abs", 1.0), ("frac", 0.5), ("exp_sq", 0.3)]
    probs, cfg = make_pair(orc, n, 10, 5e-3, 1e-3, kernels=kernels, px=8, every=5)
    ctx = api.Context(cfg)
    ss, ms, refs = [], [], []
    for b, P in enumerate(probs):
        truth, guess = truth_and_guess(orc, P, 20 + b, 30 + b, scale=2.0)
        _, m = orc.forward(P, truth)
        ss.append(guess)
        ms.append(m)
        refs.append(orc.cost_grad(P, guess, m))
    ctx.set_observations(stack(ms))
    J, g = ctx.cost_grad(stack(ss))
    for b in range(len(kernels)):
        assert abs(J[b].item() - refs[b][0]) <= COST_TOL * refs[b][0]
        assert rel(g[b].cpu().numpy(), refs[b][1]) < GRAD_TOL


def test_adjoint_from_terminal_field(orc, api):
    n = 64
    probs, cfg = make_pair(orc, n, 20, 5e-3, 5e-4, kernels=[("exp_abs", 0.5)], px=8, every=10)
    P = probs[0]
    ctx = api.Context(cfg)
    s, _ = truth_and_guess(orc, P, 8, 9)
    lamT = synthetic.unit_norm_terminal_hat(n, 10)
    lam0, g = orc.adjoint_terminal(P, s, lamT)
    gg = ctx.adjoint_terminal(cu(s[None]), cu(lamT[None]))
    assert rel(gg.cpu().numpy()[0], g) < GRAD_TOL
    l0, _ = ctx.last_adjoint()
    assert rel(l0.cpu().numpy()[0], lam0) < GRAD_TOL


def test_filtered_gradient_output(orc, api):
    """G-metric gradient IDFT(|k| W lambda0_hat) (Eq. 17 in the scalar representation)."""
    n = 32
    probs, cfg = make_pair(orc, n, 6, 5e-3, 1e-3, kernels=[("exp_abs", 0.4)], px=8, every=3)
    P = probs[0]
    ctx = api.Context(cfg)
    truth, guess = truth_and_guess(orc, P, 11, 12)
    _, m = orc.forward(P, truth)
    ctx.set_observations(cu(m[None]))
    ctx.cost_grad(cu(guess[None]))
    lam0, filt = ctx.last_adjoint()
    lam0 = lam0.cpu().numpy()[0]
    KX, KY = synthetic.wavenumbers(n)
    k = np.sqrt(KX**2 + KY**2)
    W = np.exp(-0.4 * k)
    expect = np.fft.irfft2(np.where(synthetic.retained_mask(n), k * W * lam0, 0), s=(n, n))
    assert rel(filt.cpu().numpy()[0], expect) < 1e-12


def test_plain_config_window(orc, api):
    """The 64^2 decaying window: 200 RK4 steps of 5e-3, nu = 1e-3, 8x8 probes
    every 10 steps, W = exp(-0.5 |k|), unit-energy k^4 exp(-2 (k/4)^2) truth."""
    n = 64
    probs, cfg = make_pair(orc, n, 200, 5e-3, 1e-3, kernels=[("exp_abs", 0.5)], px=8, every=10)
    P = probs[0]
    ctx = api.Context(cfg)
    truth = orc.control_from_omega(P, synthetic.random_vorticity_hat(n, 0))
    guess = orc.control_from_omega(P, synthetic.random_vorticity_hat(n, 1))
    _, m = orc.forward(P, truth)
    J, g, _ = orc.cost_grad(P, guess, m)
    ctx.set_observations(cu(m[None]))
    Jg, gg = ctx.cost_grad(cu(guess[None]))
    assert abs(Jg.item() - J) <= COST_TOL * J
    assert rel(gg.cpu().numpy()[0], g) < GRAD_TOL


def test_gradient_against_gpu_finite_differences(api):
    """A property at any size: <grad, d> equals the central difference of J."""
    from paper_2602_14016_gb300.api import Config, KernelSpec

    n = 128
    cfg = Config(n=n, nsteps=40, dt=4e-3, nu=5e-4, px=16, every=10, kernels=[KernelSpec("exp_abs", 0.3)])
    ctx = api.Context(cfg)
    w_truth = cu(synthetic.random_vorticity_hat(n, 40)[None])
    w_guess = cu(synthetic.random_vorticity_hat(n, 41)[None])
    s_truth = ctx.control_from_omega(w_truth)
    s = ctx.control_from_omega(w_guess)
    _, m = ctx.forward(s_truth)
    ctx.set_observations(m)
    J, g = ctx.cost_grad(s)
    d = cu(synthetic.random_field(n, 42)[None])
    gd = float((g * d).sum())
    eps = 1e-3
    Jp, _ = ctx.cost_grad(s + eps * d)
    Jm, _ = ctx.cost_grad(s - eps * d)
    fd = (Jp.item() - Jm.item()) / (2 * eps)
    assert abs(fd - gd) < 1e-6 * abs(gd)


@pytest.mark.parametrize("ckpt", [0, 3])
def test_sobolev_regularised_cost_and_gradient(orc, api, ckpt):
    n = 32
    probs, cfg = make_pair(orc, n, 12, 5e-3, 1e-3, kernels=[("exp_abs", 0.5)], px=8, every=4)
    cfg.ckpt_every = ckpt
    P = probs[0]
    P.sobolev = 1e-2
    truth, guess = truth_and_guess(orc, P, 150, 151, scale=2.0)
    _, m = orc.forward(P, truth)
    J, g, _ = orc.cost_grad(P, guess, m)
    ctx = api.Context(cfg)
    ctx.set_sobolev(1e-2)
    ctx.set_observations(cu(m[None]))
    Jg, gg = ctx.cost_grad(cu(guess[None]))
    assert abs(Jg.item() - J) <= COST_TOL * J
    assert rel(gg.cpu().numpy()[0], g) < GRAD_TOL
