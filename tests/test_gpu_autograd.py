"""The differentiable window (autograd wrapper over da_forward / da_vjp):
gradients of torch losses agree with da_cost_grad, with central finite
differences and with the oracle, with and without checkpointing."""
import numpy as np
import pytest

from cases import make_pair, noisy_observations, truth_and_guess
from conftest import rel
from paper_2602_14016_gb300 import synthetic

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a GPU")
    from paper_2602_14016_gb300 import api, autograd, build

    build.build()
    return api, autograd


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def setup(orc, n=32, nsteps=16, ckpt=0, forcing="kolmogorov"):
    probs, cfg = make_pair(orc, n, nsteps, 5e-3, 1e-2, kernels=[("frac", 0.5)], px=8, every=4, forcing=forcing, nf=3)
    cfg.ckpt_every = ckpt
    P = probs[0]
    truth, guess = truth_and_guess(orc, P, 110, 111, scale=2.0)
    _, m = orc.forward(P, truth)
    return P, cfg, guess, noisy_observations(m, 112)


@pytest.mark.parametrize("ckpt", [0, 5])
def test_misfit_gradient_equals_cost_grad(orc, mods, ckpt):
    api, ag = mods
    P, cfg, guess, m = setup(orc, ckpt=ckpt)
    ctx = api.Context(cfg)
    ctx.set_observations(cu(m[None]))
    _, g_ref = ctx.cost_grad(cu(guess[None]))
    s = cu(guess[None]).requires_grad_(True)
    obs, wT = ag.solve(s, ctx)
    L = ag.misfit(obs, cu(m[None])).sum()
    L.backward()
    assert rel(s.grad.cpu().numpy(), g_ref.cpu().numpy()) < 1e-14


def test_final_state_loss_against_oracle_and_finite_differences(orc, mods):
    api, ag = mods
    P, cfg, guess, m = setup(orc)
    ctx = api.Context(cfg)
    n = cfg.n
    rng = np.random.default_rng(5)
    c = rng.standard_normal((n, n // 2 + 1)) + 1j * rng.standard_normal((n, n // 2 + 1))
    c_t = cu(c[None])

    def loss(obs, wT):
        return ag.misfit(obs, cu(m[None])).sum() + 1e-3 * torch.sum(torch.real(c_t * wT))

    s = cu(guess[None]).requires_grad_(True)
    obs, wT = ag.solve(s, ctx)
    loss(obs, wT).backward()
    g = s.grad.cpu().numpy()[0]

    def oracle_loss(x):
        wT_o, obs_o = orc.forward(P, x)
        r = obs_o - m
        return 0.5 * np.sum(r * r) + 1e-3 * np.sum(np.real(c * wT_o))

    for seed in range(3):
        d = synthetic.random_field(n, 120 + seed)
        eps = 1e-4
        fd = (oracle_loss(guess + eps * d) - oracle_loss(guess - eps * d)) / (2 * eps)
        gd = float(np.sum(g * d))
        assert abs(fd - gd) < 1e-7 * abs(gd), (fd, gd)


def test_hbm_use_shrinks_with_checkpoints(orc, mods):
    api, _ = mods
    _, cfg, _, _ = setup(orc, nsteps=64)
    full = api.Context(cfg)
    cfg.ckpt_every = 8
    ck = api.Context(cfg)
    assert ck.device_bytes < full.device_bytes / 4


def test_kolmogorov_copy_at_64_against_oracle(orc, mods):
    """A 64^2 copy of the differentiable Kolmogorov window (checkpoints every
    8 steps): the autograd gradient of the misfit equals the oracle's."""
    api, ag = mods
    probs, cfg = make_pair(orc, 64, 48, 1e-3 * 4, 1 / 200, kernels=[("frac", 0.5)], px=16, every=8,
                           forcing="kolmogorov", nf=4)
    cfg.ckpt_every = 8
    P = probs[0]
    truth, guess = truth_and_guess(orc, P, 130, 131, scale=2.0)
    _, m = orc.forward(P, truth)
    J, g, _ = orc.cost_grad(P, guess, m)
    ctx = api.Context(cfg)
    s = cu(guess[None]).requires_grad_(True)
    obs, _ = ag.solve(s, ctx)
    L = ag.misfit(obs, cu(m[None])).sum()
    L.backward()
    assert abs(L.item() - J) <= 1e-12 * J
    assert rel(s.grad.cpu().numpy()[0], g) < 1e-8
