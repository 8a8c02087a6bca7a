"""Checkpoint-and-recompute and the vector-Jacobian product.

The kernels are deterministic, so recomputing a segment from its checkpoint
reproduces the stored stage fields bit for bit: the checkpointed gradient
must equal the full-storage gradient exactly.  da_vjp is checked against
da_cost_grad (the case dobs = obs - m), against da_adjoint_terminal (the
case dwT only), for linearity, and against the oracle."""
import numpy as np
import pytest

from cases import make_pair, noisy_observations, truth_and_guess
from conftest import rel
from paper_2602_14016_gb300 import synthetic

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


def problem(orc, n=32, nsteps=20, kernels=(("exp_abs", 0.5), ("frac", 1.0)), **kw):
    probs, cfg = make_pair(orc, n, nsteps, 5e-3, 1e-3, kernels=list(kernels), px=8, every=5, **kw)
    ss, ms = [], []
    for b, P in enumerate(probs):
        truth, guess = truth_and_guess(orc, P, 60 + b, 70 + b, scale=2.0)
        _, m = orc.forward(P, truth)
        ss.append(guess)
        ms.append(noisy_observations(m, 80 + b))
    return probs, cfg, np.stack(ss), np.stack(ms)


@pytest.mark.parametrize("K", [1, 3, 7, 20, 50])
def test_checkpointed_gradient_equals_full_storage(orc, api, K):
    probs, cfg, s, m = problem(orc)
    full = api.Context(cfg)
    full.set_observations(cu(m))
    J0, g0 = full.cost_grad(cu(s))
    ck = api.Context(api.Config(**{**cfg.__dict__, "ckpt_every": K}))
    ck.set_observations(cu(m))
    J1, g1 = ck.cost_grad(cu(s))
    assert torch.equal(J0, J1)
    assert torch.equal(g0, g1)
    if K < cfg.nsteps:
        assert ck.device_bytes < full.device_bytes
    # and against the oracle
    for b, P in enumerate(probs):
        J, g, _ = orc.cost_grad(P, s[b], m[b])
        assert abs(J1[b].item() - J) <= 1e-12 * J
        assert rel(g1[b].cpu().numpy(), g) < 1e-8


def test_checkpointed_kolmogorov_uneven_segments(orc, api):
    probs, cfg, s, m = problem(orc, nsteps=25, kernels=(("frac", 0.5),), forcing="kolmogorov", nf=3)
    ck = api.Context(api.Config(**{**cfg.__dict__, "ckpt_every": 4}))
    ck.set_observations(cu(m))
    J1, g1 = ck.cost_grad(cu(s))
    J, g, _ = orc.cost_grad(probs[0], s[0], m[0])
    assert abs(J1[0].item() - J) <= 1e-12 * J
    assert rel(g1[0].cpu().numpy(), g) < 1e-8


@pytest.mark.parametrize("K", [0, 4])
def test_vjp_special_cases_and_linearity(orc, api, K):
    probs, cfg, s, m = problem(orc)
    ctx = api.Context(api.Config(**{**cfg.__dict__, "ckpt_every": K}))
    ctx.set_observations(cu(m))
    J, g_cg = ctx.cost_grad(cu(s))
    wT, obs = ctx.forward(cu(s))
    g_obs = ctx.vjp(dobs=obs - cu(m))
    assert torch.equal(g_obs, g_cg)
    lamT = cu(np.stack([synthetic.unit_norm_terminal_hat(cfg.n, 90 + b) for b in range(cfg.batch)]))
    ctx.forward(cu(s))
    g_T = ctx.vjp(dwT=lamT)
    g_term = ctx.adjoint_terminal(cu(s), lamT)
    assert torch.equal(g_T, g_term)
    ctx.forward(cu(s))
    g_both = ctx.vjp(dobs=obs - cu(m), dwT=lamT)
    assert float(torch.linalg.norm(g_both - g_obs - g_T) / torch.linalg.norm(g_both)) < 1e-13
    for b, P in enumerate(probs):
        _, g_ref = orc.adjoint_terminal(P, s[b], lamT[b].cpu().numpy())
        assert rel(g_T[b].cpu().numpy(), g_ref) < 1e-8


def test_vjp_needs_a_stored_forward(api, orc):
    from paper_2602_14016_gb300._native import DAError, DA_EINVAL

    probs, cfg, s, m = problem(orc)
    ctx = api.Context(cfg)
    with pytest.raises(DAError) as e:
        ctx.vjp(dobs=cu(np.zeros((cfg.batch, ctx.nt, 64, 2))))
    assert e.value.status == DA_EINVAL
