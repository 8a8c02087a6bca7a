"""The headline workload at its full size (256^2, 2000 RK4 steps, 16x16
probes every 20 steps, the seven-kernel sweep as one batch, CUDA-graph
replay as bench.py runs it), checked through properties that hold at any
size and on samples the oracle can compute; plus the largest grid."""
import numpy as np
import pytest

from cases import make_pair
from conftest import rel
from paper_2602_14016_gb300 import synthetic

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SWEEP = [("frac", 0.0), ("frac", 0.5), ("frac", 1.0), ("frac", 1.5), ("exp_abs", 0.1), ("exp_abs", 0.3),
         ("exp_abs", 1.0)]
N, STEPS, DT, NU = 256, 2000, 2e-3, 1e-2


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a GPU")
    from paper_2602_14016_gb300 import api as A, build

    build.build()
    return A


def config(api, kernels, nsteps=STEPS, ckpt=0):
    return api.Config(n=N, nsteps=nsteps, dt=DT, nu=NU, forcing="kolmogorov", nf=4, px=16, every=20,
                      kernels=[api.KernelSpec(*k) for k in kernels], ckpt_every=ckpt)


@pytest.fixture(scope="module")
def workload(api):
    """Truth (a spun-up Kolmogorov state), noisy observations, first guesses."""
    from paper_2602_14016_gb300 import workloads

    w = workloads.spin_up(api, torch, N, DT, NU, 5000, seed=0, forcing="kolmogorov", nf=4)
    one = api.Context(api.Config(n=N, nsteps=STEPS, dt=DT, nu=NU, forcing="kolmogorov", nf=4, px=16, every=20,
                                 store=False))
    _, obs = one.forward(one.control_from_omega(w))
    obs = obs.cpu().numpy()
    m = obs + 0.01 * np.sqrt(np.mean(obs**2)) * synthetic.gaussian_draws(obs.shape, 1)
    guess = workloads.first_guess_from_probes(w.cpu().numpy()[0], N, 16)
    one.close()
    return np.repeat(m, len(SWEEP), 0), np.repeat(guess[None], len(SWEEP), 0)


def test_batched_members_equal_single_member_runs(api, workload):
    m, guess = workload
    ctx = api.Context(config(api, SWEEP))
    ctx.set_graphs(True)
    ctx.set_observations(torch.from_numpy(m).cuda())
    s = ctx.control_from_omega(torch.from_numpy(guess).cuda())
    J, g = ctx.cost_grad(s)
    assert torch.all(torch.isfinite(J)) and torch.all(torch.isfinite(g))
    for b in (0, 3, 6):
        one = api.Context(config(api, [SWEEP[b]]))
        one.set_observations(torch.from_numpy(m[b:b + 1]).cuda())
        J1, g1 = one.cost_grad(s[b:b + 1].contiguous())
        assert torch.equal(J1[0], J[b]) and torch.equal(g1[0], g[b])
        one.close()


def test_full_window_gradient_against_central_differences(api, workload):
    """Central differences of J along a seeded unit direction per member.
    Over a chaotic 2000-step window their error is truncation (eps^2 times
    large higher derivatives) at large eps and amplified rounding at small
    eps, about 1e-8..3e-6 relative at the best eps for these members (the
    smallest |g.d|, under exp(-|k|), is the noisiest).  A missing or
    mis-signed term of the adjoint gives errors of order one, so the bound is
    1e-5 at the best of three step sizes, and 1e-6 for the median member."""
    m, guess = workload
    ctx = api.Context(config(api, SWEEP))
    ctx.set_graphs(True)
    ctx.set_observations(torch.from_numpy(m).cuda())
    s = ctx.control_from_omega(torch.from_numpy(guess).cuda())
    J, g = ctx.cost_grad(s)
    d = torch.from_numpy(np.stack([synthetic.random_field(N, 700 + b) for b in range(len(SWEEP))])).cuda()
    d = d / torch.linalg.norm(d.reshape(len(SWEEP), -1), dim=1)[:, None, None]
    gd = (g * d).sum(dim=(1, 2)).cpu().numpy()
    errs = []
    for eps in (1e-4, 3e-5, 1e-5):
        Jp, _ = ctx.cost_grad(s + eps * d)
        Jm, _ = ctx.cost_grad(s - eps * d)
        fd = (Jp - Jm).cpu().numpy() / (2 * eps)
        errs.append(np.abs(fd - gd) / np.abs(gd))
    best = np.min(errs, axis=0)
    assert np.all(best < 1e-5) and np.median(best) < 1e-6, (gd, errs)


def test_checkpointed_full_window_equals_full_storage(api, workload):
    m, guess = workload
    kern = SWEEP[:2]
    full = api.Context(config(api, kern))
    ck = api.Context(config(api, kern, ckpt=100))
    for c in (full, ck):
        c.set_graphs(True)
        c.set_observations(torch.from_numpy(m[:2]).cuda())
    s = full.control_from_omega(torch.from_numpy(guess[:2]).cuda())
    J0, g0 = full.cost_grad(s)
    J1, g1 = ck.cost_grad(s)
    assert torch.equal(J0, J1) and torch.equal(g0, g1)
    assert ck.device_bytes < full.device_bytes / 10


def test_first_steps_of_the_window_against_the_oracle(orc, api, workload):
    """The first 20 steps (one observation time) at the full grid size."""
    m, guess = workload
    nsteps = 20
    probs, cfg = make_pair(orc, N, nsteps, DT, NU, kernels=[SWEEP[1]], forcing="kolmogorov", nf=4, px=16,
                           every=20)
    P = probs[0]
    ctx = api.Context(cfg)
    ctx.set_graphs(True)
    s = ctx.control_from_omega(torch.from_numpy(guess[:1]).cuda()).cpu().numpy()
    mm = m[:1, :1].copy()
    J, g, _ = orc.cost_grad(P, s[0], mm[0])
    ctx.set_observations(torch.from_numpy(mm).cuda())
    Jg, gg = ctx.cost_grad(torch.from_numpy(s).cuda())
    assert abs(Jg.item() - J) <= 1e-12 * J
    assert rel(gg.cpu().numpy()[0], g) < 1e-8


def test_largest_grid_cost_and_gradient_against_the_oracle(orc, api):
    n = 1024
    probs, cfg = make_pair(orc, n, 2, 5e-4, 1e-3, kernels=[("exp_abs", 0.2)], px=32, every=1)
    P = probs[0]
    ctx = api.Context(cfg)
    truth = orc.control_from_omega(P, synthetic.random_vorticity_hat(n, 41))
    guess = orc.control_from_omega(P, synthetic.random_vorticity_hat(n, 42))
    _, mm = orc.forward(P, truth)
    J, g, _ = orc.cost_grad(P, guess, mm)
    ctx.set_observations(torch.from_numpy(mm[None]).cuda())
    Jg, gg = ctx.cost_grad(torch.from_numpy(guess[None]).cuda())
    assert abs(Jg.item() - J) <= 1e-12 * J
    assert rel(gg.cpu().numpy()[0], g) < 1e-8
