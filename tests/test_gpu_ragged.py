"""Ragged batches (da_set_member) and the stepwise optimiser (da_lbfgs_*).

Members of one grid size with their own horizons, probe lattices, viscosities
and forcing switches share every launch, end-aligned in each evaluation.
- each member's cost and gradient match the oracle's for its own window, and
  are bitwise those of a batch-1 context holding that window alone (same plan
  variant), with and without graph replay; an idle slot costs 0;
- a member started between rounds of the stepwise optimiser follows exactly
  the iterates of da_assimilate run on it alone.
"""
import numpy as np
import pytest

from cases import noisy_observations
from conftest import rel
from paper_2602_14016_gb300 import synthetic

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N, DT, NSTEPS, EVERY, PMAX = 32, 5e-3, 40, 5, 8
# (nsteps, px, nu, forcing, kernel) per member; nsteps 0: idle slot
WINDOWS = [(40, 8, 1e-3, False, ("exp_abs", 0.5)), (20, 4, 1e-2, True, ("frac", 1.0)), (0, 8, 1e-3, False, None),
           (35, 8, 5e-3, True, ("exp_sq", 0.7))]


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a GPU")
    from paper_2602_14016_gb300 import api as A, build

    build.build()
    return A


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def oracle_problem(orc, nsteps, px, nu, forcing, kernel):
    return orc.Problem(n=N, nsteps=nsteps, dt=DT, nu=nu, forcing="kolmogorov" if forcing else "none", amp=1.0, nf=4,
                       px=px, every=EVERY, kernel=kernel[0], kparam=kernel[1])


def member_data(orc, b, win):
    nsteps, px, nu, forcing, kernel = win
    P = oracle_problem(orc, nsteps, px, nu, forcing, kernel)
    truth = orc.control_from_omega(P, synthetic.random_vorticity_hat(N, 300 + b) * 2)
    guess = orc.control_from_omega(P, synthetic.random_vorticity_hat(N, 400 + b) * 2)
    _, m = orc.forward(P, truth)
    return P, guess, noisy_observations(m, 500 + b)


def ragged_context(api, graphs=False, ckpt=0):
    cfg = api.Config(n=N, nsteps=NSTEPS, dt=DT, nu=1e-3, forcing="kolmogorov", nf=4, px=PMAX, every=EVERY,
                     kernels=[api.KernelSpec("identity", 0.0)] * len(WINDOWS), ckpt_every=ckpt)
    ctx = api.Context(cfg)
    ctx.set_plan(0)
    if graphs:
        ctx.set_graphs(True)
    return ctx


def alone_context(api, win, m):
    nsteps, px, nu, forcing, kernel = win
    cfg = api.Config(n=N, nsteps=nsteps, dt=DT, nu=nu, forcing="kolmogorov" if forcing else "none", nf=4, px=px,
                     every=EVERY, kernels=[api.KernelSpec(*kernel)])
    ctx = api.Context(cfg)
    ctx.set_plan(0)
    ctx.set_observations(cu(m[None]))
    return ctx


@pytest.mark.parametrize("graphs,ckpt", [(False, 0), (True, 0), (False, 7), (True, 3)])
def test_ragged_members_match_the_oracle_and_their_alone_runs(orc, api, graphs, ckpt):
    """With checkpoints every 7 or 3 steps the segments cut through the
    members' windows (starts at steps 0, 5 and 20 of the 40-step evaluation)."""
    ctx = ragged_context(api, graphs, ckpt)
    data = {}
    s = np.zeros((len(WINDOWS), N, N))
    for b, win in enumerate(WINDOWS):
        if win[0] == 0:
            ctx.set_member(b, 0)
            continue
        P, guess, m = member_data(orc, b, win)
        data[b] = (P, guess, m)
        s[b] = guess
        ctx.set_member(b, win[0], win[1], win[2], win[3], api.KernelSpec(*win[4]), cu(m))
    for rep in range(2):  # the second evaluation replays the captured graph
        J, g = ctx.cost_grad(cu(s))
        J, g = J.cpu().numpy(), g.cpu().numpy()
        assert J[2] == 0.0 and not np.any(g[2])
        for b, (P, guess, m) in data.items():
            Jr, gr, _ = orc.cost_grad(P, guess, m)
            assert abs(J[b] - Jr) <= 1e-12 * Jr, (b, J[b], Jr)
            assert rel(g[b], gr) < 1e-8, b
            one = alone_context(api, WINDOWS[b], m)
            J1, g1 = one.cost_grad(cu(guess[None]))
            assert J1.item() == J[b] and np.array_equal(g1.cpu().numpy()[0], g[b]), b
            one.close()
    ctx.close()


def test_member_started_between_rounds_follows_its_alone_run(orc, api):
    """Members 0 and 3 start at once, member 1 after two rounds; each ends
    with the J history and control of da_assimilate on it alone."""
    iters = 4
    ctx = ragged_context(api)
    data = {}
    for b in (0, 1, 3):
        win = WINDOWS[b]
        P, guess, m = member_data(orc, b, win)
        data[b] = (guess, m)
        ctx.set_member(b, win[0], win[1], win[2], win[3], api.KernelSpec(*win[4]), cu(m))
    ctx.set_member(2, 0)
    ctx.lbfgs_start(0, cu(data[0][0]), iters)
    ctx.lbfgs_start(3, cu(data[3][0]), iters)
    for _ in range(2):
        ctx.lbfgs_iterate()
    ctx.lbfgs_start(1, cu(data[1][0]), iters)
    rounds = 0
    while ctx.lbfgs_iterate() > 0:
        rounds += 1
        assert rounds < 50
    for b in (0, 1, 3):
        rep, hist, s = ctx.lbfgs_member(b, iters + 1, control=True)
        assert rep["phase"] == 3
        one = alone_context(api, WINDOWS[b], data[b][1])
        s1 = cu(data[b][0][None]).clone()
        res = one.assimilate(s1, iters)
        assert rep["iters"] == res.iters[0] and rep["status"] == res.member_status[0], (b, rep)
        assert np.array_equal(hist, res.J_hist[0]), (b, hist, res.J_hist[0])
        assert torch.equal(s, s1[0]), b
        assert hist[-1] < hist[0]
        one.close()
    ctx.close()


def test_set_member_rejects_bad_windows(api):
    from paper_2602_14016_gb300._native import DAError

    ctx = ragged_context(api)
    m = torch.zeros((NSTEPS // EVERY, PMAX * PMAX, 2), dtype=torch.float64, device="cuda")
    for kw in (dict(nsteps=NSTEPS + EVERY), dict(nsteps=7), dict(px=16), dict(px=3), dict(nu=-1.0)):
        args = dict(nsteps=NSTEPS, px=PMAX, nu=1e-3)
        args.update(kw)
        with pytest.raises(DAError):
            ctx.set_member(0, args["nsteps"], args["px"], args["nu"], False, api.KernelSpec("identity", 0.0), m)
    with pytest.raises(DAError):  # exp(800 |k|) is not finite on the retained set
        ctx.set_member(0, NSTEPS, PMAX, 1e-3, False, api.KernelSpec("exp_abs", -800.0), m)
    ctx.close()
