"""da_assimilate (L-BFGS on the control, Sec. II.C) against the oracle's
L-BFGS: the cost histories agree on the first iterations (beyond them line
search branching and chaos make iterates drift apart, so only monotone
decrease is checked), batch members follow their single runs, and a
non-finite cost is reported as DA_EDIVERGED."""
import numpy as np
import pytest

from cases import make_pair, noisy_observations, truth_and_guess
from oracle import lbfgs

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


def _setup(orc, kernels, n=32, nsteps=20, seed=0):
    probs, cfg = make_pair(orc, n, nsteps, 5e-3, 1e-3, kernels=kernels, px=8, every=5)
    data = []
    for b, P in enumerate(probs):
        truth, guess = truth_and_guess(orc, P, seed + 10 * b, seed + 10 * b + 1, scale=2.0)
        _, m = orc.forward(P, truth)
        data.append((guess, noisy_observations(m, seed + 10 * b + 2)))
    return probs, cfg, data


@pytest.mark.parametrize("kernel", [("exp_abs", 0.5), ("frac", 0.5), ("identity", 0.0)])
def test_cost_history_matches_oracle(orc, api, kernel):
    probs, cfg, data = _setup(orc, [kernel])
    P, (guess, m) = probs[0], data[0]
    iters = 6

    def fg(x):
        J, g, _ = orc.cost_grad(P, x.reshape(P.n, P.n), m)
        return J, g.ravel()

    ref = lbfgs.minimize(fg, guess.ravel(), iters)
    ref_hist = np.array(ref["J_hist"])
    ctx = api.Context(cfg)
    ctx.set_observations(cu(m[None]))
    s = cu(guess[None]).clone()
    J, it, st, ms = ctx.assimilate(s, iters)
    assert ms[0] in (0, 6) and st == ms[0]
    hist = J[0, : it[0] + 1]
    k = min(4, len(ref_hist), len(hist))
    assert np.all(np.abs(hist[:k] - ref_hist[:k]) <= 1e-6 * ref_hist[:k]), (hist[:k], ref_hist[:k])
    assert np.all(np.diff(hist) < 0)
    assert hist[-1] < 0.5 * hist[0]


def test_batch_members_follow_their_single_runs(orc, api):
    kernels = [("exp_abs", 0.5), ("frac", 1.0), ("identity", 0.0)]
    probs, cfg, data = _setup(orc, kernels, seed=3)
    iters = 4
    ctx = api.Context(cfg)
    ctx.set_observations(cu(np.stack([m for _, m in data])))
    s = cu(np.stack([g for g, _ in data])).clone()
    J, it, _, _ = ctx.assimilate(s, iters)
    for b, k in enumerate(kernels):
        one = api.Context(api.Config(**{**cfg.__dict__, "kernels": [api.KernelSpec(*k)]}))
        one.set_observations(cu(data[b][1][None]))
        s1 = cu(data[b][0][None]).clone()
        J1, it1, _, _ = one.assimilate(s1, iters)
        assert it1[0] == it[b]
        assert np.allclose(J1[0], J[b], rtol=1e-12, atol=0)
        assert torch.allclose(s1[0], s[b], rtol=1e-10, atol=1e-12 * float(s1.abs().max()))


def test_non_finite_cost_is_reported(orc, api):
    from paper_2602_14016_gb300._native import DAError, DA_EDIVERGED

    probs, cfg, data = _setup(orc, [("identity", 0.0)])
    ctx = api.Context(cfg)
    ctx.set_observations(cu(data[0][1][None]))
    s = cu(data[0][0][None]) * 1e200  # overflows to inf in the forward solve
    res = ctx.assimilate(s.contiguous(), 3)
    assert res.status == DA_EDIVERGED and res.member_status[0] == DA_EDIVERGED
    with pytest.raises(DAError) as e:
        ctx.assimilate(s.contiguous(), 3, raise_on_diverged=True)
    assert e.value.status == DA_EDIVERGED


def test_one_diverging_member_leaves_the_others_intact(orc, api):
    """Member 1 starts from an overflowing control; members 0 and 2 must
    return the same histories and controls as in a batch without it."""
    from paper_2602_14016_gb300._native import DA_EDIVERGED

    kernels = [("exp_abs", 0.5), ("frac", 1.0), ("identity", 0.0)]
    probs, cfg, data = _setup(orc, kernels, seed=5)
    iters = 3
    m = cu(np.stack([mm for _, mm in data]))
    s_good = cu(np.stack([g for g, _ in data]))
    s_bad = s_good.clone()
    s_bad[1] *= 1e200
    ref = api.Context(cfg)
    ref.set_observations(m)
    s_ref = s_good.clone()
    R = ref.assimilate(s_ref, iters)
    ctx = api.Context(cfg)
    ctx.set_observations(m)
    s = s_bad.clone()
    res = ctx.assimilate(s, iters)
    assert res.status == DA_EDIVERGED
    assert res.member_status[1] == DA_EDIVERGED
    for b in (0, 2):
        assert res.member_status[b] == R.member_status[b] and res.member_status[b] != DA_EDIVERGED
        assert res.iters[b] == R.iters[b]
        assert np.array_equal(res.J_hist[b], R.J_hist[b])
        assert torch.equal(s[b], s_ref[b])
