"""FFT plan variants and the autotuner: every variant of every grid size
agrees with the oracle; the autotuner keeps the fastest variant it measured,
and later contexts of the same grid and batch start on it."""
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


PLAN_COUNTS = {16: 1, 32: 2, 64: 3, 128: 4, 256: 3, 512: 3, 1024: 3}
VARIANTS = [(n, v) for n in PLAN_COUNTS for v in range(PLAN_COUNTS[n])]


def test_plan_counts_match_the_library(api):
    from paper_2602_14016_gb300 import _native

    lib = _native.load()
    for n in (16, 32, 64, 128, 256, 512, 1024):
        assert lib.da_plan_count(n) == sum(1 for m, _ in VARIANTS if m == n)
    assert lib.da_plan_count(48) == 0 and lib.da_plan_count(2048) == 0


@pytest.mark.parametrize("n,v", VARIANTS, ids=[f"n{n}-v{v}" for n, v in VARIANTS])
def test_every_variant_matches_the_oracle(orc, api, n, v):
    """One forward step, and a short cost-and-gradient window, on variant v."""
    steps = 1 if n == 1024 else 4
    probs, cfg = make_pair(orc, n, steps, 2e-3, 1e-2, kernels=[("exp_abs", 0.4)], forcing="kolmogorov",
                           nf=min(4, (n - 1) // 3), px=8, every=steps)
    P = probs[0]
    ctx = api.Context(cfg)
    ctx.set_plan(v)
    assert ctx.plan == v
    truth, guess = truth_and_guess(orc, P, 61, 62, scale=2.0)
    _, m = orc.forward(P, truth)
    m = noisy_observations(m, 63)
    J, g, _ = orc.cost_grad(P, guess, m)
    ctx.set_observations(cu(m[None]))
    Jg, gg = ctx.cost_grad(cu(guess[None]))
    assert abs(Jg.item() - J) <= 1e-12 * J
    assert rel(gg.cpu().numpy()[0], g) < 1e-8
    wT, _ = ctx.forward(cu(guess[None]))
    assert rel(wT.cpu().numpy()[0], orc.forward(P, guess)[0]) < 1e-12 * max(1, steps)


def test_set_plan_rejects_out_of_range(api):
    cfg = api.Config(n=64, nsteps=4, dt=1e-2, nu=1e-2, px=8, every=4)
    ctx = api.Context(cfg)
    with pytest.raises(Exception):
        ctx.set_plan(PLAN_COUNTS[64])
    with pytest.raises(Exception):
        ctx.set_plan(-1)


def test_autotune_keeps_the_fastest_and_later_contexts_reuse_it(api):
    cfg = api.Config(n=128, nsteps=10, dt=4e-3, nu=1e-3, px=8, every=5,
                     kernels=[api.KernelSpec("frac", 0.5)] * 3)
    ctx = api.Context(cfg)

    def control(seed):
        w = torch.from_numpy(np.stack([synthetic.random_vorticity_hat(128, seed + b) for b in range(3)])).cuda()
        return ctx.control_from_omega(w)

    _, m = ctx.forward(control(70))
    ctx.set_observations(m)
    s = control(80)
    J0, g0 = ctx.cost_grad(s)  # still in flight when the tuner starts: it must wait for it
    chosen, ms = ctx.autotune(steps=4)
    assert len(ms) == PLAN_COUNTS[128] and all(t > 0 for t in ms)
    assert chosen == int(np.argmin(ms)) and ctx.plan == chosen
    # observations survive the tuning; the evaluation is the same up to rounding
    J1, g1 = ctx.cost_grad(s)
    assert torch.all(J0 > 1e-3)
    assert torch.allclose(J1, J0, rtol=1e-12, atol=0) and rel(g1.cpu().numpy(), g0.cpu().numpy()) < 1e-10
    later = api.Context(cfg)
    assert later.plan == chosen
    other = api.Context(api.Config(n=128, nsteps=10, dt=4e-3, nu=1e-3, px=8, every=5))  # batch 1: not tuned
    assert other.plan == 0
