"""Behaviour of the C ABI on a GPU beyond parity: error statuses, launch
accounting, kernel timing, determinism."""
import numpy as np
import pytest

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


def small(api, **kw):
    base = dict(n=32, nsteps=8, dt=5e-3, nu=1e-3, px=8, every=4, kernels=[api.KernelSpec("exp_abs", 0.5)])
    base.update(kw)
    return api.Config(**base)


def test_cost_grad_needs_observations(api):
    from paper_2602_14016_gb300._native import DAError, DA_EINVAL

    ctx = api.Context(small(api))
    with pytest.raises(DAError) as e:
        ctx.cost_grad(torch.zeros(1, 32, 32, dtype=torch.float64, device="cuda"))
    assert e.value.status == DA_EINVAL


def test_forward_only_context_rejects_adjoint(api):
    from paper_2602_14016_gb300._native import DAError, DA_EINVAL

    ctx = api.Context(small(api, store=False))
    ctx.set_observations(torch.zeros(1, ctx.nt, 64, 2, dtype=torch.float64, device="cuda"))
    with pytest.raises(DAError) as e:
        ctx.cost_grad(torch.zeros(1, 32, 32, dtype=torch.float64, device="cuda"))
    assert e.value.status == DA_EINVAL
    wT, obs = ctx.forward(torch.zeros(1, 32, 32, dtype=torch.float64, device="cuda"))
    assert torch.all(wT == 0) and torch.all(obs == 0)


def test_launch_accounting_and_kernel_timing(api):
    cfg = small(api)
    ctx = api.Context(cfg)
    s = ctx.control_from_omega(torch.from_numpy(synthetic.random_vorticity_hat(32, 1)[None]).cuda())
    _, m = ctx.forward(s)
    ctx.set_observations(m + 0.1)
    l0 = ctx.launches
    ctx.time_kernels("adj_rows")
    J, g = ctx.cost_grad(s)
    ms, cnt = ctx.kernel_time()
    # forward: 2 + 8 per step + final observation; residual + init; adjoint 8 per step; gradient 2
    assert ctx.launches - l0 == 2 + 8 * cfg.nsteps + 1 + 2 + 8 * cfg.nsteps + 2
    assert cnt == 4 * cfg.nsteps and ms > 0
    assert abs(J.item() - 0.5 * 0.01 * m.numel()) < 1e-9 * J.item()
    ctx.time_kernels("off")


def test_bitwise_deterministic(api):
    ctx = api.Context(small(api, kernels=[api.KernelSpec("frac", 0.5), api.KernelSpec("identity", 0.0)]))
    w = np.stack([synthetic.random_vorticity_hat(32, 3), synthetic.random_vorticity_hat(32, 4)])
    s = ctx.control_from_omega(torch.from_numpy(w).cuda())
    _, m = ctx.forward(s)
    ctx.set_observations(m * 1.01)
    J1, g1 = ctx.cost_grad(s * 0.9)
    J2, g2 = ctx.cost_grad(s * 0.9)
    assert torch.equal(J1, J2) and torch.equal(g1, g2)


@pytest.mark.parametrize("ckpt", [0, 3])
def test_graph_replay_equals_direct_launches(api, ckpt):
    cfg = small(api, kernels=[api.KernelSpec("frac", 0.5), api.KernelSpec("exp_abs", 0.3)], ckpt_every=ckpt)
    direct, graph = api.Context(cfg), api.Context(cfg)
    graph.set_graphs(True)
    w = np.stack([synthetic.random_vorticity_hat(32, 7), synthetic.random_vorticity_hat(32, 8)])
    s = direct.control_from_omega(torch.from_numpy(w).cuda())
    _, m = direct.forward(s)
    for c in (direct, graph):
        c.set_observations(m * 1.02)
    for scale in (0.9, 1.1, 0.95):  # several replays with different controls
        J1, g1 = direct.cost_grad(s * scale)
        J2, g2 = graph.cost_grad(s * scale)
        assert torch.equal(J1, J2) and torch.equal(g1, g2)
    s1, s2 = (s * 0.9).contiguous(), (s * 0.9).contiguous()
    H1, i1, _, _ = direct.assimilate(s1, 3)
    H2, i2, _, _ = graph.assimilate(s2, 3)
    assert np.array_equal(H1, H2) and np.array_equal(i1, i2) and torch.equal(s1, s2)


def test_trajectory_larger_than_device_memory_gives_enomem(api):
    """A window whose stage-field store (64 n^2 bytes per step) is twice the
    device's memory: da_create returns DA_ENOMEM with a message, frees what it
    had allocated, and the process carries on."""
    from paper_2602_14016_gb300._native import DAError, DA_ENOMEM

    free0, total = torch.cuda.mem_get_info()
    n = 1024
    nsteps = int(2 * total // (64 * n * n)) // 10 * 10
    cfg = api.Config(n=n, nsteps=nsteps, dt=1e-4, nu=1e-3, px=32, every=nsteps,
                     kernels=[api.KernelSpec("exp_abs", 0.5)])
    with pytest.raises(DAError) as e:
        api.Context(cfg)
    assert e.value.status == DA_ENOMEM and "cudaMalloc" in str(e.value)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0 - (64 << 20)  # nothing of the failed context stays allocated
    ctx = api.Context(small(api))
    ctx.set_observations(torch.zeros((1, ctx.nt, 64, 2), dtype=torch.float64, device="cuda"))
    J, g = ctx.cost_grad(torch.from_numpy(synthetic.random_field(32, 3)[None]).cuda())
    assert torch.isfinite(J).all() and torch.isfinite(g).all()
