"""Serving with continuous batching: admission by memory and slots, latency
accounting (fake executor on the CPU), the memory model against the
library's own count, and on the GPU the equality of every job's result alone
and in the mix."""
import time

import numpy as np
import pytest

from paper_2602_14016_gb300 import serve


def job(i, arrival, n=32, nsteps=20, iters=3):
    return serve.Job(job_id=i, n=n, nsteps=nsteps, dt=5e-3, nu=1e-3, px=8, every=5, iters=iters, arrival=arrival)


def test_checkpoint_plan_respects_the_job_cap():
    j = job(0, 0.0, n=256, nsteps=2000)
    full = serve.context_bytes(256, 2000, 8, 5, 0)
    serve.plan_storage(j, full + 1)
    assert j.ckpt_every == 0 and j.bytes == full
    serve.plan_storage(j, full // 10)
    assert 0 < j.ckpt_every < 2000 and j.bytes <= full // 10
    assert serve.context_bytes(256, 2000, 8, 5, j.ckpt_every + 1) > full // 10


def test_admission_by_memory_limits_concurrency():
    per = serve.context_bytes(32, 20, 8, 5, 0)
    srv = serve.Server(serve.FakeExecutor(lambda j: 0.05), memory_budget=int(2.5 * per), slots=8)
    jobs = [job(i, 0.0) for i in range(6)]
    out = srv.run(jobs)
    assert srv.peak_running == 2  # memory admits two at a time
    assert out["jobs"] == 6 and all(j.status == 0 for j in jobs)
    assert all(j.t_admit >= j.arrival and j.t_done > j.t_admit for j in jobs)


def test_slots_limit_concurrency_and_latency_accounting():
    srv = serve.Server(serve.FakeExecutor(lambda j: 0.05), memory_budget=1 << 40, slots=3)
    arr = serve.poisson_arrivals(rate=200.0, count=9, seed=1)
    jobs = [job(i, float(a)) for i, a in enumerate(arr)]
    out = srv.run(jobs)
    assert srv.peak_running <= 3
    lat = np.array([j.latency for j in jobs])
    assert np.all(lat >= 0.05 - 1e-3)
    assert abs(out["p50_latency_s"] - np.percentile(lat, 50)) < 1e-12
    assert out["solves_per_s"] > 0


def test_late_arrival_starts_while_others_run():
    """Continuous batching: a job arriving mid-run is admitted at once if a slot is free."""
    srv = serve.Server(serve.FakeExecutor(lambda j: 0.2 if j.job_id == 0 else 0.02), memory_budget=1 << 40, slots=2)
    jobs = [job(0, 0.0), job(1, 0.05)]
    srv.run(jobs)
    assert jobs[1].t_admit < jobs[0].t_done  # overlapped with job 0
    assert jobs[1].t_admit - jobs[1].arrival < 0.05


def test_oversized_job_is_rejected():
    srv = serve.Server(serve.FakeExecutor(lambda j: 0.0), memory_budget=1000, slots=1, job_cap=1000)
    with pytest.raises(ValueError):
        srv.run([job(0, 0.0)])


@pytest.mark.gpu
def test_memory_model_matches_the_library():
    torch = pytest.importorskip("torch")
    from paper_2602_14016_gb300 import api, build

    build.build()
    for n, nsteps, ck in [(32, 20, 0), (64, 40, 7), (128, 16, 0)]:
        cfg = api.Config(n=n, nsteps=nsteps, dt=1e-3, nu=1e-3, px=8, every=4, ckpt_every=ck)
        ctx = api.Context(cfg)
        m = torch.zeros((1, ctx.nt, 64, 2), dtype=torch.float64, device="cuda")
        ctx.set_observations(m)
        ctx.assimilate(torch.zeros((1, n, n), dtype=torch.float64, device="cuda"), 0)
        est = serve.context_bytes(n, nsteps, 8, 4, ck)
        assert abs(est - ctx.device_bytes) <= 0.01 * ctx.device_bytes, (est, ctx.device_bytes)


@pytest.mark.gpu
def test_results_are_the_same_alone_and_in_the_mix():
    torch = pytest.importorskip("torch")
    import oracle
    from paper_2602_14016_gb300 import synthetic

    specs = [(32, 20, ("exp_abs", 0.5)), (64, 20, ("frac", 0.5)), (32, 40, ("identity", 0.0)), (64, 10, ("frac", 1.0))]
    jobs = []
    for i, (n, nsteps, kern) in enumerate(specs):
        P = oracle.Problem(n=n, nsteps=nsteps, dt=5e-3, nu=1e-3, px=8, every=5, kernel=kern[0], kparam=kern[1])
        truth = oracle.control_from_omega(P, synthetic.random_vorticity_hat(n, 400 + i) * 2)
        guess = oracle.control_from_omega(P, synthetic.random_vorticity_hat(n, 500 + i) * 2)
        _, m = oracle.forward(P, truth)
        j = serve.Job(job_id=i, n=n, nsteps=nsteps, dt=5e-3, nu=1e-3, px=8, every=5, kernel=kern, iters=4,
                      arrival=0.01 * i, m=m[None].copy(), s0=guess[None].copy())
        jobs.append(j)
    alone = []
    for j in jobs:
        a = serve.Job(**{f.name: getattr(j, f.name) for f in serve.dataclasses.fields(serve.Job)})
        serve.Server(serve.CudaExecutor(), memory_budget=1 << 36, slots=1).run([a])
        alone.append(a)
    out = serve.Server(serve.CudaExecutor(), memory_budget=1 << 36, slots=4).run(jobs)
    assert out["jobs"] == len(jobs)
    for a, j in zip(alone, jobs):
        assert j.iters_done == a.iters_done
        assert np.array_equal(j.J_hist, a.J_hist)
        assert np.array_equal(j.s, a.s)


@pytest.mark.gpu
def test_co_batched_results_equal_the_alone_results():
    """Jobs of two grid sizes through the co-batching server (pool slots,
    admission between L-BFGS rounds, shared launches) end with bitwise the
    histories and controls of the same jobs run one at a time."""
    torch = pytest.importorskip("torch")
    import oracle
    from paper_2602_14016_gb300 import synthetic

    specs = [(32, 20, ("exp_abs", 0.5), "none", 1e-3), (32, 40, ("frac", 1.0), "kolmogorov", 1e-2),
             (64, 20, ("frac", 0.5), "none", 1e-3), (32, 10, ("identity", 0.0), "kolmogorov", 1e-2),
             (64, 10, ("exp_sq", 0.7), "kolmogorov", 1e-2)]
    jobs = []
    for i, (n, nsteps, kern, flow, nu) in enumerate(specs):
        px = 8 if i % 2 == 0 else 4
        P = oracle.Problem(n=n, nsteps=nsteps, dt=5e-3, nu=nu, forcing=flow, nf=4, px=px, every=5, kernel=kern[0],
                           kparam=kern[1])
        truth = oracle.control_from_omega(P, synthetic.random_vorticity_hat(n, 600 + i) * 2)
        guess = oracle.control_from_omega(P, synthetic.random_vorticity_hat(n, 700 + i) * 2)
        _, m = oracle.forward(P, truth)
        jobs.append(serve.Job(job_id=i, n=n, nsteps=nsteps, dt=5e-3, nu=nu, px=px, every=5, kernel=kern,
                              forcing=flow, nf=4, iters=4, arrival=0.02 * i, m=m[None].copy(), s0=guess[None].copy()))
    alone = []
    for j in jobs:
        a = serve.Job(**{f.name: getattr(j, f.name) for f in serve.dataclasses.fields(serve.Job)})
        serve.Server(serve.CudaExecutor(), memory_budget=1 << 36, slots=1).run([a])
        alone.append(a)
    srv = serve.CoBatchServer({32: dict(slots=2, nsteps=40, px=8, dt=5e-3), 64: dict(slots=2, nsteps=20, px=8,
                                                                                      dt=5e-3)}, every=5)
    out = srv.run(jobs)
    srv.close()
    assert out["jobs"] == len(jobs) and out["failed"] == 0 and out["peak_members"] >= 2
    for a, j in zip(alone, jobs):
        assert j.status == a.status and j.iters_done == a.iters_done, (j.job_id, j.status, a.status)
        assert np.array_equal(j.J_hist, a.J_hist), (j.job_id, j.J_hist, a.J_hist)
        assert np.array_equal(j.s, a.s), j.job_id
    # the hybrid server: 32^2 jobs co-batched, 64^2 jobs in their own contexts
    mixed = [serve.Job(**{f.name: getattr(j, f.name) for f in serve.dataclasses.fields(serve.Job)}) for j in jobs]
    for j in mixed:
        j.s, j.J_hist, j.status = None, None, -1
    hy = serve.HybridServer({32: dict(slots=2, nsteps=40, px=8, dt=5e-3)}, big_budget=1 << 34, big_slots=2, every=5)
    out = hy.run(mixed)
    hy.close()
    assert out["failed"] == 0 and out["co_batched_jobs"] == 3 and out["own_context_jobs"] == 2
    for a, j in zip(alone, mixed):
        assert np.array_equal(j.J_hist, a.J_hist) and np.array_equal(j.s, a.s), j.job_id
