"""Drivers of the workloads built on the cost-and-gradient path: input
preparation shared with bench.py, the adjoint-statistics ensemble of
Sec. IV, the differentiable 512^2 Kolmogorov window, and Poisson-arrival
serving.  Inputs are seeded and synthetic (see synthetic.py); all
assimilation arithmetic runs in the CUDA library.
"""
from __future__ import annotations

import time

import numpy as np

from . import synthetic


def first_guess_from_probes(w_hat: np.ndarray, n: int, px: int) -> np.ndarray:
    """Vorticity of the trigonometric interpolation of the t = 0 probe
    velocities (the 'initial interpolated state' of Sec. III.A).

    Host-side input preparation: u, v of the truth at the probe lattice,
    their px x px DFT, vorticity i kx v - i ky u on the coarse modes,
    zero-padded into the n^2 half spectrum."""
    KX, KY = synthetic.wavenumbers(n)
    k2 = (KX**2 + KY**2).astype(float)
    ik2 = np.where(k2 > 0, 1.0 / np.where(k2 > 0, k2, 1.0), 0.0)
    u = np.fft.irfft2(1j * KY * ik2 * w_hat, s=(n, n))
    v = np.fft.irfft2(-1j * KX * ik2 * w_hat, s=(n, n))
    st = n // px
    Uc, Vc = np.fft.rfft2(u[::st, ::st]), np.fft.rfft2(v[::st, ::st])
    kxc, kyc = np.meshgrid(np.arange(px // 2 + 1), np.fft.fftfreq(px, 1.0 / px).astype(int))
    Wc = 1j * kxc * Vc - 1j * kyc * Uc
    out = np.zeros((n, n // 2 + 1), complex)
    scale = (n / px) ** 2
    for q in range(px):
        ky = kyc[q, 0]
        if abs(ky) >= px // 2:
            continue
        for p in range(px // 2):
            out[ky % n, p] = Wc[q, p] * scale
    out[0, 0] = 0
    return out


def spin_up(api, torch, n, dt, nu, steps, seed, forcing="none", amp=1.0, nf=4, device=None, chunk=2500):
    """Forward-only spin-up from a seeded unit-energy field; returns w_hat [1, n, nh] on the device."""
    chunk = max(1, min(chunk, steps)) if steps else 1
    ctx = api.Context(api.Config(n=n, nsteps=chunk, dt=dt, nu=nu, forcing=forcing, amp=amp, nf=nf, px=1,
                                 every=chunk, kernels=[api.KernelSpec("identity", 0.0)], store=False), device)
    w = torch.from_numpy(synthetic.random_vorticity_hat(n, seed)[None]).to(ctx.device)
    for _ in range(steps // chunk if steps else 0):
        w, _ = ctx.forward(ctx.control_from_omega(w))
    ctx.close()
    return w


# ---------------------------------------------------------------------------
# Whole assimilations (the plain method of Sec. II and the kernel sweep of
# Sec. III.B)
# ---------------------------------------------------------------------------

def initial_velocity_error(w_est: np.ndarray, w_true: np.ndarray) -> float:
    """Relative L2 error of the initial velocity, ||u_est - u_true|| / ||u_true||
    over the grid (the initial-condition error over u_rms of Sec. III), from
    the two vorticity half spectra (|u_hat|^2 = |w_hat|^2 / k^2)."""
    n = w_true.shape[0]
    KX, KY = synthetic.wavenumbers(n)
    k2 = (KX**2 + KY**2).astype(float)
    wgt = np.where(KX == 0, 1.0, 2.0) / np.where(k2 > 0, k2, np.inf)
    num = np.sum(wgt * np.abs(w_est - w_true) ** 2)
    den = np.sum(wgt * np.abs(w_true) ** 2)
    return float(np.sqrt(num / den))


def assimilation_run(api, torch, cfg, m, w_guess, w_truth, iters, graphs=True, tune_steps=4, plan=None):
    """One cost-and-gradient evaluation at the first guess, then `iters` L-BFGS
    iterations of every member (da_assimilate).  m: observations [B, nt, P^2, 2];
    w_guess, w_truth: vorticity half spectra [B or 1, n, nh].  plan: a fixed
    FFT plan variant instead of the autotuner's choice.  Returns timings,
    J histories, statuses and initial-velocity errors before and after."""
    ctx = api.Context(cfg)
    if plan is not None:
        ctx.set_plan(plan)
    elif tune_steps > 0:
        ctx.autotune(tune_steps)
    if graphs:
        ctx.set_graphs(True)
    B = cfg.batch
    dev = ctx.device
    ctx.set_observations(torch.from_numpy(np.ascontiguousarray(m)).to(dev))
    wg = np.broadcast_to(w_guess, (B,) + w_guess.shape[-2:]).copy()
    s = ctx.control_from_omega(torch.from_numpy(wg).to(dev))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J0, g0 = ctx.cost_grad(s)
    torch.cuda.synchronize()
    t_eval = time.perf_counter() - t0
    t0 = time.perf_counter()
    res = ctx.assimilate(s, iters)
    torch.cuda.synchronize()
    t_assim = time.perf_counter() - t0
    w_est = ctx.omega_from_control(s).cpu().numpy()
    wt = np.broadcast_to(w_truth, w_est.shape)
    out = {"seconds_first_evaluation": t_eval, "seconds_assimilation": t_assim, "plan": ctx.plan,
           "members": [{"kernel": f"{k.kind}:{k.param}", "J0": float(res.J_hist[b][0]), "J_final": float(res.J_hist[b][-1]),
                        "iters": int(res.iters[b]), "status": int(res.member_status[b]),
                        "ic_error_first_guess": initial_velocity_error(wg[b], wt[b]),
                        "ic_error_final": initial_velocity_error(w_est[b], wt[b]),
                        "J_hist": [float(x) for x in res.J_hist[b]]}
                       for b, k in enumerate(cfg.kernels)]}
    ctx.close()
    return out


# ---------------------------------------------------------------------------
# Adjoint statistics ensemble (Sec. IV)
# ---------------------------------------------------------------------------

def ensemble_statistics(api, torch, groups, nsteps=1000, save_every=10, ckpt_every=50, streams=True):
    """Adjoint Green's-function statistics of ensembles of decaying turbulence.

    groups: list of dicts (n, count, nu, dt, seed0).  Every realisation is a
    seeded unit-energy field (spectrum k^4 exp(-2 (k/4)^2)) run forward
    nsteps steps; its adjoint runs back from a seeded unit-norm terminal
    field.  Returns per group the ensemble-mean shell energy of the adjoint
    velocity, the shell energy of the ensemble-mean adjoint, their ratio,
    fitted backward growth rates per shell, and the throughput."""
    out = []
    ctxs, sts, jobs = [], [], []
    for g in groups:
        n, B = g["n"], g["count"]
        cfg = api.Config(n=n, nsteps=nsteps, dt=g["dt"], nu=g["nu"], px=1, every=nsteps,
                         kernels=[api.KernelSpec("identity", 0.0)] * B, ckpt_every=ckpt_every)
        ctx = api.Context(cfg)
        g["fft_plan"], g["plan_ms_per_step"] = ctx.autotune(4)  # the autotuner picks the plan per grid and batch
        ctx.set_graphs(True)  # the whole sweep (forward, recompute, adjoint, spectra) as one CUDA graph
        w = torch.from_numpy(np.stack([synthetic.random_vorticity_hat(n, g["seed0"] + b) for b in range(B)]))
        s = ctx.control_from_omega(w.to(ctx.device))
        lamT = torch.from_numpy(np.stack([synthetic.unit_norm_terminal_hat(n, 10_000 + g["seed0"] + b)
                                          for b in range(B)])).to(ctx.device)
        ctxs.append(ctx)
        jobs.append((s, lamT))
        sts.append(torch.cuda.Stream() if streams else torch.cuda.current_stream())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    results = []
    for ctx, (s, lamT), st in zip(ctxs, jobs, sts):
        with torch.cuda.stream(st):
            results.append(ctx.adjoint_spectra(s, lamT, save_every, stream=st))
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    units = sum(g["count"] * g["n"] ** 2 * nsteps for g in groups)
    for g, ctx, (member, mean) in zip(groups, ctxs, results):
        member = member.cpu().numpy()
        mean = mean.cpu().numpy()
        tau = np.arange(member.shape[1]) * save_every * g["dt"]
        avg_energy = member.mean(axis=0)  # mean over realisations of the shell energy
        rates = fit_growth_rates(tau, avg_energy)
        out.append({"n": g["n"], "count": g["count"], "tau": tau, "mean_of_energy": avg_energy,
                    "energy_of_mean": mean, "snr": mean.sum(axis=1) / avg_energy.sum(axis=1),
                    "growth_rates": rates, "device_bytes": ctx.device_bytes})
        ctx.close()
    return out, {"gridpoint_steps": units, "seconds": secs, "value": units / secs}


def fit_growth_rates(tau: np.ndarray, energy: np.ndarray, skip: float = 0.3) -> np.ndarray:
    """Least-squares slope of log E(k, tau) against backward time per shell,
    after an initial transient of `skip` time units (Sec. IV)."""
    sel = tau >= skip
    rates = np.full(energy.shape[1], np.nan)
    for k in range(energy.shape[1]):
        e = energy[sel, k]
        if np.all(e > 0) and sel.sum() >= 2:
            rates[k] = np.polyfit(tau[sel], np.log(e), 1)[0]
    return rates


# ---------------------------------------------------------------------------
# Differentiable Kolmogorov window
# ---------------------------------------------------------------------------

def autograd_check(api, torch, n=512, nsteps=4000, dt=1e-3, nu=1 / 200, nf=4, ckpt_every=64, directions=8,
                   eps=(1e-4, 1e-5, 1e-6), px=16, every=40, seed=3):
    """Gradient of a torch loss through the autograd wrapper against central
    finite differences of the same loss along seeded random directions, at
    several step sizes: over a long chaotic window the difference quotient is
    truncation-limited at large steps and rounding-limited at small ones, so
    the agreement is reported per step size and at the best one."""
    from . import autograd as ag

    cfg = api.Config(n=n, nsteps=nsteps, dt=dt, nu=nu, forcing="kolmogorov", nf=nf, px=px, every=every,
                     kernels=[api.KernelSpec("frac", 0.5)], ckpt_every=ckpt_every)
    ctx = api.Context(cfg)
    truth = spin_up(api, torch, n, dt, nu, 2000, seed, forcing="kolmogorov", nf=nf)
    s_truth = ctx.control_from_omega(truth)
    _, m = ctx.forward(s_truth)
    guess = torch.from_numpy(first_guess_from_probes(truth.cpu().numpy()[0], n, px)[None]).cuda()
    s0 = ctx.control_from_omega(guess)
    # the first gradient of a process can also pay one-time set-up: on a
    # fresh GB300 machine the first autograd backward took about 5 s more
    # than later ones (not when an earlier process had run there), while a
    # first da_vjp called directly takes about 0.3 s more; the second
    # gradient is the steady cost
    t_grad = []
    for _ in range(2):
        s = s0.clone().requires_grad_(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        obs, _ = ag.solve(s, ctx)
        L = ag.misfit(obs, m).sum()
        L.backward()
        torch.cuda.synchronize()
        t_grad.append(time.perf_counter() - t0)
    g = s.grad.detach()
    errs = np.zeros((len(eps), directions))
    for k in range(directions):
        d = torch.from_numpy(synthetic.random_field(n, 9000 + k)[None]).cuda()
        d = d / torch.linalg.norm(d)
        gd = float((g * d).sum())
        for i, e in enumerate(eps):
            Lp = ag.misfit(ctx.forward(s0 + e * d)[1], m).sum().item()
            Lm = ag.misfit(ctx.forward(s0 - e * d)[1], m).sum().item()
            errs[i, k] = abs((Lp - Lm) / (2 * e) - gd) / max(abs(gd), 1e-300)
    best = errs.min(axis=0)
    out = {"n": n, "nsteps": nsteps, "ckpt_every": ckpt_every, "device_bytes": ctx.device_bytes,
           "full_storage_bytes": nsteps * 8 * n * n * 8, "loss": float(L.detach()), "grad_seconds": t_grad[1],
           "grad_seconds_first_call": t_grad[0],
           "directions": directions, "eps": list(eps),
           "fd_rel_err_median_per_eps": [float(np.median(r)) for r in errs],
           "fd_rel_err_best_eps_median": float(np.median(best)), "fd_rel_err_best_eps_max": float(best.max())}
    ctx.close()
    return out


# ---------------------------------------------------------------------------
# Throughput per grid size
# ---------------------------------------------------------------------------

def grid_sweep(api, torch, grids=(64, 128, 256, 512, 1024), batches=(1, 8), steps=200, repeats=3, tune_steps=4):
    """Cost-and-gradient throughput (gridpoint-steps/s, graph replay) of a
    decaying-turbulence window per grid size and batch, each context on the
    plan its autotuner keeps.  Inputs: seeded unit-energy fields, probe data
    of a second seed, 8x8 probes every 10 steps."""
    dts = {64: 5e-3, 128: 4e-3, 256: 2e-3, 512: 1e-3, 1024: 5e-4}
    rows = []
    for n in grids:
        for B in batches:
            cfg = api.Config(n=n, nsteps=steps, dt=dts[n], nu=1e-3, px=8, every=10,
                             kernels=[api.KernelSpec("exp_abs", 0.5)] * B)
            ctx = api.Context(cfg)
            plan, plan_ms = ctx.autotune(tune_steps) if tune_steps > 0 else (ctx.plan, None)
            w = torch.from_numpy(np.stack([synthetic.random_vorticity_hat(n, 1000 + b) for b in range(B)])).cuda()
            _, m = ctx.forward(ctx.control_from_omega(w))
            ctx.set_observations(m)
            s = ctx.control_from_omega(
                torch.from_numpy(np.stack([synthetic.random_vorticity_hat(n, 2000 + b) for b in range(B)])).cuda())
            ctx.set_graphs(True)
            for _ in range(2):
                ctx.cost_grad(s)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(repeats):
                ctx.cost_grad(s)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / repeats
            rows.append({"n": n, "batch": B, "steps": steps, "ms_per_evaluation": ms,
                         "gridpoint_steps_per_s": B * n * n * steps / (ms / 1e3), "fft_plan": plan,
                         "plan_ms_per_step": plan_ms})
            ctx.close()
    return rows


# ---------------------------------------------------------------------------
# Serving
# ---------------------------------------------------------------------------

def serving_jobs(api, torch, count, rate, seed, grids=(128, 256, 512), weights=(0.5, 0.35, 0.15),
                 steps=(200, 600), iters=5):
    """Seeded job mix: grid by weight, horizon uniform (multiple of 10),
    probes 4..32 per side, decaying or Kolmogorov flow, exponential or
    fractional kernel; observations of a seeded truth, first guess from
    another seed.  Poisson arrival times at `rate` jobs/s."""
    from . import serve

    rng = np.random.default_rng(seed)
    arr = serve.poisson_arrivals(rate, count, seed + 1)
    jobs = []
    for i in range(count):
        n = int(rng.choice(grids, p=np.array(weights) / np.sum(weights)))
        nsteps = int(rng.integers(steps[0] // 10, steps[1] // 10 + 1)) * 10
        px = int(rng.choice([p for p in (4, 8, 16, 32) if n % p == 0]))
        kolm = bool(rng.integers(0, 2))
        kern = ("exp_abs", float(rng.choice([0.1, 0.3, 1.0]))) if rng.integers(0, 2) else \
            ("frac", float(rng.choice([0.0, 0.5, 1.0, 1.5])))
        dt = {128: 4e-3, 256: 2e-3, 512: 1e-3, 1024: 5e-4}[n]
        nu = 1e-2 if kolm else 1e-3
        cfg = api.Config(n=n, nsteps=nsteps, dt=dt, nu=nu, forcing="kolmogorov" if kolm else "none", nf=4, px=px,
                         every=10, kernels=[api.KernelSpec(*kern)], store=False)
        ctx = api.Context(cfg)
        w_t = torch.from_numpy(synthetic.random_vorticity_hat(n, 20_000 + i)[None]).cuda()
        _, m = ctx.forward(ctx.control_from_omega(w_t))
        s0 = ctx.control_from_omega(torch.from_numpy(synthetic.random_vorticity_hat(n, 30_000 + i)[None]).cuda())
        jobs.append(serve.Job(job_id=i, n=n, nsteps=nsteps, dt=dt, nu=nu, px=px, every=10, kernel=kern,
                              forcing="kolmogorov" if kolm else "none", nf=4, iters=iters, arrival=float(arr[i]),
                              m=m.cpu().numpy(), s0=s0.cpu().numpy()))
        ctx.close()
    return jobs
