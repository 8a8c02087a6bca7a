#!/usr/bin/env python
"""Throughput of the FP64 cost-and-gradient evaluation on GB300.

Workload (one "step" = one batched cost-and-gradient evaluation, the whole
hot path): forced Kolmogorov flow on a 256^2 grid, f = (sin 4y, 0),
nu = 1/100, spun up 50 time units (25,000 RK4 steps of 2e-3, untimed) from a
seeded unit-energy field; window of 2000 RK4 steps of 2e-3; 16x16 velocity
probes every 20 steps with 1 % Gaussian noise; first guess from the
trigonometric interpolation of the t = 0 probe velocities; the seven kernels
of the sweep |k|^(-2s), s in {0, 0.5, 1, 1.5}, and exp(-a|k|), a in
{0.1, 0.3, 1}, evaluated together as one batch of seven members.

Metric: fwd+adjoint gridpoint-steps/s (FP64) = members x n^2 x nsteps per
evaluation / time.  The timed region holds K evaluations with the inputs
resident on the device; the stage-field trajectory of an evaluation
(58.7 GB) is far larger than L2, so no flush is needed.  `e2e` repeats the
measurement through the public API from pinned host memory (controls in,
cost and gradient out).  `--impl reference` times the CPU oracle on a
bounded sample of the same workload.  Under torchrun each rank runs its
own batch (replicas; weak scaling).
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SWEEP = [("frac", 0.0), ("frac", 0.5), ("frac", 1.0), ("frac", 1.5), ("exp_abs", 0.1), ("exp_abs", 0.3),
         ("exp_abs", 1.0)]
W = dict(n=256, nsteps=2000, dt=2e-3, nu=1e-2, forcing="kolmogorov", amp=1.0, nf=4, px=16, every=20, noise=0.01,
         spinup_steps=25000, seed=0)
WORKLOAD_NAME = "kolmogorov-256sq-2000steps-16x16probes-7kernel-sweep"
METRIC = "fwd+adjoint gridpoint-steps/s FP64"
UNIT = "gridpoint-steps/s"

PROBE_KINDS = {0: "dfma_reg_const", 1: "dfma_3reg", 2: "dadd", 3: "dmul"}


def sm_max_mhz() -> tuple:
    """Maximum SM clock: MEASURED_PEAKS.json, else the recipe's 2070 MHz."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"]), "MEASURED_PEAKS.json sm_max_mhz"
    except (OSError, KeyError, ValueError):
        return 2070.0, "recipe maximum SM clock"


def fp64_probe(kinds=(0, 1, 2, 3), iters: int = 100000) -> dict:
    """Runs da_fp64_probe (csrc/fp64_probe.cu) for each kind on the current
    device: {name: {gflops, ops_per_clk_per_sm, sm_mhz}}."""
    import ctypes

    import torch

    from paper_2602_14016_gb300 import _native as NN

    lib = NN.load()
    out = {}
    for k in kinds:
        g, r, mhz = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        st = lib.da_fp64_probe(k, iters, ctypes.byref(g), ctypes.byref(r), ctypes.byref(mhz),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        if st != NN.DA_OK:
            raise RuntimeError(f"da_fp64_probe({k}) returned {st}")
        out[PROBE_KINDS[k]] = {"gflops": g.value, "ops_per_clk_per_sm": r.value, "sm_mhz": mhz.value}
    return out


def fp64_peak(probe: dict, sms: int) -> dict:
    """Roofline denominator of the FP64-bound pass kernels, derived from unit
    counts and clocks: SMs x DFMA per clock per SM x 2 flop x maximum SM clock.
    The DFMA rate per SM is the probe's best DFMA rate rounded to a whole
    number of operations per clock (the pipe issues whole operations)."""
    best = max(probe[k]["ops_per_clk_per_sm"] for k in ("dfma_reg_const", "dfma_3reg") if k in probe)
    units = max(1, round(best))
    mhz, src = sm_max_mhz()
    return {"gflops": sms * units * 2 * mhz / 1e3, "sms": sms, "dfma_per_clk_per_sm": units,
            "probe_best_dfma_per_clk_per_sm": best, "sm_max_mhz": mhz, "clock_source": src,
            "source": "derived: SMs x DFMA/clk/SM (da_fp64_probe, this run) x 2 flop x max SM clock"}

# DRAM bytes (read + write) per launch of each pass kernel at this workload
# (256^2, batch 7), from one ncu capture of the same launch configuration on
# a 40-step window (per-launch data are the same for any window length);
# valid only for the kernel sources they were taken from.
TRAFFIC = {"src_hash": "ebf205b24a74b487", "adj_rows": 12301312, "adj_cols": 10530816, "fwd_rows": 4977152,
           "fwd_cols": 10495744}


def src_hash() -> str:
    """Hash of the sources of the pass kernels and their launch configuration
    (kernels, FFT engine, launchers, instantiations), with comments and blank
    space removed: what the measured traffic figures depend on.  Host code
    that only orders launches is left out."""
    csrc = os.path.join(ROOT, "paper_2602_14016_gb300", "csrc")
    files = [os.path.join(csrc, f) for f in ("kernels.cuh", "fft.cuh", "ops.h", "ops_impl.cuh")]
    files += glob.glob(os.path.join(csrc, "inst_n*.cu"))
    h = hashlib.sha256()
    for p in sorted(files):
        with open(p, encoding="utf-8") as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def hbm_fraction(traffic, avg_ms):
    """DRAM bandwidth the dominant kernel uses (measured bytes per launch over
    its launch time) against the measured HBM copy peak: the %HBM view of a
    kernel whose bound is the FP64 pipe."""
    if traffic is None or not avg_ms:
        return None
    peak, src = 6800.0, "fallback"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak, src = float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        pass
    gbs = traffic / (avg_ms * 1e-3) / 1e9
    return {"achieved_gbs": gbs, "peak_gbs": peak, "frac": gbs / peak, "peak_source": src}


def pass_flops(n: int, batch: int, variant: int = 0) -> dict:
    """Algorithmic FP64 flops per launch of each pass kernel: the nominal
    count of the transforms it performs plus its pointwise arithmetic.  A
    transform counts 5 n log2 n less the operations the kernels skip on the
    gap of the 2/3 rule under this plan variant (da_plan_flops: zero inputs
    of an inverse transform's first stage, unused outputs of a forward
    transform's last stage)."""
    from paper_2602_14016_gb300 import api

    K = (n - 1) // 3
    Kc, Kr = K + 1, 2 * K + 1
    fi, ff = api.plan_flops(n, variant)
    # rows: per row pair one inverse transform of the packed pair (u + i v,
    # or the adjoint fields a + i b) per row and one forward transform of the
    # two products per row; columns: two forward and two inverse transforms
    # per retained column kx
    return {
        "fwd_rows": batch * (n * (fi + ff) + 4.0 * n * n),
        "fwd_cols": batch * (2.0 * Kc * (fi + ff) + 26.0 * Kr * Kc),
        "adj_rows": batch * (n * (fi + ff) + 8.0 * n * n),
        "adj_cols": batch * (2.0 * Kc * (fi + ff) + 32.0 * Kr * Kc),
    }


def flops_per_gridpoint_step(n: int, variant: int = 0) -> float:
    p = pass_flops(n, 1, variant)
    return 4.0 * sum(p.values()) / (n * n)


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.p = None
        return self

    def __exit__(self, *exc):
        if self.p is not None:
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                out, _ = self.p.communicate()
            self.out = out
        return False

    def summary(self):
        if self.p is None:
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in getattr(self, "out", "").splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def prepare(api, torch, kernels, device):
    """Spin-up, truth observations with noise, first-guess controls."""
    from paper_2602_14016_gb300 import synthetic

    n, nsteps = W["n"], W["nsteps"]
    chunk = min(2500, W["spinup_steps"]) or 1
    spin = api.Context(api.Config(n=n, nsteps=chunk, dt=W["dt"], nu=W["nu"], forcing=W["forcing"], amp=W["amp"],
                                  nf=W["nf"], px=W["px"], every=chunk, kernels=[api.KernelSpec("identity", 0.0)],
                                  store=False), device)
    w = torch.from_numpy(synthetic.random_vorticity_hat(n, W["seed"])[None]).to(device)
    for _ in range(W["spinup_steps"] // chunk if W["spinup_steps"] else 0):
        s0 = spin.control_from_omega(w)
        w, _ = spin.forward(s0)
    win = api.Context(api.Config(n=n, nsteps=nsteps, dt=W["dt"], nu=W["nu"], forcing=W["forcing"], amp=W["amp"],
                                 nf=W["nf"], px=W["px"], every=W["every"], kernels=[api.KernelSpec("identity", 0.0)],
                                 store=False), device)
    s_truth = win.control_from_omega(w)
    _, obs = win.forward(s_truth)
    obs = obs.cpu().numpy()[0]
    rms = float(np.sqrt(np.mean(obs**2)))
    m = obs + W["noise"] * rms * synthetic.gaussian_draws(obs.shape, W["seed"] + 1)
    w_truth = w.cpu().numpy()[0]
    spin.close()
    win.close()
    from paper_2602_14016_gb300.workloads import first_guess_from_probes

    w_guess = first_guess_from_probes(w_truth, n, W["px"])
    B = len(kernels)
    return np.repeat(m[None], B, 0), np.repeat(w_guess[None], B, 0), w_truth


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2602_14016_gb300 import api, build, replicas

    rank, local, world = replicas.env_world()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    kernels = SWEEP
    B = len(kernels)
    n, nsteps = W["n"], W["nsteps"]
    m, w_guess, _ = prepare(api, torch, kernels, device)
    cfg = api.Config(n=n, nsteps=nsteps, dt=W["dt"], nu=W["nu"], forcing=W["forcing"], amp=W["amp"], nf=W["nf"],
                     px=W["px"], every=W["every"], kernels=[api.KernelSpec(k, a) for k, a in kernels])
    ctx = api.Context(cfg, device)
    # FFT plan: the autotuner times each variant on this batch (outside the
    # timed region) and keeps the fastest
    tune = {"chosen": ctx.plan, "ms_per_step": None}
    if args.plan is not None:
        ctx.set_plan(args.plan)
        tune["chosen"] = ctx.plan
    elif args.tune_steps > 0:
        tune["chosen"], tune["ms_per_step"] = ctx.autotune(args.tune_steps)
    ctx.set_observations(torch.from_numpy(m).to(device))
    s = ctx.control_from_omega(torch.from_numpy(w_guess).to(device))
    stream = torch.cuda.current_stream()

    # warm-up; with at least four, the first four time one pass-kernel class
    # each (direct launches), the rest replay the captured CUDA graph
    classes = ["fwd_rows", "fwd_cols", "adj_rows", "adj_cols"]
    class_ms = {}
    warm = max(args.warmup, 5 if args.warmup >= 4 else 1) if args.graphs else args.warmup
    for i in range(warm):
        timed = i < 4 and args.warmup >= 4
        if timed:
            ctx.time_kernels(classes[i])
        else:
            ctx.time_kernels("off")
            ctx.set_graphs(args.graphs)
        J, g = ctx.cost_grad(s)
        torch.cuda.synchronize()
        if timed:
            class_ms[classes[i]] = ctx.kernel_time()
    ctx.time_kernels("off")
    ctx.set_graphs(args.graphs)
    dom = args.roofline_class or (max(class_ms, key=lambda c: class_ms[c][0]) if class_ms else "adj_rows")
    Jw = J.cpu().numpy()
    if not np.all(np.isfinite(Jw)):
        raise RuntimeError(f"non-finite cost in warm-up: {Jw}")

    # timed region: K evaluations, inputs resident
    launches0 = ctx.launches
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed")
        ev0.record(stream)
        for _ in range(args.steps):
            J, g = ctx.cost_grad(s)
        ev1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    ms = ev0.elapsed_time(ev1)
    launches = ctx.launches - launches0
    # whole job: the units of every rank over the slowest rank's time
    value = replicas.whole_job_rate(B * n * n * nsteps * args.steps, ms / 1e3, device)
    ms = replicas.max_over_ranks(ms, device)
    if world > 1:
        dist.barrier()

    # roofline pass: the same evaluation with direct launches and CUDA events
    # around every launch of the dominant pass kernel
    ctx.time_kernels(dom)
    rp0, rp1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rp0.record(stream)
    for _ in range(args.roofline_evals):
        ctx.cost_grad(s)
    rp1.record(stream)
    torch.cuda.synchronize()
    dom_ms, dom_n = ctx.kernel_time()
    roof_pass_ms = rp0.elapsed_time(rp1) / args.roofline_evals
    ctx.time_kernels("off")
    ctx.set_graphs(args.graphs)

    # end to end through the public API from pinned host memory
    s_host = s.cpu().pin_memory()
    J_host = torch.empty(B, dtype=torch.float64).pin_memory()
    g_host = torch.empty_like(s_host).pin_memory()
    ctx.cost_grad(s_host.to(device, non_blocking=True))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_steps = max(1, min(args.steps, 3))
    e0.record(stream)
    for _ in range(e_steps):
        s_dev = s_host.to(device, non_blocking=True)
        J, g = ctx.cost_grad(s_dev)
        J_host.copy_(J, non_blocking=True)
        g_host.copy_(g, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e_ms = e0.elapsed_time(e1)
    e2e_value = replicas.whole_job_rate(B * n * n * nsteps * e_steps, e_ms / 1e3, device)

    plan = ctx.plan  # the batch context is freed before the plain path runs
    # the plain one-job-per-launch path: the same members one at a time
    plain = None
    if rank == 0 and args.plain:
        cfg1 = api.Config(n=n, nsteps=nsteps, dt=W["dt"], nu=W["nu"], forcing=W["forcing"], amp=W["amp"],
                          nf=W["nf"], px=W["px"], every=W["every"], kernels=[api.KernelSpec(*kernels[0])])
        del ctx
        torch.cuda.empty_cache()
        ctx1 = api.Context(cfg1, device)
        if args.tune_steps > 0:
            ctx1.autotune(args.tune_steps)
        ctx1.set_observations(torch.from_numpy(m[:1]).to(device))
        s1 = [ctx1.control_from_omega(torch.from_numpy(w_guess[:1]).to(device))]
        ctx1.cost_grad(s1[0])
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(B):
            ctx1.cost_grad(s1[0])
        p1.record(stream)
        torch.cuda.synchronize()
        p_ms = p0.elapsed_time(p1)
        plain = {"value": B * n * n * nsteps / (p_ms / 1e3), "unit": UNIT, "ms_per_member": p_ms / B,
                 "note": "same members evaluated one per launch sequence (batch 1)"}
        ctx1.close()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    pf = pass_flops(n, B, plan)[dom]
    avg_ms = dom_ms / max(dom_n, 1)
    achieved = pf / (avg_ms / 1e3) / 1e9
    probe = fp64_probe((0, 1), iters=50000)
    peak = fp64_peak(probe, torch.cuda.get_device_properties(device).multi_processor_count)
    peak_gflops = peak["gflops"]
    traffic = TRAFFIC.get(dom) if (TRAFFIC.get("src_hash") == src_hash() and n == 256 and B == 7) else None
    cpu = cpu_baseline(args) if args.cpu_baseline else None
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded spun-up Kolmogorov flow, noisy probe observations)",
        "config": {"workload": WORKLOAD_NAME, "grid": n, "nsteps": nsteps, "dt": W["dt"], "nu": W["nu"],
                   "launch": "CUDA graph replay of each evaluation" if args.graphs else "stream launches",
                   "probes": f"{W['px']}x{W['px']} every {W['every']}", "members_per_gpu": B,
                   "kernels": [f"{k}:{a}" for k, a in kernels], "l2": "inputs larger than L2 (58.7 GB stage-field "
                   "trajectory streamed per evaluation)", "parallelism": f"replicas x{world}"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(s_host.numel() * 8),
                "d2h_bytes_per_step": int(J_host.numel() * 8 + g_host.numel() * 8)},
        "gpu_launches": int(launches),
        "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak_gflops,
                     "unit": "GFLOP/s", "frac": achieved / peak_gflops, "traffic": traffic,
                     "flops_per_launch": pf, "avg_launch_ms": avg_ms, "launches_timed": dom_n,
                     "timed_in": "roofline pass of the same workload, direct launches, CUDA events per launch",
                     "roofline_pass_ms_per_step": roof_pass_ms,
                     "class_ms_warmup": {k: v[0] for k, v in class_ms.items()},
                     "hbm": hbm_fraction(traffic, avg_ms), "peak_derivation": peak, "fp64_probe": probe},
        "flops_per_gridpoint_step": flops_per_gridpoint_step(n, plan),
        "achieved_gflops_step": value * flops_per_gridpoint_step(n, plan) / 1e9,
        "cpu_baseline": cpu,
        "plain_path": plain,
        "fft_plan": tune,
        "clocks": clk.summary(),
        "J_mean": float(np.mean(J.cpu().numpy())),
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _oracle_member_sample(args):
    """One oracle cost-and-gradient evaluation of the first n_sample_steps
    steps of the window (one observation time) for one sweep member; returns
    its wall seconds (spawned worker)."""
    n_sample_steps, kernel, kp = args
    import oracle
    from paper_2602_14016_gb300 import synthetic

    n = W["n"]
    P = oracle.Problem(n=n, nsteps=n_sample_steps, dt=W["dt"], nu=W["nu"], forcing=W["forcing"], amp=W["amp"],
                       nf=W["nf"], px=W["px"], every=n_sample_steps, kernel=kernel, kparam=kp)
    truth = oracle.control_from_omega(P, synthetic.random_vorticity_hat(n, W["seed"]))
    guess = oracle.control_from_omega(P, synthetic.random_vorticity_hat(n, W["seed"] + 2))
    _, m = oracle.forward(P, truth)
    t0 = time.perf_counter()
    oracle.cost_grad(P, guess, m)
    return time.perf_counter() - t0


def oracle_sample(n_sample_steps: int, members=SWEEP):
    """The oracle on a bounded sample of the workload: the first
    n_sample_steps steps of the window for every sweep member, one
    single-threaded process per member running at the same time (the batch's
    members are independent jobs).  Returns (gridpoint-steps/s over the wall
    time of the slowest member, that wall time, processes)."""
    import multiprocessing as mp

    import oracle

    oracle.build()
    procs = min(len(members), os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(procs) as pool:
        secs = pool.map(_oracle_member_sample, [(n_sample_steps, k, a) for k, a in members])
    wall = max(secs) if procs >= len(members) else sum(secs) / procs
    return len(members) * W["n"] ** 2 * n_sample_steps / wall, wall, procs


def cpu_baseline(args):
    oracle_steps = 20
    val, secs, procs = oracle_sample(oracle_steps)
    return {"value": val, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"one cost+gradient evaluation of the first {oracle_steps} steps of the 256^2 window for each of "
                      f"the {len(SWEEP)} sweep members, one single-threaded C oracle process per member on "
                      f"{procs} host cores ({secs:.1f} s)"}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    oracle_steps = 20
    for _ in range(args.warmup):
        oracle_sample(2)
    total_units, total_s, procs = 0.0, 0.0, 1
    for _ in range(args.steps):
        v, s, procs = oracle_sample(oracle_steps)
        total_units += len(SWEEP) * W["n"] ** 2 * oracle_steps
        total_s += s
    value = total_units / total_s
    sample = (f"each step one cost+gradient evaluation of the first {oracle_steps} steps of the 256^2 window for "
              f"each of the {len(SWEEP)} sweep members, one single-threaded C oracle process per member")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "grid": W["n"], "sample_steps": oracle_steps,
                   "members": len(SWEEP)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample},
    }), flush=True)


def run_workload(args):
    """Secondary workloads (one JSON line each): the adjoint-statistics
    ensemble, the differentiable 512^2 window, Poisson-arrival serving."""
    import torch

    from paper_2602_14016_gb300 import api, build, workloads

    build.build()
    torch.cuda.set_device(0)
    line = {"workload": args.workload, "dtype": "f64", "data": "synthetic", "n_gpus": 1}
    if args.workload == "ensemble":
        groups = [dict(n=256, count=args.ens256, nu=5e-4, dt=2e-3, seed0=0),
                  dict(n=512, count=args.ens512, nu=5e-4, dt=1e-3, seed0=256)]
        groups = [g for g in groups if g["count"] > 0]
        res, perf = workloads.ensemble_statistics(api, torch, groups, nsteps=args.ens_steps, save_every=10,
                                                  ckpt_every=args.ens_ckpt)
        line.update({"metric": "fwd+adjoint gridpoint-steps/s FP64 (recompute included)", "value": perf["value"],
                     "unit": UNIT, "seconds": perf["seconds"], "config": {"groups": groups,
                     "nsteps": args.ens_steps, "ckpt_every": args.ens_ckpt, "save_every": 10}})
        line["groups"] = [{"n": r["n"], "count": r["count"], "device_bytes": r["device_bytes"],
                           "growth_rate_per_shell": [None if not np.isfinite(x) else round(float(x), 4)
                                                     for x in r["growth_rates"][:64]],
                           "snr_first_last": [float(r["snr"][0]), float(r["snr"][-1])],
                           "total_mean_energy_first_last": [float(r["mean_of_energy"][0].sum()),
                                                            float(r["mean_of_energy"][-1].sum())]}
                          for r in res]
    elif args.workload == "autograd":
        out = workloads.autograd_check(api, torch, n=args.ag_n, nsteps=args.ag_steps, ckpt_every=64,
                                       directions=args.ag_dirs)
        line.update({"metric": "autograd gradient vs central differences", **out})
    elif args.workload == "grids":
        rows = workloads.grid_sweep(api, torch)
        line.update({"metric": "fwd+adjoint gridpoint-steps/s FP64 per grid size and batch", "unit": UNIT,
                     "rows": rows, "config": {"flow": "decaying, nu 1e-3", "probes": "8x8 every 10 steps",
                                              "kernel": "exp_abs:0.5", "launch": "CUDA graph replay"}})
    elif args.workload == "plain":
        # the plain method: 64^2 decaying turbulence, 200 RK4 steps of 5e-3, nu = 1e-3, 8x8 probes every
        # 10 steps (noise-free), W = exp(-0.5|k|), first guess from the t = 0 probes; one evaluation,
        # then 10 L-BFGS iterations
        n, nsteps = 64, 200
        cfg = api.Config(n=n, nsteps=nsteps, dt=5e-3, nu=1e-3, px=8, every=10,
                         kernels=[api.KernelSpec("exp_abs", 0.5)])
        from paper_2602_14016_gb300 import synthetic

        w_truth = synthetic.random_vorticity_hat(n, 0)
        fwd = api.Context(api.Config(**{**cfg.__dict__, "store": False}))
        _, obs = fwd.forward(fwd.control_from_omega(torch.from_numpy(w_truth[None]).cuda()))
        fwd.close()
        w_guess = workloads.first_guess_from_probes(w_truth, n, 8)
        out = workloads.assimilation_run(api, torch, cfg, obs.cpu().numpy(), w_guess[None], w_truth[None],
                                         args.assim_iters, plan=args.plan)
        line.update({"metric": "plain-method assimilation: first evaluation and L-BFGS iterations", **out,
                     "config": {"grid": n, "nsteps": nsteps, "dt": 5e-3, "nu": 1e-3, "probes": "8x8 every 10",
                                "kernel": "exp_abs:0.5", "iters": args.assim_iters}})
    elif args.workload == "sweep-assim":
        # the kernel sweep's full assimilation: the headline window, every member run through
        # --assim-iters L-BFGS iterations from the probe-interpolated first guess
        kernels = SWEEP
        dev = torch.device("cuda", 0)
        m, w_guess, w_truth = prepare(api, torch, kernels, dev)
        cfg = api.Config(n=W["n"], nsteps=W["nsteps"], dt=W["dt"], nu=W["nu"], forcing=W["forcing"], amp=W["amp"],
                         nf=W["nf"], px=W["px"], every=W["every"], kernels=[api.KernelSpec(k, a) for k, a in kernels])
        out = workloads.assimilation_run(api, torch, cfg, m, w_guess, w_truth[None], args.assim_iters)
        line.update({"metric": "kernel-sweep assimilation (Sec. III.B): J and initial-condition error per kernel",
                     **out, "config": {"workload": WORKLOAD_NAME, "iters": args.assim_iters}})
    elif args.workload == "fp64peak":
        with ClockSampler(0) as clk:
            probe = fp64_probe(iters=args.probe_iters)
        peak = fp64_peak(probe, torch.cuda.get_device_properties(0).multi_processor_count)
        line.update({"metric": "FP64 throughput per operation kind (GFLOP/s; DFMA counts 2)", "unit": "GFLOP/s",
                     "kinds": probe, "roofline_peak": peak, "clocks": clk.summary(),
                     "config": {"probe": "8 independent chains per thread, 4 CTAs x 256 threads per SM",
                                "iters": args.probe_iters}})
    elif args.workload == "serve":
        from paper_2602_14016_gb300 import serve

        summary = {}
        dts = {128: 4e-3, 256: 2e-3, 512: 1e-3, 1024: 5e-4}
        for rate in args.rates:
            mix = dict(grids=tuple(args.serve_grids), weights=tuple(args.serve_weights), steps=tuple(args.serve_steps),
                       iters=args.serve_iters)

            def fresh_jobs():
                return workloads.serving_jobs(api, torch, args.serve_jobs, rate, seed=7, **mix)

            free = torch.cuda.mem_get_info()[0]
            budget = int(0.6 * free)

            def size_pools(grids, mem):
                """One pool per grid size, `co_slots` member slots each: full
                trajectory storage when every pool's fits in `mem`, else an
                equal share each, checkpointed where full storage does not fit."""
                nmax = args.serve_steps[1] // 10 * 10
                full = {n: serve.CoBatchServer.pool_bytes(n, nmax, 32, 10, 0, args.co_slots) for n in grids}
                out = {}
                for n in grids:
                    ck = 0
                    if sum(full.values()) > mem and full[n] > mem // len(grids):
                        ck = next((K for K in range(nmax, 0, -1)
                                   if serve.CoBatchServer.pool_bytes(n, nmax, 32, 10, K, args.co_slots)
                                   <= mem // len(grids)), 1)
                    out[n] = dict(slots=args.co_slots, nsteps=nmax, px=32, dt=dts[n], ckpt_every=ck)
                return out

            pools = size_pools(args.serve_grids, budget)
            co = serve.CoBatchServer(pools, plan=None)
            out_co = co.run(fresh_jobs())
            co.close()
            torch.cuda.empty_cache()
            out = serve.Server(serve.CudaExecutor(), memory_budget=budget, slots=args.slots,
                               job_cap=int(budget / args.slots)).run(fresh_jobs())
            base = serve.Server(serve.CudaExecutor(), memory_budget=budget, slots=1,
                                job_cap=int(budget / args.slots)).run(fresh_jobs())
            # hybrid: grids up to 256^2 co-batched in pools, larger ones as their own contexts
            small = [n for n in args.serve_grids if n <= 256]
            big_budget = budget // 2
            hy_pools = size_pools(small, budget - big_budget)
            hy = serve.HybridServer(hy_pools, big_budget=big_budget, big_slots=2, plan=None)
            out_hy = hy.run(fresh_jobs())
            hy.close()
            torch.cuda.empty_cache()
            summary[str(rate)] = {"co_batched": out_co, "hybrid": out_hy, "stream_overlap": out,
                                  "one_job_at_a_time": base, "pools": {str(n): p for n, p in pools.items()},
                                  "hybrid_pools": {str(n): p for n, p in hy_pools.items()}}
        line.update({"metric": "served solves/s, p50/p99 latency", "rates": summary,
                     "config": {"jobs": args.serve_jobs, "slots": args.slots, "co_slots": args.co_slots,
                                "grids": args.serve_grids,
                                "grid_weights": args.serve_weights, "horizon_steps": args.serve_steps,
                                "lbfgs_iters": args.serve_iters}})
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--window-steps", type=int, default=W["nsteps"],
                    help="shorter window (multiple of 20) for profiling runs; the default is the workload's 2000")
    ap.add_argument("--spinup-steps", type=int, default=W["spinup_steps"])
    ap.add_argument("--roofline-class", default=None, choices=["fwd_rows", "fwd_cols", "adj_rows", "adj_cols"])
    ap.add_argument("--roofline-evals", type=int, default=1)
    ap.add_argument("--no-graphs", dest="graphs", action="store_false")
    ap.add_argument("--tune-steps", type=int, default=8, help="RK steps per plan variant in the autotuner (0: off)")
    ap.add_argument("--plan", type=int, default=None,
                    help="sweep, plain: a fixed FFT plan variant instead of the autotuner's choice "
                         "(e.g. under a profiler)")
    ap.add_argument("--probe-iters", type=int, default=100000, help="fp64peak: loop rounds per thread")
    ap.add_argument("--assim-iters", type=int, default=None,
                    help="plain / sweep-assim: L-BFGS iterations (defaults 10 and 100)")
    ap.add_argument("--workload", default="sweep", choices=["sweep", "ensemble", "autograd", "serve", "grids",
                                                            "fp64peak", "plain", "sweep-assim"],
                    help="sweep: the headline workload above; the others print their own line")
    ap.add_argument("--ens256", type=int, default=256)
    ap.add_argument("--ens512", type=int, default=64)
    ap.add_argument("--ens-steps", type=int, default=1000)
    ap.add_argument("--ens-ckpt", type=int, default=25)
    ap.add_argument("--ag-n", type=int, default=512)
    ap.add_argument("--ag-steps", type=int, default=4000)
    ap.add_argument("--ag-dirs", type=int, default=20)
    ap.add_argument("--rates", type=float, nargs="+", default=[2.0, 10.0])
    ap.add_argument("--serve-jobs", type=int, default=16)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--co-slots", type=int, default=8, help="member slots per grid-size pool of the co-batched server")
    # job mix; the defaults are a scaled-down mix that a run finishes in
    # minutes, the full one is --serve-grids 128 256 512 1024
    # --serve-weights 0.4 0.3 0.2 0.1 --serve-steps 500 4000 --serve-iters 30
    ap.add_argument("--serve-grids", type=int, nargs="+", default=[128, 256, 512])
    ap.add_argument("--serve-weights", type=float, nargs="+", default=[0.5, 0.35, 0.15])
    ap.add_argument("--serve-steps", type=int, nargs=2, default=[200, 600])
    ap.add_argument("--serve-iters", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-plain", dest="plain", action="store_false")
    args = ap.parse_args()
    if args.window_steps % W["every"]:
        ap.error("--window-steps must be a multiple of 20")
    W["nsteps"] = args.window_steps
    W["spinup_steps"] = args.spinup_steps
    if args.assim_iters is None:
        args.assim_iters = 10 if args.workload == "plain" else 100
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "sweep":
        run_workload(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
