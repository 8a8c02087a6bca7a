"""Serving assimilation jobs with continuous batching.

Jobs (each a grid, window, probe set, kernel, observations, first guess and
an L-BFGS iteration budget) arrive over time.  The server admits a job as
soon as a worker slot is idle and the job's device memory fits the free
budget; the job's trajectory storage is sized first (full stage fields, or
checkpoints every K steps when the full window would exceed the per-job
cap), so admission is by checkpoint memory.  Every slot runs its job on its
own CUDA stream, so the kernels of concurrent jobs overlap on the device:
a job that arrives while others run starts as soon as memory and a slot
free up, without waiting for a batch boundary.  Each job's result does not
depend on what else runs (own context, deterministic kernels).

`CoBatchServer` goes further and shares launches between jobs: per grid size
one pool context holds a fixed number of member slots (a ragged batch, its
memory allocated once); a job of that grid takes a free slot between two
optimiser steps of the pool and leaves it when it finishes, and every step is
one cost-and-gradient evaluation shared by all the pool's jobs, whatever
point of their iterations they are at, so their forward and adjoint sweeps
run in the same launches (da_set_member, da_lbfgs_*).

Reports per job: arrival, admission and completion times; overall:
solves/s, p50/p99 latency.  `FakeExecutor` replaces the GPU for tests of
the admission and accounting logic on the CPU.
"""
from __future__ import annotations

import dataclasses
import heapq
import threading
import time
from typing import Callable, Optional

import numpy as np


@dataclasses.dataclass
class Job:
    job_id: int
    n: int
    nsteps: int
    dt: float
    nu: float
    px: int
    every: int
    kernel: tuple = ("identity", 0.0)
    forcing: str = "none"
    nf: int = 4
    iters: int = 30
    arrival: float = 0.0  # seconds after the start of the run
    m: Optional[np.ndarray] = None  # observations [1, nt, px*px, 2]
    s0: Optional[np.ndarray] = None  # first guess [1, n, n]
    # filled by the server
    ckpt_every: int = 0
    bytes: int = 0
    t_admit: float = float("nan")
    t_done: float = float("nan")
    J_hist: Optional[np.ndarray] = None
    iters_done: int = 0
    status: int = -1  # DA_OK, DA_ENOTCONV (stopped on a line-search failure), or a failure status
    error: str = ""
    s: Optional[np.ndarray] = None

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival

    @property
    def nt(self) -> int:
        return self.nsteps // self.every


def context_bytes(n: int, nsteps: int, px: int, every: int, ckpt_every: int, batch: int = 1, memory: int = 10) -> int:
    """Device bytes of a context plus its optimiser buffers (mirrors da_create
    and da_assimilate's allocations)."""
    K = (n - 1) // 3
    Kc, Kr = K + 1, 2 * K + 1
    nt = nsteps // every
    comp = batch * Kr * Kc * 16
    b = 6 * comp + batch * 4 * n * Kc * 16 + 3 * batch * nt * px * px * 2 * 8 + comp // 2
    b += n * 16 + 64 * 16 + batch * (8 + 4 + 8) + batch * 8 + Kr * Kc * 72 + batch * (4 * 4 + 8)
    if ckpt_every == 0:
        b += batch * nsteps * 8 * n * n * 8
    else:
        kk = min(ckpt_every, nsteps)
        b += batch * kk * 8 * n * n * 8 + ((nsteps + kk - 1) // kk) * comp
    slots = memory + 1
    # optimiser: vector banks, device scalars and costs, argument tables
    b += batch * (5 + 2 * slots) * n * n * 8 + batch * 7 * 8 + (3 * batch + batch * memory) * 4
    b += (batch + batch * memory) * 8
    return int(b)


def plan_storage(job: Job, job_cap_bytes: int) -> None:
    """Full stage-field storage if it fits the per-job cap, else the largest
    checkpoint interval (a divisor-free K, last segment shorter) that fits."""
    full = context_bytes(job.n, job.nsteps, job.px, job.every, 0)
    if full <= job_cap_bytes:
        job.ckpt_every, job.bytes = 0, full
        return
    for K in range(job.nsteps, 0, -1):
        b = context_bytes(job.n, job.nsteps, job.px, job.every, K)
        if b <= job_cap_bytes:
            job.ckpt_every, job.bytes = K, b
            return
    job.ckpt_every, job.bytes = 1, context_bytes(job.n, job.nsteps, job.px, job.every, 1)


class CudaExecutor:
    """Runs a job through the C ABI on the slot's stream."""

    def __init__(self, device: int = 0):
        import torch

        self.torch = torch
        self.device = device
        self.streams = {}

    def run(self, job: Job, slot: int) -> None:
        torch = self.torch
        from . import api

        if slot not in self.streams:
            with torch.cuda.device(self.device):
                self.streams[slot] = torch.cuda.Stream()
        st = self.streams[slot]
        cfg = api.Config(n=job.n, nsteps=job.nsteps, dt=job.dt, nu=job.nu, forcing=job.forcing, nf=job.nf,
                         px=job.px, every=job.every, kernels=[api.KernelSpec(*job.kernel)],
                         ckpt_every=job.ckpt_every)
        from . import _native

        with torch.cuda.device(self.device), torch.cuda.stream(st):
            ctx = None
            try:
                ctx = api.Context(cfg, self.device)
                ctx.set_observations(torch.from_numpy(job.m).to(ctx.device), stream=st)
                s = torch.from_numpy(job.s0).to(ctx.device).contiguous()
                res = ctx.assimilate(s, job.iters, stream=st)
                st.synchronize()
                job.J_hist, job.iters_done, job.status = res.J_hist[0], int(res.iters[0]), int(res.member_status[0])
                job.s = s.cpu().numpy()
            except _native.DAError as e:  # a failed job is recorded, not lost with its worker thread
                job.status, job.error = e.status, str(e)
            finally:
                if ctx is not None:
                    ctx.close()


class FakeExecutor:
    """Stands in for the GPU: a job takes `seconds(job)` of wall time."""

    def __init__(self, seconds: Callable[[Job], float]):
        self.seconds = seconds

    def run(self, job: Job, slot: int) -> None:
        time.sleep(self.seconds(job))
        job.status, job.iters_done = 0, job.iters
        job.J_hist = np.zeros(job.iters + 1)


class Server:
    """Admission by memory, one job per slot at a time, slots run concurrently."""

    def __init__(self, executor, memory_budget: int, slots: int = 4, job_cap: Optional[int] = None):
        self.executor = executor
        self.budget = int(memory_budget)
        self.slots = slots
        self.job_cap = int(job_cap) if job_cap else int(memory_budget)
        self._lock = threading.Condition()
        self._free_bytes = self.budget
        self._idle = list(range(slots))
        self._queue: list = []
        self._running = 0
        self.peak_bytes = 0
        self.peak_running = 0

    def _admit_locked(self, now: float, t0: float):
        """First-fit over the queue in arrival order."""
        started = []
        i = 0
        while i < len(self._queue) and self._idle:
            job = self._queue[i]
            if job.bytes <= self._free_bytes:
                self._queue.pop(i)
                slot = self._idle.pop(0)
                self._free_bytes -= job.bytes
                self._running += 1
                self.peak_bytes = max(self.peak_bytes, self.budget - self._free_bytes)
                self.peak_running = max(self.peak_running, self._running)
                job.t_admit = now - t0
                started.append((job, slot))
            else:
                i += 1
        return started

    def run(self, jobs: list) -> dict:
        """Replays the jobs' arrival times; returns the summary."""
        for j in jobs:
            plan_storage(j, self.job_cap)
            if j.bytes > self.budget:
                raise ValueError(f"job {j.job_id} needs {j.bytes} bytes, more than the budget")
        pending = sorted(jobs, key=lambda j: j.arrival)
        t0 = time.perf_counter()
        threads = []

        def work(job, slot):
            try:
                self.executor.run(job, slot)
            finally:
                with self._lock:
                    job.t_done = time.perf_counter() - t0
                    self._free_bytes += job.bytes
                    self._idle.append(slot)
                    self._idle.sort()
                    self._running -= 1
                    self._lock.notify_all()

        k = 0
        while k < len(pending) or self._queue or self._running:
            with self._lock:
                now = time.perf_counter()
                while k < len(pending) and pending[k].arrival <= now - t0:
                    self._queue.append(pending[k])
                    k += 1
                for job, slot in self._admit_locked(now, t0):
                    th = threading.Thread(target=work, args=(job, slot), daemon=True)
                    th.start()
                    threads.append(th)
                if k >= len(pending) and not self._queue and not self._running:
                    break
                wait = None
                if k < len(pending):
                    wait = max(0.0, pending[k].arrival - (time.perf_counter() - t0))
                self._lock.wait(timeout=wait if wait is not None else 0.5)
        for th in threads:
            th.join()
        makespan = max(j.t_done for j in jobs) - min(j.arrival for j in jobs)
        lat = np.array([j.latency for j in jobs])
        # a solve returns a control: converged, out of iterations, or stopped by
        # the line search (DA_ENOTCONV); anything else is a failed job
        solved = [j for j in jobs if j.status in (0, 6)]
        return {"jobs": len(jobs), "solves": len(solved), "failed": len(jobs) - len(solved),
                "solves_per_s": len(solved) / makespan, "makespan_s": makespan,
                "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
                "peak_bytes": self.peak_bytes, "peak_running": self.peak_running}


def poisson_arrivals(rate: float, count: int, seed: int) -> np.ndarray:
    """Arrival times of a Poisson process (seeded exponential gaps)."""
    gaps = np.random.default_rng(seed).exponential(1.0 / rate, size=count)
    return np.cumsum(gaps) - gaps[0]


def summarize(jobs: list, **extra) -> dict:
    """solves/s and p50/p99 latency of finished jobs (a solve returns a
    control: converged, out of iterations, or stopped by the line search)."""
    makespan = max(j.t_done for j in jobs) - min(j.arrival for j in jobs)
    lat = np.array([j.latency for j in jobs])
    solved = [j for j in jobs if j.status in (0, 6)]
    out = {"jobs": len(jobs), "solves": len(solved), "failed": len(jobs) - len(solved),
           "solves_per_s": len(solved) / makespan, "makespan_s": makespan,
           "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99))}
    out.update(extra)
    return out


class CoBatchServer:
    """Continuous batching in shared launches.

    pools: {n: dict(slots=S, nsteps=max horizon, px=max probes per side,
    dt=..., ckpt_every=K)} -- one pool context per grid size, created once
    (forcing available, members switch it on or off).  Each pool runs on its
    own host thread and CUDA stream: between steps it admits the arrived jobs
    of its grid into free slots (their windows, kernels, observations and
    first guesses), runs one step (da_lbfgs_iterate: one evaluation shared by
    every member, whatever point of its iteration it is at), and retires the
    members that finished.
    Plan variant `plan` on every pool, so a job's result equals its result in
    a batch-1 context on that variant; plan=None lets the autotuner pick each
    pool's variant for its slot count (results then equal the batch-1 ones to
    rounding)."""

    def __init__(self, pools: dict, device: int = 0, graphs: bool = True, plan: Optional[int] = 0, every: int = 10):
        import torch

        from . import api

        self.torch, self.api = torch, api
        self.device = device
        self.pools = {}
        self.every = every
        for n, p in pools.items():
            cfg = api.Config(n=n, nsteps=p["nsteps"], dt=p["dt"], nu=1e-3, forcing="kolmogorov", nf=4,
                             px=p["px"], every=every, kernels=[api.KernelSpec("identity", 0.0)] * p["slots"],
                             ckpt_every=p.get("ckpt_every", 0))
            with torch.cuda.device(device):
                ctx = api.Context(cfg, device)
                if plan is None:
                    ctx.autotune(4)
                else:
                    ctx.set_plan(plan)
                if graphs:
                    ctx.set_graphs(True)
                for b in range(p["slots"]):
                    ctx.set_member(b, 0)
                self.pools[n] = {"ctx": ctx, "slots": p["slots"], "stream": torch.cuda.Stream(device),
                                 "jobs": [None] * p["slots"], "steps": 0}
        self.peak_members = 0

    @staticmethod
    def pool_bytes(n: int, nsteps: int, px: int, every: int, ckpt_every: int, slots: int) -> int:
        return context_bytes(n, nsteps, px, every, ckpt_every, batch=slots)

    def _pool_loop(self, n, pool, queue, lock, t0, errors):
        torch, api = self.torch, self.api
        ctx, st = pool["ctx"], pool["stream"]
        slots = pool["jobs"]
        try:
            with torch.cuda.device(self.device), torch.cuda.stream(st):
                while True:
                    now = time.perf_counter() - t0
                    with lock:
                        arrived = [j for j in queue if j.arrival <= now]
                        for j in arrived:
                            if None not in slots:
                                break
                            b = slots.index(None)
                            queue.remove(j)
                            slots[b] = j
                            j.t_admit = now
                            kern = api.KernelSpec(*j.kernel)
                            ctx.set_member(b, j.nsteps, j.px, j.nu, j.forcing == "kolmogorov", kern,
                                           torch.from_numpy(j.m[0]), stream=st)
                            ctx.lbfgs_start(b, torch.from_numpy(j.s0[0]).to(ctx.device), j.iters, stream=st)
                        busy = sum(x is not None for x in slots)
                        self.peak_members = max(self.peak_members, busy)
                        remaining = len(queue)
                    if busy == 0:
                        if remaining == 0:
                            return
                        nxt = min(j.arrival for j in queue)
                        time.sleep(max(0.0, min(0.05, nxt - (time.perf_counter() - t0))))
                        continue
                    ctx.lbfgs_iterate(stream=st)
                    pool["steps"] += 1
                    for b, j in enumerate(slots):
                        if j is None:
                            continue
                        rep, hist, s = ctx.lbfgs_member(b, j.iters + 1, control=True, stream=st)
                        if rep["phase"] != 3:
                            continue
                        st.synchronize()
                        j.J_hist, j.iters_done, j.status = hist, rep["iters"], rep["status"]
                        j.s = s.cpu().numpy()[None]
                        j.t_done = time.perf_counter() - t0
                        ctx.lbfgs_release(b)
                        ctx.set_member(b, 0, stream=st)
                        slots[b] = None
        except Exception as e:  # recorded; the run reports it
            errors.append((n, repr(e)))

    def run(self, jobs: list) -> dict:
        for j in jobs:
            if j.n not in self.pools:
                raise ValueError(f"job {j.job_id}: no pool for grid {j.n}")
            if j.every != self.every:
                raise ValueError(f"job {j.job_id}: observation interval {j.every} != the pools' {self.every}")
        lock = threading.Lock()
        t0 = time.perf_counter()
        errors = []
        threads = []
        for n, pool in self.pools.items():
            queue = sorted([j for j in jobs if j.n == n], key=lambda j: j.arrival)
            th = threading.Thread(target=self._pool_loop, args=(n, pool, queue, lock, t0, errors), daemon=True)
            th.start()
            threads.append(th)
        for th in threads:
            th.join()
        if errors:
            raise RuntimeError(f"pool failures: {errors}")
        return summarize(jobs, peak_members=self.peak_members,
                         steps={int(n): p["steps"] for n, p in self.pools.items()})

    def close(self):
        for p in self.pools.values():
            p["ctx"].close()


class HybridServer:
    """Co-batching where it pays, own contexts where it does not.

    A grid small enough that one member leaves most of the GPU idle gains
    from sharing launches (CoBatchServer pools); a large grid fills the GPU
    with one member, and its jobs run best as their own contexts overlapped
    on streams (Server with CudaExecutor), with full trajectory storage when
    it fits their memory cap.  Jobs are split by grid size between the two,
    which run at the same time on the same GPU, each with its own memory
    budget."""

    def __init__(self, pools: dict, big_budget: int, big_slots: int = 2, big_job_cap: Optional[int] = None,
                 device: int = 0, plan: Optional[int] = 0, every: int = 10):
        self.co = CoBatchServer(pools, device=device, plan=plan, every=every)
        self.big = Server(CudaExecutor(device), memory_budget=big_budget, slots=big_slots,
                          job_cap=big_job_cap or big_budget // max(1, big_slots))

    def run(self, jobs: list) -> dict:
        small = [j for j in jobs if j.n in self.co.pools]
        big = [j for j in jobs if j.n not in self.co.pools]
        out, errors = {}, []

        def go(name, srv, js):
            try:
                if js:
                    out[name] = srv.run(js)
            except Exception as e:  # recorded; the run reports it
                errors.append((name, repr(e)))

        th = [threading.Thread(target=go, args=("co", self.co, small)),
              threading.Thread(target=go, args=("big", self.big, big))]
        for t in th:
            t.start()
        for t in th:
            t.join()
        if errors:
            raise RuntimeError(f"server failures: {errors}")
        return summarize(jobs, co_batched_jobs=len(small), own_context_jobs=len(big))

    def close(self):
        self.co.close()
