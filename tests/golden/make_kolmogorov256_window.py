"""Writes tests/golden/kolmogorov256_window<nsteps>.npz: the oracle's cost,
gradient and adjoint for the forced Kolmogorov window of the headline
workload (256^2, nu = 1/100, f = (sin 4y, 0), RK4 with dt = 2e-3,
16 x 16 velocity probes every 20 steps with 1 % Gaussian noise) over the
full 2000-step horizon, for two members of the kernel sweep of Sec. III.B:
|k|^{-1} (frac 0.5) and exp(-|k|) (exp_abs 1).

Everything here comes from the oracle (oracle/) and the seeded input
generators (paper_2602_14016_gb300.synthetic), nothing from the CUDA path:
- truth: the seeded unit-energy random-phase field (seed 0), not spun up
  (a 25,000-step spin-up takes the oracle over an hour);
- observations: the oracle's forward solve of the truth plus 1 % noise
  (sigma = 0.01 x RMS of the clean samples, seeded draws, seed 1);
- point of evaluation: the control of a second seeded field (seed 2) under
  each member's kernel (oracle control map, recomputed by the test);
- stored: the noisy observations, and per member J, the gradient g_s on the
  grid and the adjoint lambda_0 on the retained set (compact [Kr][Kc]).

Run: python tests/golden/make_kolmogorov256_window.py [--nsteps 2000]
(about 35 minutes on a few cores: one forward solve, then the members'
cost-and-gradient evaluations in parallel processes).
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

N, DT, NU, AMP, NF, PX, EVERY = 256, 2e-3, 1e-2, 1.0, 4, 16, 20
MEMBERS = [("frac", 0.5), ("exp_abs", 1.0)]
SEED_TRUTH, SEED_NOISE, SEED_GUESS = 0, 1, 2


def problem(nsteps, kernel="identity", kparam=0.0):
    import oracle

    return oracle.Problem(n=N, nsteps=nsteps, dt=DT, nu=NU, forcing="kolmogorov", amp=AMP, nf=NF, px=PX, every=EVERY,
                          kernel=kernel, kparam=kparam)


def compact(h):
    """Retained set of a half spectrum, [Kr][Kc] with rows ky = 0..K, -K..-1."""
    K = (N - 1) // 3
    rows = list(range(0, K + 1)) + list(range(N - K, N))
    return h[rows, : K + 1]


def member_job(args):
    nsteps, kernel, kp, m = args
    import oracle
    from paper_2602_14016_gb300 import synthetic

    P = problem(nsteps, kernel, kp)
    s = oracle.control_from_omega(P, synthetic.random_vorticity_hat(N, SEED_GUESS))
    t0 = time.time()
    J, g, lam0 = oracle.cost_grad(P, s, m)
    return kernel, kp, J, g, compact(lam0), time.time() - t0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nsteps", type=int, default=2000)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    import oracle
    from paper_2602_14016_gb300 import synthetic

    oracle.build()
    t0 = time.time()
    P = problem(args.nsteps)
    s_truth = oracle.control_from_omega(P, synthetic.random_vorticity_hat(N, SEED_TRUTH))
    _, obs = oracle.forward(P, s_truth)
    rms = float(np.sqrt(np.mean(obs**2)))
    m = obs + 0.01 * rms * synthetic.gaussian_draws(obs.shape, SEED_NOISE)
    print(f"truth forward: {time.time() - t0:.0f} s", flush=True)
    with mp.get_context("spawn").Pool(len(MEMBERS)) as pool:
        res = pool.map(member_job, [(args.nsteps, k, a, m) for k, a in MEMBERS])
    out = {"m": m, "nsteps": args.nsteps, "members": np.array([f"{k}:{a}" for k, a in MEMBERS])}
    for i, (k, a, J, g, lam0c, secs) in enumerate(res):
        out[f"J{i}"] = np.float64(J)
        out[f"g{i}"] = g
        out[f"lam0c{i}"] = lam0c
        print(f"{k}:{a} J = {J:.16e}  ({secs:.0f} s)", flush=True)
    path = args.out or os.path.join(HERE, f"kolmogorov256_window{args.nsteps}.npz")
    np.savez(path, **out)
    print(f"wrote {path}", flush=True)


if __name__ == "__main__":
    main()
