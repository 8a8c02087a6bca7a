"""Shared problem definitions: the same numbers build an oracle Problem and a
CUDA-path Config, and the seeded inputs come from the synthetic module."""
from __future__ import annotations

import numpy as np

from paper_2602_14016_gb300 import synthetic


def make_pair(orc, n, nsteps, dt, nu, kernels=(("identity", 0.0),), forcing="none", amp=1.0, nf=4, px=8, every=5,
              include_t0=False):
    """Returns (list of oracle Problems, one per member, CUDA Config)."""
    from paper_2602_14016_gb300.api import Config, KernelSpec

    probs = [orc.Problem(n=n, nsteps=nsteps, dt=dt, nu=nu, forcing=forcing, amp=amp, nf=nf, px=px, every=every,
                         include_t0=include_t0, kernel=k, kparam=a) for k, a in kernels]
    cfg = Config(n=n, nsteps=nsteps, dt=dt, nu=nu, forcing=forcing, amp=amp, nf=nf, px=px, every=every,
                 include_t0=include_t0, kernels=[KernelSpec(k, a) for k, a in kernels])
    return probs, cfg


def truth_and_guess(orc, prob, seed_truth, seed_guess, scale=1.0):
    """Controls of a seeded truth field and of a seeded first guess (oracle maps)."""
    n = prob.n
    truth = orc.control_from_omega(prob, synthetic.random_vorticity_hat(n, seed_truth) * scale)
    guess = orc.control_from_omega(prob, synthetic.random_vorticity_hat(n, seed_guess) * scale)
    return truth, guess


def noisy_observations(obs: np.ndarray, seed: int, level: float = 0.01) -> np.ndarray:
    """obs + level * RMS(obs) * N(0, 1) draws (1 % noise reading)."""
    rms = float(np.sqrt(np.mean(obs**2)))
    return obs + level * rms * synthetic.gaussian_draws(obs.shape, seed)


def kolmogorov256_oracle_member(args):
    """Oracle cost, gradient and compact lambda_0 of one member of the 256^2
    Kolmogorov window (spawned worker: imports only the oracle and numpy)."""
    import oracle

    nsteps, kernel, kp, m, seed_guess = args
    n = 256
    P = oracle.Problem(n=n, nsteps=nsteps, dt=2e-3, nu=1e-2, forcing="kolmogorov", amp=1.0, nf=4, px=16, every=20,
                       kernel=kernel, kparam=kp)
    s = oracle.control_from_omega(P, synthetic.random_vorticity_hat(n, seed_guess))
    J, g, lam0 = oracle.cost_grad(P, s, m)
    K = (n - 1) // 3
    rows = list(range(0, K + 1)) + list(range(n - K, n))
    return J, g, lam0[rows, : K + 1]
