"""Oracle parity over the full horizon of the headline window: 256^2
Kolmogorov flow, 2000 RK4 steps of 2e-3, 16 x 16 probes every 20 steps,
the seven-kernel sweep as one batch with CUDA-graph replay (as bench.py runs
it).

- test_full_window_against_the_oracle: the cost, the gradient and the adjoint
  lambda_0 of members |k|^{-1} and exp(-|k|) against the oracle's values in
  tests/golden/kolmogorov256_window2000.npz (written by
  make_kolmogorov256_window.py, oracle only): J to 1e-12, g_s to 1e-8 in
  relative L2 and in max-abs over max-abs, lambda_0 to 1e-8 per wavenumber
  shell.
- test_200_steps_against_the_live_oracle: the first 200 steps of the same
  window, the oracle run on this machine's host cores (spawned processes)
  for members |k|^{-3} and exp(-|k|), compared the same way.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

import cases
from conftest import rel
from paper_2602_14016_gb300 import synthetic

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "kolmogorov256_window2000.npz")
SWEEP = [("frac", 0.0), ("frac", 0.5), ("frac", 1.0), ("frac", 1.5), ("exp_abs", 0.1), ("exp_abs", 0.3),
         ("exp_abs", 1.0)]
N, DT, NU, PX, EVERY = 256, 2e-3, 1e-2, 16, 20
SEED_GUESS = 2


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a GPU")
    from paper_2602_14016_gb300 import api as A, build

    build.build()
    return A


def oracle_problem(orc, nsteps, kernel, kp):
    return orc.Problem(n=N, nsteps=nsteps, dt=DT, nu=NU, forcing="kolmogorov", amp=1.0, nf=4, px=PX, every=EVERY,
                       kernel=kernel, kparam=kp)


def compact(h):
    K = (N - 1) // 3
    rows = list(range(0, K + 1)) + list(range(N - K, N))
    return h[rows, : K + 1]


def shell_errors(a_c, b_c):
    """Relative error per shell k <= |k| < k+1 of two compact spectra."""
    K = (N - 1) // 3
    ky = np.array(list(range(0, K + 1)) + list(range(-K, 0)))[:, None]
    kx = np.arange(K + 1)[None, :]
    k = np.sqrt(kx**2 + ky**2)
    sh = np.floor(k).astype(int)
    out = []
    for s in range(1, sh.max() + 1):
        sel = (sh == s) & (k > 0)
        out.append(np.linalg.norm(a_c[sel] - b_c[sel]) / np.linalg.norm(b_c[sel]))
    return np.array(out)


def run_gpu_sweep(api, orc, nsteps, m):
    cfg = api.Config(n=N, nsteps=nsteps, dt=DT, nu=NU, forcing="kolmogorov", nf=4, px=PX, every=EVERY,
                     kernels=[api.KernelSpec(*k) for k in SWEEP])
    ctx = api.Context(cfg)
    ctx.set_graphs(True)
    w_guess = synthetic.random_vorticity_hat(N, SEED_GUESS)
    s = np.stack([orc.control_from_omega(oracle_problem(orc, nsteps, *k), w_guess) for k in SWEEP])
    ctx.set_observations(torch.from_numpy(np.repeat(m[None], len(SWEEP), 0)).cuda())
    ctx.cost_grad(torch.from_numpy(s).cuda())  # first call captures the graph
    J, g = ctx.cost_grad(torch.from_numpy(s).cuda())  # replay
    lam0, _ = ctx.last_adjoint()
    torch.cuda.synchronize()
    out = (J.cpu().numpy(), g.cpu().numpy(), lam0.cpu().numpy())
    ctx.close()
    return out


def check_member(J, g, lam0_half, Jr, gr, lam0c_r, label):
    errs = {"J": abs(J - Jr) / Jr, "g_rel_l2": rel(g, gr),
            "g_max_abs": float(np.max(np.abs(g - gr)) / np.max(np.abs(gr))),
            "lam0_worst_shell": float(np.max(shell_errors(compact(lam0_half), lam0c_r)))}
    print(f"{label}: " + ", ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    assert errs["J"] <= 1e-12, errs
    assert errs["g_rel_l2"] < 1e-8 and errs["g_max_abs"] < 1e-8, errs
    assert errs["lam0_worst_shell"] < 1e-8, errs


def test_full_window_against_the_oracle(orc, api):
    z = np.load(GOLDEN)
    nsteps = int(z["nsteps"])
    assert nsteps == 2000
    members = [str(x) for x in z["members"]]
    J, g, lam0 = run_gpu_sweep(api, orc, nsteps, z["m"])
    for i, name in enumerate(members):
        k, a = name.split(":")
        b = SWEEP.index((k, float(a)))
        check_member(J[b], g[b], lam0[b], float(z[f"J{i}"]), z[f"g{i}"], z[f"lam0c{i}"], f"{name} 2000 steps")


def test_200_steps_against_the_live_oracle(orc, api):
    nsteps = 200
    m = np.load(GOLDEN)["m"][: nsteps // EVERY].copy()
    members = [("frac", 1.5), ("exp_abs", 1.0)]
    with mp.get_context("spawn").Pool(len(members)) as pool:
        ref = pool.map(cases.kolmogorov256_oracle_member, [(nsteps, k, a, m, SEED_GUESS) for k, a in members])
    J, g, lam0 = run_gpu_sweep(api, orc, nsteps, m)
    for (k, a), (Jr, gr, lr) in zip(members, ref):
        b = SWEEP.index((k, a))
        check_member(J[b], g[b], lam0[b], Jr, gr, lr, f"{k}:{a} 200 steps")
