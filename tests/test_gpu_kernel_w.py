"""The CUDA path's control multiplier and gradient, element by element.

- k_make_mult (the CUDA multiplier |k| W^{1/2}, Eq. 18-19) against the exact
  values that special parameters fix (the same values that pin the oracle
  in test_oracle_kernel_w.py), through single Fourier modes;
- the table kernel (DA_KERNEL_TABLE) against the oracle;
- the gradient of the sweep's most skewed members, exp(-|k|) and
  |k|^{-3}, compared element-wise (max-abs error over max-abs value) and per
  wavenumber shell k <= |k| < k + 1, not only in relative L2.  The adjoint
  lambda_0 is compared per shell on every shell; g_s = IDFT(m lambda_0_hat)
  per shell where the shell holds at least 1e-6 of the largest shell's norm
  (below that, the rounding of g_s's own grid values, about 1e-16 of its
  norm, exceeds 1e-10 of the shell).
"""
import math

import numpy as np
import pytest

from cases import make_pair, noisy_observations, truth_and_guess
from conftest import rel
from paper_2602_14016_gb300 import synthetic
from test_oracle_kernel_w import EXACT

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GRAD_TOL = 1e-8
SHELL_TOL = 1e-8


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a GPU")
    from paper_2602_14016_gb300 import api as A, build

    build.build()
    return A


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _grid(n):
    return np.meshgrid(2 * np.pi * np.arange(n) / n, 2 * np.pi * np.arange(n) / n, indexing="ij")


def gpu_mode_multipliers(api, n, kernel, kp, nu, modes, table=None):
    cfg = api.Config(n=n, nsteps=1, dt=1e-3, nu=nu, px=4, every=1,
                     kernels=[api.KernelSpec(kernel, kp, table)] * len(modes), store=False)
    ctx = api.Context(cfg)
    y, x = _grid(n)
    s = np.stack([np.cos(kx * x + ky * y) for kx, ky in modes])
    w0 = ctx.omega_from_control(cu(s)).cpu().numpy()
    ctx.close()
    out = []
    for b, (kx, ky) in enumerate(modes):
        q = ky % n
        out.append((w0[b, q, kx] / np.fft.rfft2(s[b])[q, kx]).real)
    return out


@pytest.mark.parametrize("kernel,kp,nu,cases", EXACT, ids=[f"{e[0]}:{e[1]:.3g}:nu{e[2]:g}" for e in EXACT])
def test_gpu_multiplier_exact_values(api, kernel, kp, nu, cases):
    got = gpu_mode_multipliers(api, 16, kernel, kp, nu, [(kx, ky) for kx, ky, _ in cases])
    for (kx, ky, m), g in zip(cases, got):
        assert abs(g - m) <= 1e-14 * m, (kernel, kp, kx, ky, g, m)


def test_gpu_table_multiplier_exact_values(api):
    n = 16
    KX, KY = synthetic.wavenumbers(n)
    table = 4.0 ** (-np.abs(KX)) * 9.0 ** (-np.abs(KY))
    cases = [(1, 0, 0.5), (0, 1, 1 / 3), (3, 4, 5 / 648), (4, -3, 5 / 432), (2, 5, math.sqrt(29) / (4 * 243))]
    got = gpu_mode_multipliers(api, n, "table", 0.0, 1e-2, [(kx, ky) for kx, ky, _ in cases], table)
    for (kx, ky, m), g in zip(cases, got):
        assert abs(g - m) <= 1e-14 * m, (kx, ky, g, m)


def shell_index(n):
    KX, KY = synthetic.wavenumbers(n)
    k = np.sqrt(KX**2 + KY**2)
    return np.floor(k).astype(int), synthetic.retained_mask(n) & (k > 0)


def per_shell_rel(a, b, n, floor=0.0):
    """Relative error per shell of two half spectra, over shells whose norm
    in b is at least `floor` times the largest shell norm."""
    sh, R = shell_index(n)
    norms, errs = [], []
    for s in range(1, sh[R].max() + 1):
        sel = R & (sh == s)
        norms.append(np.linalg.norm(b[sel]))
        errs.append(np.linalg.norm(a[sel] - b[sel]))
    norms, errs = np.array(norms), np.array(errs)
    keep = norms >= floor * norms.max()
    return np.max(errs[keep] / norms[keep]), int(keep.sum())


def max_abs_rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


ELEMENTWISE = [
    dict(n=64, nsteps=60, dt=4e-3, nu=1e-3, kernels=[("exp_abs", 1.0)], px=8, every=10),
    dict(n=64, nsteps=60, dt=4e-3, nu=1e-2, kernels=[("frac", 1.5)], forcing="kolmogorov", nf=4, px=8, every=20),
    dict(n=128, nsteps=20, dt=4e-3, nu=1e-3, kernels=[("exp_abs", 1.0)], px=16, every=10),
    dict(n=128, nsteps=20, dt=4e-3, nu=1e-2, kernels=[("frac", 1.5)], forcing="kolmogorov", nf=4, px=16, every=10),
    dict(n=32, nsteps=20, dt=5e-3, nu=1e-3, kernels=[("table", 0.0)], px=8, every=5),
]


@pytest.mark.parametrize("case", ELEMENTWISE, ids=[f"n{c['n']}-{c['kernels'][0][0]}{c['kernels'][0][1]}" for c in ELEMENTWISE])
def test_gradient_elementwise_and_per_shell(orc, api, case):
    case = dict(case)
    n = case["n"]
    table = None
    if case["kernels"][0][0] == "table":
        KX, KY = synthetic.wavenumbers(n)
        table = (1.0 + 0.5 * np.cos(KX) + 0.25 * np.sin(KY) ** 2) / (1.0 + KX**2 + 2.0 * KY**2)
    probs, cfg = make_pair(orc, **case)
    P = probs[0]
    if table is not None:
        P.ktable = table
        cfg.kernels[0].table = table
    ctx = api.Context(cfg)
    truth, guess = truth_and_guess(orc, P, 5, 6, scale=2.0)
    _, m = orc.forward(P, truth)
    m = noisy_observations(m, 7)
    J, g, lam0 = orc.cost_grad(P, guess, m)
    ctx.set_observations(cu(m[None]))
    Jg, gg = ctx.cost_grad(cu(guess[None]))
    gg = gg.cpu().numpy()[0]
    l0, _ = ctx.last_adjoint()
    l0 = l0.cpu().numpy()[0]
    assert abs(Jg.item() - J) <= 1e-12 * J
    assert rel(gg, g) < GRAD_TOL
    assert max_abs_rel(gg, g) < GRAD_TOL
    e_lam, _ = per_shell_rel(l0, lam0, n)
    assert e_lam < SHELL_TOL, e_lam
    e_g, kept = per_shell_rel(np.fft.rfft2(gg), np.fft.rfft2(g), n, floor=1e-6)
    assert kept >= 10 and e_g < SHELL_TOL, (e_g, kept)
    ctx.close()
