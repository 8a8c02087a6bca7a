"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake (a dropped term, a wrong sign, a wrong index or
coefficient, a missing conjugation) in a copy of the oracle's C source,
compiles it, and checks that at least one pin of the battery below fails,
while the unmodified source passes all of them."""
import math

import numpy as np
import pytest

from conftest import dot, phys, rel
from paper_2602_14016_gb300 import synthetic
from test_oracle_kernel_w import mode_multiplier


def _grid(n):
    return np.meshgrid(2 * np.pi * np.arange(n) / n, 2 * np.pi * np.arange(n) / n, indexing="ij")


def battery(orc):
    """Returns the names of the pins that fail."""
    failed = []
    n = 16
    y, x = _grid(n)

    def check(name, fn):
        try:
            ok = bool(fn())
        except Exception:
            ok = False
        if not ok:
            failed.append(name)

    P = orc.Problem(n=n, nsteps=6, dt=2e-2, nu=5e-3, px=4, every=2, kernel="exp_abs", kparam=0.3)

    def biot_savart():
        Q = orc.Problem(n=n, nsteps=1, dt=1e-3, nu=0.0, px=n, every=1)
        w = np.cos(2 * x - 3 * y)
        o = orc.observe(Q, np.fft.rfft2(w)).reshape(n, n, 2)
        return np.abs(o[..., 0] - 3 * np.sin(2 * x - 3 * y) / 13).max() < 1e-13 and np.abs(
            o[..., 1] - 2 * np.sin(2 * x - 3 * y) / 13).max() < 1e-13

    def closed_form_advection():
        Q = orc.Problem(n=n, nsteps=1, dt=1e-3, nu=0.0, px=4, every=1)
        F = phys(orc.rhs(Q, np.fft.rfft2(np.cos(x) + np.cos(2 * y))))
        return np.abs(F - 1.5 * np.sin(x) * np.sin(2 * y)).max() < 1e-12

    def taylor_green():
        Q = orc.Problem(n=n, nsteps=1, dt=0.01, nu=0.05, px=4, every=1)
        w0 = np.cos(x) * np.cos(y)
        z = -2 * 0.05 * 0.01
        R = 1 + z + z * z / 2 + z**3 / 6 + z**4 / 24
        return np.abs(phys(orc.step(Q, np.fft.rfft2(w0))) - R * w0).max() < 1e-14

    def kolmogorov():
        Q = orc.Problem(n=n, nsteps=1, dt=0.01, nu=0.05, px=4, every=1, forcing="kolmogorov", amp=1.0, nf=3)
        w = np.fft.rfft2(-(1.0 / (0.05 * 3)) * np.cos(3 * y))
        return rel(orc.step(Q, w), w) < 1e-14

    def conservation():
        Q = orc.Problem(n=n, nsteps=1, dt=1e-3, nu=0.0, px=4, every=1)
        h = synthetic.random_vorticity_hat(n, 0)
        F = orc.rhs(Q, h)
        return abs(dot(h, F)) < 1e-12 * np.sqrt(dot(F, F) * dot(h, h))

    def rhs_dot():
        yy = synthetic.random_vorticity_hat(n, 3) * 2
        d = synthetic.random_retained_hat(n, 4)
        mu = synthetic.random_retained_hat(n, 5)
        a = dot(orc.rhs_tlm(P, yy, d), mu)
        b = dot(d, orc.rhs_adj(P, yy, mu))
        return abs(a - b) < 1e-12 * abs(a)

    def rhs_tangent():
        yy = synthetic.random_vorticity_hat(n, 1) * 3
        d = synthetic.random_retained_hat(n, 2, 0.1)
        return rel((orc.rhs(P, yy + d) - orc.rhs(P, yy - d)) / 2, orc.rhs_tlm(P, yy, d)) < 1e-12

    def step_dot():
        w = synthetic.random_vorticity_hat(n, 6) * 3
        d = synthetic.random_retained_hat(n, 7)
        lam = synthetic.random_retained_hat(n, 8)
        _, dw = orc.step_tlm(P, w, d)
        fd = (orc.step(P, w + 1e-3 * d) - orc.step(P, w - 1e-3 * d)) / 2e-3
        return rel(fd, dw) < 1e-8 and abs(dot(dw, lam) - dot(d, orc.step_adj(P, w, lam))) < 1e-11 * abs(dot(dw, lam))

    def obs_transpose():
        d = synthetic.random_retained_hat(n, 9)
        r = synthetic.gaussian_draws((16, 2), 10)
        a = float(np.sum(orc.observe(P, d) * r))
        return abs(a - dot(d, orc.observe_adj(P, r))) < 1e-12 * abs(a)

    def vorticity_control():
        Q = orc.Problem(n=n, nsteps=1, dt=1e-3, nu=0.0, px=4, every=1, kernel="frac", kparam=1.0)
        s = synthetic.random_field(n, 13)
        e = np.where(synthetic.retained_mask(n), np.fft.rfft2(s), 0)
        e[0, 0] = 0
        return rel(orc.omega_from_control(Q, s), e) < 1e-13

    def control_transpose():
        s = synthetic.random_field(n, 11)
        lam = synthetic.random_retained_hat(n, 12)
        a = dot(orc.omega_from_control(P, s), lam)
        return abs(a - float(np.sum(s * orc.gradient_map(P, lam)))) < 1e-12 * abs(a)

    def sobolev_fd():
        Q = orc.Problem(**{**P.__dict__, "sobolev": 1e-2})
        truth = orc.control_from_omega(Q, synthetic.random_vorticity_hat(n, 20) * 2)
        _, m = orc.forward(Q, truth)
        s = orc.control_from_omega(Q, synthetic.random_vorticity_hat(n, 21) * 2)
        _, g, _ = orc.cost_grad(Q, s, m)
        d = synthetic.random_field(n, 31)
        fd = (orc.cost(Q, s + 1e-4 * d, m) - orc.cost(Q, s - 1e-4 * d, m)) / 2e-4
        return abs(fd - np.sum(g * d)) < 1e-7 * abs(fd)

    def kernel_values():
        # m(k) = |k| W^{1/2} at modes where special parameters fix exact values
        KX, KY = synthetic.wavenumbers(n)
        table = 4.0 ** (-np.abs(KX)) * 9.0 ** (-np.abs(KY))
        cases = [("exp_abs", math.log(4.0), 1e-2, None, [(1, 0, 0.5), (3, 4, 5 / 32)]),
                 ("frac", 0.5, 1e-2, None, [(0, 4, 2.0), (3, 4, math.sqrt(5.0))]),
                 ("frac", 1.5, 1e-2, None, [(0, 4, 0.5)]),
                 ("exp_sq", 100 * math.log(2.0), 1e-2, None, [(1, 1, math.sqrt(2.0) / 2), (0, 2, 0.5)]),
                 ("table", 0.0, 1e-2, table, [(0, 1, 1 / 3), (4, -3, 5 / 432)])]
        for kernel, kp, nu, tab, vals in cases:
            Q = orc.Problem(n=n, nsteps=1, dt=1e-3, nu=nu, px=4, every=1, kernel=kernel, kparam=kp, ktable=tab)
            for kx, ky, m in vals:
                if abs(mode_multiplier(orc, Q, kx, ky) - m) > 4e-15 * m:
                    return False
        return True

    def gradient_fd():
        truth = orc.control_from_omega(P, synthetic.random_vorticity_hat(n, 20) * 2)
        _, m = orc.forward(P, truth)
        s = orc.control_from_omega(P, synthetic.random_vorticity_hat(n, 21) * 2)
        J, g, _ = orc.cost_grad(P, s, m)
        d = synthetic.random_field(n, 30)
        fd = (orc.cost(P, s + 1e-4 * d, m) - orc.cost(P, s - 1e-4 * d, m)) / 2e-4
        return abs(fd - np.sum(g * d)) < 1e-7 * abs(fd)

    for name, fn in [("biot_savart", biot_savart), ("advection", closed_form_advection), ("taylor_green", taylor_green),
                     ("kolmogorov", kolmogorov), ("conservation", conservation), ("rhs_dot", rhs_dot),
                     ("rhs_tangent", rhs_tangent), ("step", step_dot), ("obs_transpose", obs_transpose),
                     ("vorticity_control", vorticity_control), ("control_transpose", control_transpose),
                     ("gradient_fd", gradient_fd), ("sobolev_fd", sobolev_fd), ("kernel_values", kernel_values)]:
        check(name, fn)
    return failed


MUTATIONS = [
    ("drop_adjoint_term", "for (int t = 0; t < 4; ++t) {", "for (int t = 0; t < 3; ++t) {"),
    ("v_sign", "return k2 > 0 ? -I * kx / k2 : 0;", "return k2 > 0 ? I * kx / k2 : 0;"),
    ("u_symbol_index", "return k2 > 0 ? I * ky / k2 : 0;", "return k2 > 0 ? I * kx / k2 : 0;"),
    ("adjoint_stage_coeff", "const double a_yb[4] = {0, dt, dt / 2, dt / 2};", "const double a_yb[4] = {0, dt / 2, dt / 2, dt / 2};"),
    ("adjoint_uses_wrong_stage", "orc_rhs_adj(c, (double*)ys[j], (double*)kb, (double*)yb);",
     "orc_rhs_adj(c, (double*)ys[s], (double*)kb, (double*)yb);"),
    ("no_conjugate_in_transpose", "if (transpose) s = conj(s);", "if (transpose) s = s;"),
    ("forcing_sign", "double v = -c->amp * c->nf * (double)n * n / 2.0;", "double v = c->amp * c->nf * (double)n * n / 2.0;"),
    ("rk4_weight", "o[i] = w[i] + dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);",
     "o[i] = w[i] + dt / 6.0 * (k1[i] + 2.0 * k2[i] + k3[i] + 2.0 * k4[i]);"),
    ("hermitian_index", "a[q * n + p] = conj(h[((n - q) % n) * nh(n) + (n - p)]);", "a[q * n + p] = conj(h[q * nh(n) + (n - p)]);"),
    ("dropped_k_in_control", "return k * sqrt(kernel_W(c, kx, ky, q, p));", "return sqrt(kernel_W(c, kx, ky, q, p));"),
    ("viscous_sign_in_adjoint", "o[i] = in_R(kx, ky, n) ? (acc[i] - c->nu * k2 * mu[i]) : 0;",
     "o[i] = in_R(kx, ky, n) ? (acc[i] + c->nu * k2 * mu[i]) : 0;"),
    ("dealias_cut", "return abs(kx) <= K && abs(ky) <= K;", "return abs(kx) <= K + 1 && abs(ky) <= K + 1;"),
    ("nonlinear_term_dropped", "nl[i] = g.u[i] * g.wx[i] + g.v[i] * g.wy[i];", "nl[i] = g.u[i] * g.wx[i];"),
    ("exp_abs_squared_exponent", "case 1: return exp(-c->kparam * k);", "case 1: return exp(-c->kparam * k2);"),
    ("exp_sq_drops_nu", "case 3: return exp(-c->nu * c->kparam * k2);", "case 3: return exp(-c->kparam * k2);"),
    ("W_in_place_of_sqrt_W", "return k * sqrt(kernel_W(c, kx, ky, q, p));", "return k * kernel_W(c, kx, ky, q, p);"),
    ("frac_half_exponent", "case 2: return pow(k, -2.0 * c->kparam);", "case 2: return pow(k, -c->kparam);"),
    ("table_transposed", "case 4: return c->ktable[q * nh(c->n) + p];", "case 4: return c->ktable[p * nh(c->n) + q];"),
    ("sobolev_gradient_sign", "for (int i = 0; i < nn; ++i) lam[i] += c->sobolev * t2[i];",
     "for (int i = 0; i < nn; ++i) lam[i] -= c->sobolev * t2[i];"),
]


def test_unmodified_oracle_passes_battery(orc):
    assert battery(orc) == []


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(orc, tmp_path, name, old, new):
    src = orc.source_text()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    lib = orc.compile_variant(src.replace(old, new), str(tmp_path / f"mut_{name}.so"))
    with orc.use_library(lib):
        failed = battery(orc)
    assert failed, f"planted mistake {name} passed every pin"
