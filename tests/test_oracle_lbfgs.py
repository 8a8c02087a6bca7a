"""Pins of the oracle's optimiser: the toy problem printed in Sec. II.C
(Fig. 1), quadratics with known minimisers, the strong Wolfe conditions, and
scipy's MINPACK line search (a separate implementation of More-Thuente)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import lbfgs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "toy_problem.json")


def toy():
    with open(GOLDEN) as f:
        return json.load(f)


def test_toy_gradients_match_the_printed_forms():
    t = toy()
    a = np.array(t["J_coefficients"])
    G = np.array(t["G_diag"])
    u = np.array([0.7, -1.3])
    grad_u = 2 * a * u
    assert np.allclose(grad_u, np.array(t["gradient_u_coefficients"]) * u, rtol=0, atol=1e-15)
    s = u / np.sqrt(G)
    assert abs(np.sum(a * u * u) - np.sum(s * s)) < 1e-15
    assert np.allclose(np.sqrt(G) * grad_u, np.array(t["gradient_s_coefficients"]) * s, atol=1e-15)


def _toy_run(space, max_iter=30):
    t = toy()
    a = np.array(t["J_coefficients"])
    G = np.array(t["G_diag"])
    u0 = np.array([3.0, 0.5])
    if space == "u":
        fg = lambda u: (float(np.sum(a * u * u)), 2 * a * u)
        x0 = u0
    else:
        fg = lambda s: (float(np.sum(a * G * s * s)), 2 * a * G * s)
        x0 = u0 / np.sqrt(G)
    return lbfgs.minimize(fg, x0, max_iter, gtol_rel=1e-12)


def test_toy_problem_converges_faster_in_latent_space():
    rs = _toy_run("s")
    ru = _toy_run("u")
    assert rs["f"] < 1e-20 and rs["iters"] <= 2
    assert ru["iters"] > rs["iters"]
    assert ru["f"] < 1e-12


def test_steepest_descent_zigzags_without_preconditioner():
    """Memory 0 is steepest descent with a Wolfe line search: many iterations in u, one in s."""
    t = toy()
    a = np.array(t["J_coefficients"])
    G = np.array(t["G_diag"])
    fu = lambda u: (float(np.sum(a * u * u)), 2 * a * u)
    fs = lambda s: (float(np.sum(a * G * s * s)), 2 * a * G * s)
    ru = lbfgs.minimize(fu, np.array([3.0, 0.5]), 8, memory=0)
    rs = lbfgs.minimize(fs, np.array([3.0, 0.5]) / np.sqrt(G), 8, memory=0)
    assert rs["f"] < 1e-20
    assert ru["f"] > 1e-6


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_quadratic_known_minimiser(seed):
    rng = np.random.default_rng(seed)
    n = 40
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(np.logspace(0, 3, n)) @ Q.T
    b = rng.standard_normal(n)
    fg = lambda x: (0.5 * x @ A @ x - b @ x, A @ x - b)
    r = lbfgs.minimize(fg, np.zeros(n), 500, gtol_rel=1e-11)
    xs = np.linalg.solve(A, b)
    # a value-based line search stops where f can no longer resolve the
    # decrease: |dx|/|x| ~ sqrt(eps cond(A)) ~ 3e-7 here
    assert np.linalg.norm(r["x"] - xs) < 1e-6 * np.linalg.norm(xs)
    assert all(h1 < h0 for h0, h1 in zip(r["J_hist"], r["J_hist"][1:]))


def _wolfe_ok(phi, a, f0, g0, c1=1e-4, c2=0.9):
    f, g = phi(a)
    return f <= f0 + c1 * a * g0 and abs(g) <= c2 * abs(g0)


FUNCS = {
    "quartic": lambda a: ((a - 1.3) ** 4 + 0.1 * (a - 1.3) ** 2, 4 * (a - 1.3) ** 3 + 0.2 * (a - 1.3)),
    "rosen_line": lambda a: ((1 - a) ** 2 + 100 * (a * 0.3 - a * a) ** 2,
                             -2 * (1 - a) + 200 * (a * 0.3 - a * a) * (0.3 - 2 * a)),
    "exp_quad": lambda a: (math.exp(2 * a) - 6 * a, 2 * math.exp(2 * a) - 6),
    "far_min": lambda a: ((a - 40.0) ** 2, 2 * (a - 40.0)),
    "near_min": lambda a: ((a - 1e-3) ** 2 + a ** 4, 2 * (a - 1e-3) + 4 * a ** 3),
}


@pytest.mark.parametrize("name", list(FUNCS))
def test_line_search_satisfies_strong_wolfe(name):
    phi = FUNCS[name]
    f0, g0 = phi(0.0)
    a, f, g, ne, ok = lbfgs.more_thuente(phi, 1.0, f0, g0)
    assert ok and _wolfe_ok(phi, a, f0, g0)


@pytest.mark.parametrize("name", list(FUNCS))
def test_line_search_matches_minpack(name):
    """Same algorithm and parameters as scipy's MINPACK-based search."""
    ls = pytest.importorskip("scipy.optimize._linesearch")
    phi = FUNCS[name]
    f0, g0 = phi(0.0)
    ref = ls.scalar_search_wolfe1(lambda a: phi(a)[0], lambda a: phi(a)[1], f0, None, g0,
                                  c1=1e-4, c2=0.9, amax=50, amin=1e-8, xtol=1e-14)
    a, f, g, ne, ok = lbfgs.more_thuente(phi, 1.0, f0, g0, xtol=1e-14, stpmin=1e-8, stpmax=50, max_evals=100)
    assert ref[0] is not None and ok
    assert abs(a - ref[0]) <= 1e-12 * max(1.0, abs(ref[0]))
