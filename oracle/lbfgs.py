"""Plain L-BFGS with a More-Thuente line search -- oracle of the optimiser
that drives the assimilation (Sec. II.C: L-BFGS on the transformed control
s0 in the Euclidean metric).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper names L-BFGS but not its settings.  Reading used here: memory 10;
initial inverse-Hessian scaling s^T y / y^T y; first trial step
min(1, 1/||g||) on the first iteration and 1 afterwards; a line search that
enforces the strong Wolfe conditions (c1 = 1e-4, c2 = 0.9) by the
safeguarded cubic/quadratic interval updates of More and Thuente (ACM TOMS
20, 1994); stop at max_iter, at ||g|| <= gtol_rel ||g0||, or when the line
search fails (reported as not converged: the "step-size collapse" the paper
describes for badly scaled kernels, Sec. III.C-D).
"""
from __future__ import annotations

import math

import numpy as np

C1 = 1e-4
C2 = 0.9
XTOL = 1e-10
STPMIN = 1e-20
STPMAX = 1e20
MAX_LS_EVALS = 20


def _cubic_min(a, fa, da, b, fb, db):
    """Minimiser of the cubic that interpolates (a, fa, da) and (b, fb, db),
    written with the scaling that avoids overflow."""
    theta = 3.0 * (fa - fb) / (b - a) + da + db
    s = max(abs(theta), abs(da), abs(db))
    disc = (theta / s) ** 2 - (da / s) * (db / s)
    gamma = s * math.sqrt(max(disc, 0.0))
    if b < a:
        gamma = -gamma
    p = (gamma - da) + theta
    q = ((gamma - da) + gamma) + db
    return a + (p / q) * (b - a)


def _safeguarded_step(stx, fx, dx, sty, fy, dy, stp, fp, dp, brackt, lo, hi):
    """One More-Thuente interval update.  Returns the new
    (stx, fx, dx, sty, fy, dy, next trial step, brackt)."""
    opposite = dp * math.copysign(1.0, dx) < 0
    if fp > fx:
        # higher value: the minimiser lies between stx and stp
        c = _cubic_min(stx, fx, dx, stp, fp, dp)
        qd = stx + (dx / ((fx - fp) / (stp - stx) + dx)) / 2.0 * (stp - stx)
        nxt = c if abs(c - stx) < abs(qd - stx) else c + (qd - c) / 2.0
        brackt = True
    elif opposite:
        # derivative changed sign: bracketed between stp and stx
        c = _cubic_min(stp, fp, dp, stx, fx, dx)
        sec = stp + (dp / (dp - dx)) * (stx - stp)
        nxt = c if abs(c - stp) > abs(sec - stp) else sec
        brackt = True
    elif abs(dp) < abs(dx):
        # same sign, slope shrinking: the cubic may have no minimiser on the
        # far side, in which case step to the bound
        theta = 3.0 * (fx - fp) / (stp - stx) + dx + dp
        s = max(abs(theta), abs(dx), abs(dp))
        gamma = s * math.sqrt(max(0.0, (theta / s) ** 2 - (dx / s) * (dp / s)))
        if stp > stx:
            gamma = -gamma
        p = (gamma - dp) + theta
        q = (gamma + (dx - dp)) + gamma
        r = p / q
        if r < 0.0 and gamma != 0.0:
            c = stp + r * (stx - stp)
        else:
            c = hi if stp > stx else lo
        sec = stp + (dp / (dp - dx)) * (stx - stp)
        if brackt:
            nxt = c if abs(c - stp) < abs(sec - stp) else sec
            lim = stp + 0.66 * (sty - stp)
            nxt = min(lim, nxt) if stp > stx else max(lim, nxt)
        else:
            nxt = c if abs(c - stp) > abs(sec - stp) else sec
            nxt = min(hi, max(lo, nxt))
    else:
        # same sign, slope not shrinking: extrapolate, or use the far end
        if brackt:
            nxt = _cubic_min(stp, fp, dp, sty, fy, dy)
        else:
            nxt = hi if stp > stx else lo
    if fp > fx:
        sty, fy, dy = stp, fp, dp
    else:
        if opposite:
            sty, fy, dy = stx, fx, dx
        stx, fx, dx = stp, fp, dp
    return stx, fx, dx, sty, fy, dy, nxt, brackt


def more_thuente(phi, stp, f0, g0, c1=C1, c2=C2, xtol=XTOL, stpmin=STPMIN, stpmax=STPMAX, max_evals=MAX_LS_EVALS):
    """Strong-Wolfe line search.  ``phi(a)`` returns (f, f'(a)).

    Returns (step, f, g, evals, ok)."""
    if g0 >= 0 or stp <= 0:
        return 0.0, f0, g0, 0, False
    brackt = False
    stage1 = True
    gtest = c1 * g0
    width = stpmax - stpmin
    width1 = 2.0 * width
    stx, fx, gx = 0.0, f0, g0
    sty, fy, gy = 0.0, f0, g0
    lo, hi = 0.0, stp + 4.0 * stp
    evals = 0
    while True:
        f, g = phi(stp)
        evals += 1
        ftest = f0 + stp * gtest
        if stage1 and f <= ftest and g >= 0:
            stage1 = False
        if f <= ftest and abs(g) <= c2 * (-g0):
            return stp, f, g, evals, True
        if brackt and (stp <= lo or stp >= hi):
            return stp, f, g, evals, False
        if brackt and hi - lo <= xtol * hi:
            return stp, f, g, evals, False
        if stp == stpmax and f <= ftest and g <= gtest:
            return stp, f, g, evals, False
        if stp == stpmin and (f > ftest or g >= gtest):
            return stp, f, g, evals, False
        if evals >= max_evals:
            return stp, f, g, evals, False
        if stage1 and f <= fx and f > ftest:
            # work with the auxiliary function psi(a) = phi(a) - a gtest
            stx, fxm, gxm, sty, fym, gym, stp_new, brackt = _safeguarded_step(
                stx, fx - stx * gtest, gx - gtest, sty, fy - sty * gtest, gy - gtest,
                stp, f - stp * gtest, g - gtest, brackt, lo, hi)
            fx, gx = fxm + stx * gtest, gxm + gtest
            fy, gy = fym + sty * gtest, gym + gtest
        else:
            stx, fx, gx, sty, fy, gy, stp_new, brackt = _safeguarded_step(
                stx, fx, gx, sty, fy, gy, stp, f, g, brackt, lo, hi)
        stp = stp_new
        if brackt:
            if abs(sty - stx) >= 0.66 * width1:
                stp = stx + 0.5 * (sty - stx)
            width1 = width
            width = abs(sty - stx)
            lo, hi = min(stx, sty), max(stx, sty)
        else:
            lo, hi = stp + 1.1 * (stp - stx), stp + 4.0 * (stp - stx)
        stp = min(max(stp, stpmin), stpmax)
        if (brackt and (stp <= lo or stp >= hi)) or (brackt and hi - lo <= xtol * hi):
            stp = stx


def two_loop(g, S, Y):
    """H g for the L-BFGS inverse-Hessian approximation built from the pairs
    (s_i, y_i), oldest first, with H0 = (s^T y / y^T y) I from the newest."""
    q = g.copy()
    alphas = []
    for s, y in reversed(list(zip(S, Y))):
        rho = 1.0 / float(np.dot(y, s))
        a = rho * float(np.dot(s, q))
        alphas.append((a, rho))
        q -= a * y
    if S:
        q *= float(np.dot(S[-1], Y[-1])) / float(np.dot(Y[-1], Y[-1]))
    for (s, y), (a, rho) in zip(zip(S, Y), reversed(alphas)):
        b = rho * float(np.dot(y, q))
        q += (a - b) * s
    return q


def minimize(fg, x0, max_iter, memory=10, gtol_rel=1e-10):
    """Minimise f with gradient from ``fg(x) -> (f, g)``.

    Returns dict(x, f, J_hist, iters, evals, converged, status) where status
    is "max_iter", "gtol" or "linesearch"."""
    x = np.array(x0, dtype=np.float64, copy=True)
    f, g = fg(x)
    g = np.asarray(g, dtype=np.float64)
    g0n = float(np.linalg.norm(g))
    hist = [float(f)]
    S, Y = [], []
    evals = 1
    status = "max_iter"
    it = 0
    while it < max_iter:
        if float(np.linalg.norm(g)) <= gtol_rel * g0n:
            status = "gtol"
            break
        d = -two_loop(g, S, Y)
        gd = float(np.dot(g, d))
        if gd >= 0:  # not a descent direction: restart from steepest descent
            S, Y = [], []
            d = -g
            gd = float(np.dot(g, d))
        stp0 = min(1.0, 1.0 / float(np.linalg.norm(g))) if it == 0 else 1.0
        cache = {}

        def phi(a):
            xa = x + a * d
            fa, ga = fg(xa)
            ga = np.asarray(ga, dtype=np.float64)
            cache[a] = (xa, fa, ga)
            return float(fa), float(np.dot(ga, d))

        stp, fn, _, ne, ok = more_thuente(phi, stp0, float(f), gd)
        evals += ne
        if not ok:
            status = "linesearch"
            if stp in cache and cache[stp][1] < f:
                x, f, g = cache[stp]
                hist.append(float(f))
                it += 1
            break
        xn, fn, gn = cache[stp]
        s_, y_ = xn - x, gn - g
        if float(np.dot(s_, y_)) > 1e-16 * float(np.dot(y_, y_)):
            S.append(s_)
            Y.append(y_)
            if len(S) > memory:
                S.pop(0)
                Y.pop(0)
        x, f, g = xn, fn, gn
        hist.append(float(f))
        it += 1
    return dict(x=x, f=float(f), J_hist=hist, iters=it, evals=evals,
                converged=status != "linesearch", status=status)
