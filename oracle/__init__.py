"""Plain FP64 CPU oracle for preconditioned adjoint data assimilation.

TEST INFRASTRUCTURE ONLY.  This package may be imported, called, linked or
executed only by ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The product
path (``paper_2602_14016_gb300``) never imports it, and it imports nothing
from the product.

The arithmetic lives in ``da_oracle.c`` (plain loops, radix-2 FFT, FP64);
this module compiles it with gcc and wraps it with ctypes.  Spectral arrays
are numpy complex128 of shape (n, n//2 + 1) holding the half spectrum
``w_hat[q, p]`` (ky index q, kx = p); physical arrays are float64 (n, n).

Parity status: all wrapped functions are pinned by ``tests/test_oracle_*``
(brute-force DFT, closed forms, Taylor-Green decay, laminar Kolmogorov,
conservation, dot-product tests, finite differences; the control multiplier
|k| W^{1/2} of every kernel family by exact values at special parameters and
by the families' semigroup and power identities).  The L-BFGS driver in
``oracle/lbfgs.py`` is pinned on the toy problem of Sec. II.C and on
quadratics; beyond that, full assimilation trajectories are compared only on
their first iterations.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "da_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libda_oracle.so")
_lib = None
_lock = threading.Lock()

KERNELS = {"identity": 0, "exp_abs": 1, "frac": 2, "exp_sq": 3, "table": 4}
# no FMA contraction: the oracle rounds every operation as written, the same
# way on x86 and Arm hosts
_CFLAGS = ["-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile da_oracle.c into libda_oracle.so next to it (gcc, -O2)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *_CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int),
        ("nsteps", ctypes.c_int),
        ("dt", ctypes.c_double),
        ("nu", ctypes.c_double),
        ("force_kind", ctypes.c_int),
        ("amp", ctypes.c_double),
        ("nf", ctypes.c_int),
        ("px", ctypes.c_int),
        ("every", ctypes.c_int),
        ("include_t0", ctypes.c_int),
        ("kernel_kind", ctypes.c_int),
        ("kparam", ctypes.c_double),
        ("ktable", ctypes.c_void_p),
        ("sobolev", ctypes.c_double),
    ]


@dataclasses.dataclass
class Problem:
    """One assimilation window: grid, physics, probes and kernel."""

    n: int
    nsteps: int
    dt: float
    nu: float
    forcing: str = "none"  # "none" or "kolmogorov"
    amp: float = 1.0
    nf: int = 4
    px: int = 8
    every: int = 10
    include_t0: bool = False
    kernel: str = "identity"
    kparam: float = 0.0
    ktable: np.ndarray | None = None
    sobolev: float = 0.0  # lambda of the regularisation term of Eq. (4)

    def cfg(self) -> _Cfg:
        c = _Cfg()
        c.n, c.nsteps, c.dt, c.nu = self.n, self.nsteps, self.dt, self.nu
        c.force_kind = 1 if self.forcing == "kolmogorov" else 0
        c.amp, c.nf = self.amp, self.nf
        c.px, c.every, c.include_t0 = self.px, self.every, int(self.include_t0)
        c.kernel_kind, c.kparam = KERNELS[self.kernel], self.kparam
        if self.ktable is not None:
            self._tab = np.ascontiguousarray(self.ktable, dtype=np.float64)
            c.ktable = self._tab.ctypes.data
        else:
            c.ktable = None
        c.sobolev = self.sobolev
        return c

    @property
    def nt(self) -> int:
        return self.nsteps // self.every + (1 if self.include_t0 else 0)

    @property
    def nh(self) -> int:
        return self.n // 2 + 1


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(ctypes.CDLL(_LIB_PATH))
    return _lib


class use_library:
    """Context manager that points this module at another build of the
    oracle source (used by the tests that plant mistakes in a copy)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        _load()
        self._saved = _lib
        _lib = _bind(ctypes.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def compile_variant(source_text: str, out_path: str) -> str:
    """Compile a modified copy of da_oracle.c (test use only)."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.check_call(["gcc", *_CFLAGS, "-o", out_path, src, "-lm"])
    return out_path


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _bind(lib):
    """Declare the C signatures on a loaded oracle library."""
    P = ctypes.c_void_p
    C = ctypes.POINTER(_Cfg)
    sigs = {
        "orc_rhs": [C, P, P],
        "orc_rhs_tlm": [C, P, P, P],
        "orc_rhs_adj": [C, P, P, P],
        "orc_step": [C, P, P],
        "orc_step_tlm": [C, P, P, P, P],
        "orc_step_adj": [C, P, P, P],
        "orc_observe": [C, P, P],
        "orc_observe_adj": [C, P, P],
        "orc_omega_from_control": [C, P, P],
        "orc_control_from_omega": [C, P, P],
        "orc_gradient_map": [C, P, P],
        "orc_forward": [C, P, P, P, P],
        "orc_cost_grad": [C, P, P, P, P, P],
        "orc_forward_tlm": [C, P, P, P],
        "orc_adjoint_terminal": [C, P, P, P, P],
        "orc_fft1d": [P, ctypes.c_int, ctypes.c_int],
        "orc_r2c": [P, P, ctypes.c_int],
        "orc_c2r": [P, P, ctypes.c_int],
    }
    for name, args in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = None
    lib.orc_num_obs_times.argtypes = [C]
    lib.orc_num_obs_times.restype = ctypes.c_int
    lib.orc_sobolev_term.argtypes = [C, P]
    lib.orc_sobolev_term.restype = ctypes.c_double
    return lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


def _spec(a, n) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    assert a.shape == (n, n // 2 + 1), a.shape
    return a


def _phys(a, n) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    assert a.shape == (n, n), a.shape
    return a


# ---- transforms -----------------------------------------------------------

def fft1d(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """Radix-2 complex DFT sum_j x_j exp(sign 2 pi i jk/m), unscaled."""
    y = np.ascontiguousarray(x, dtype=np.complex128).copy()
    _load().orc_fft1d(_ptr(y), y.size, sign)
    return y


def r2c(f: np.ndarray) -> np.ndarray:
    n = f.shape[0]
    f = _phys(f, n)
    h = np.zeros((n, n // 2 + 1), np.complex128)
    _load().orc_r2c(_ptr(f), _ptr(h), n)
    return h


def c2r(h: np.ndarray) -> np.ndarray:
    n = h.shape[0]
    h = _spec(h, n)
    f = np.zeros((n, n), np.float64)
    _load().orc_c2r(_ptr(h), _ptr(f), n)
    return f


# ---- operators ------------------------------------------------------------

def _call_spec_out(name, prob: Problem, *args, shape=None, dtype=np.complex128):
    n = prob.n
    out = np.zeros(shape or (n, n // 2 + 1), dtype)
    c = prob.cfg()
    getattr(_load(), name)(ctypes.byref(c), *[_ptr(a) for a in args], _ptr(out))
    return out


def rhs(prob: Problem, w: np.ndarray) -> np.ndarray:
    return _call_spec_out("orc_rhs", prob, _spec(w, prob.n))


def rhs_tlm(prob: Problem, y: np.ndarray, dy: np.ndarray) -> np.ndarray:
    return _call_spec_out("orc_rhs_tlm", prob, _spec(y, prob.n), _spec(dy, prob.n))


def rhs_adj(prob: Problem, y: np.ndarray, mu: np.ndarray) -> np.ndarray:
    return _call_spec_out("orc_rhs_adj", prob, _spec(y, prob.n), _spec(mu, prob.n))


def step(prob: Problem, w: np.ndarray) -> np.ndarray:
    return _call_spec_out("orc_step", prob, _spec(w, prob.n))


def step_tlm(prob: Problem, w: np.ndarray, dw: np.ndarray):
    n = prob.n
    w2 = np.zeros((n, n // 2 + 1), np.complex128)
    dw2 = np.zeros_like(w2)
    c = prob.cfg()
    _load().orc_step_tlm(ctypes.byref(c), _ptr(_spec(w, n)), _ptr(_spec(dw, n)), _ptr(w2), _ptr(dw2))
    return w2, dw2


def step_adj(prob: Problem, w: np.ndarray, lam: np.ndarray) -> np.ndarray:
    return _call_spec_out("orc_step_adj", prob, _spec(w, prob.n), _spec(lam, prob.n))


def observe(prob: Problem, w: np.ndarray) -> np.ndarray:
    return _call_spec_out("orc_observe", prob, _spec(w, prob.n), shape=(prob.px * prob.px, 2), dtype=np.float64)


def observe_adj(prob: Problem, r: np.ndarray) -> np.ndarray:
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(prob.px * prob.px, 2)
    return _call_spec_out("orc_observe_adj", prob, r)


def omega_from_control(prob: Problem, s: np.ndarray) -> np.ndarray:
    return _call_spec_out("orc_omega_from_control", prob, _phys(s, prob.n))


def control_from_omega(prob: Problem, w0: np.ndarray) -> np.ndarray:
    return _call_spec_out("orc_control_from_omega", prob, _spec(w0, prob.n), shape=(prob.n, prob.n), dtype=np.float64)


def gradient_map(prob: Problem, lam0: np.ndarray) -> np.ndarray:
    return _call_spec_out("orc_gradient_map", prob, _spec(lam0, prob.n), shape=(prob.n, prob.n), dtype=np.float64)


# ---- window ---------------------------------------------------------------

def forward(prob: Problem, s: np.ndarray, trajectory: bool = False):
    """Returns (wT_hat, obs[nt, px*px, 2]) and, if asked, the states [nsteps+1, n, nh]."""
    n = prob.n
    wT = np.zeros((n, n // 2 + 1), np.complex128)
    obs = np.zeros((prob.nt, prob.px * prob.px, 2), np.float64)
    traj = np.zeros((prob.nsteps + 1, n, n // 2 + 1), np.complex128) if trajectory else None
    c = prob.cfg()
    _load().orc_forward(ctypes.byref(c), _ptr(_phys(s, n)), _ptr(wT), _ptr(obs), _ptr(traj))
    return (wT, obs, traj) if trajectory else (wT, obs)


def cost_grad(prob: Problem, s: np.ndarray, m: np.ndarray):
    """Returns (J, grad_s[n, n], lam0_hat[n, nh])."""
    n = prob.n
    m = np.ascontiguousarray(m, dtype=np.float64)
    assert m.size == prob.nt * prob.px * prob.px * 2
    J = ctypes.c_double(0.0)
    g = np.zeros((n, n), np.float64)
    lam0 = np.zeros((n, n // 2 + 1), np.complex128)
    c = prob.cfg()
    _load().orc_cost_grad(ctypes.byref(c), _ptr(_phys(s, n)), _ptr(m), ctypes.byref(J), _ptr(g), _ptr(lam0))
    return J.value, g, lam0


def forward_tlm(prob: Problem, s: np.ndarray, ds: np.ndarray) -> np.ndarray:
    return _call_spec_out("orc_forward_tlm", prob, _phys(s, prob.n), _phys(ds, prob.n))


def adjoint_terminal(prob: Problem, s: np.ndarray, lamT: np.ndarray):
    """Adjoint driven by a terminal field only: returns (lam0_hat, grad_s)."""
    n = prob.n
    lam0 = np.zeros((n, n // 2 + 1), np.complex128)
    g = np.zeros((n, n), np.float64)
    c = prob.cfg()
    _load().orc_adjoint_terminal(ctypes.byref(c), _ptr(_phys(s, n)), _ptr(_spec(lamT, n)), _ptr(lam0), _ptr(g))
    return lam0, g


def sobolev_term(prob: Problem, w0: np.ndarray) -> float:
    """lambda/2 sum_grid |grad u0|^2 of Eq. (4) for the initial vorticity w0."""
    c = prob.cfg()
    return float(_load().orc_sobolev_term(ctypes.byref(c), _ptr(_spec(w0, prob.n))))


def cost(prob: Problem, s: np.ndarray, m: np.ndarray) -> float:
    """J alone, from a forward solve (used by finite-difference pins)."""
    _, obs = forward(prob, s)
    r = obs - np.asarray(m).reshape(obs.shape)
    J = 0.5 * float(np.sum(r * r))
    if prob.sobolev:
        J += sobolev_term(prob, omega_from_control(prob, s))
    return J
