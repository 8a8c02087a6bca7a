"""ctypes declarations of the C ABI in include/da.h (argument marshalling only).

The library is the in-tree ``libda_gb300.so`` built by ``build.py``.  There
is no fallback: if the library is missing or cannot be loaded, every entry
point raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libda_gb300.so")

DA_OK, DA_EINVAL, DA_ENOMEM, DA_ECUDA, DA_ETIMEOUT, DA_EDIVERGED, DA_ENOTCONV = range(7)
STATUS_NAMES = {0: "DA_OK", 1: "DA_EINVAL", 2: "DA_ENOMEM", 3: "DA_ECUDA", 4: "DA_ETIMEOUT", 5: "DA_EDIVERGED",
                6: "DA_ENOTCONV"}

KERNEL_KINDS = {"identity": 0, "exp_abs": 1, "frac": 2, "exp_sq": 3, "table": 4}

# Entry points declared in include/da.h, in order.
EXPORTS = ("da_create", "da_set_sobolev", "da_set_graphs", "da_plan_count", "da_get_plan", "da_set_plan", "da_autotune",
           "da_plan_flops", "da_set_observations", "da_forward", "da_cost_grad", "da_vjp", "da_last_adjoint",
           "da_adjoint_terminal", "da_adjoint_spectra", "da_num_shells", "da_assimilate", "da_set_member",
           "da_lbfgs_start", "da_lbfgs_iterate", "da_lbfgs_member", "da_lbfgs_release", "da_omega_from_control",
           "da_control_from_omega",
           "da_omega_from_control_static", "da_fp64_probe", "da_num_obs_times", "da_device_bytes", "da_launch_count",
           "da_time_kernels", "da_kernel_time", "da_last_error", "da_destroy")


class Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("L", ctypes.c_double), ("dt", ctypes.c_double), ("nsteps", ctypes.c_int),
                ("ckpt_every", ctypes.c_int), ("batch", ctypes.c_int)]


class Forcing(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("amp", ctypes.c_double), ("nf", ctypes.c_int)]


class ObsOperator(ctypes.Structure):
    _fields_ = [("px", ctypes.c_int), ("py", ctypes.c_int), ("every", ctypes.c_int), ("include_t0", ctypes.c_int)]


class Kernel(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("param", ctypes.c_double), ("table", ctypes.c_void_p)]


class MemberWindow(ctypes.Structure):
    _fields_ = [("nsteps", ctypes.c_int), ("px", ctypes.c_int), ("nu", ctypes.c_double), ("forcing", ctypes.c_int)]


class LbfgsReport(ctypes.Structure):
    _fields_ = [("phase", ctypes.c_int), ("status", ctypes.c_int), ("iters", ctypes.c_int), ("J0", ctypes.c_double),
                ("J", ctypes.c_double)]


class LbfgsOpts(ctypes.Structure):
    _fields_ = [("memory", ctypes.c_int), ("c1", ctypes.c_double), ("c2", ctypes.c_double),
                ("gtol_rel", ctypes.c_double), ("max_ls_evals", ctypes.c_int)]


class DAError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Load and declare the library (raises if it is absent)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError(f"CUDA library {path} is not built; run paper_2602_14016_gb300.build.build()")
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        C = ctypes.c_void_p  # da_ctx*
        I = ctypes.c_int
        D = ctypes.c_double
        sig = {
            "da_create": (I, [ctypes.POINTER(C), ctypes.POINTER(Grid), D, ctypes.POINTER(Forcing),
                              ctypes.POINTER(ObsOperator), ctypes.POINTER(Kernel)]),
            "da_set_sobolev": (I, [C, D]),
            "da_set_graphs": (I, [C, I]),
            "da_plan_count": (I, [I]),
            "da_get_plan": (I, [C]),
            "da_set_plan": (I, [C, I]),
            "da_autotune": (I, [C, I, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
            "da_plan_flops": (I, [I, I, ctypes.POINTER(D), ctypes.POINTER(D)]),
            "da_set_observations": (I, [C, P, P]),
            "da_forward": (I, [C, P, P, P, P]),
            "da_cost_grad": (I, [C, P, P, P, P]),
            "da_vjp": (I, [C, P, P, P, P]),
            "da_last_adjoint": (I, [C, P, P, P]),
            "da_adjoint_terminal": (I, [C, P, P, P, P]),
            "da_adjoint_spectra": (I, [C, P, P, I, P, P, P]),
            "da_num_shells": (I, [C]),
            "da_assimilate": (I, [C, P, I, ctypes.POINTER(LbfgsOpts), P, P, P, P]),
            "da_set_member": (I, [C, I, ctypes.POINTER(MemberWindow), ctypes.POINTER(Kernel), P, P]),
            "da_lbfgs_start": (I, [C, I, P, I, ctypes.POINTER(LbfgsOpts), P]),
            "da_lbfgs_iterate": (I, [C, ctypes.POINTER(ctypes.c_int), P]),
            "da_lbfgs_member": (I, [C, I, ctypes.POINTER(LbfgsReport), P, I, P, P]),
            "da_lbfgs_release": (I, [C, I]),
            "da_omega_from_control": (I, [C, P, P, P]),
            "da_control_from_omega": (I, [C, P, P, P]),
            "da_omega_from_control_static": (I, [I, D, ctypes.POINTER(Kernel), P, P, P,
                                                 ctypes.POINTER(ctypes.c_char_p)]),
            "da_fp64_probe": (I, [I, I, ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D), P]),
            "da_num_obs_times": (I, [C]),
            "da_device_bytes": (ctypes.c_ulonglong, [C]),
            "da_launch_count": (ctypes.c_ulonglong, [C]),
            "da_time_kernels": (I, [C, I]),
            "da_kernel_time": (I, [C, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_ulonglong)]),
            "da_last_error": (ctypes.c_char_p, [C]),
            "da_destroy": (None, [C]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def check(status: int, ctx) -> None:
    if status != DA_OK:
        msg = load().da_last_error(ctx)
        raise DAError(status, msg.decode() if msg else "")
