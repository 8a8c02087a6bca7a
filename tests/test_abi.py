"""The C-ABI library loads, exports every entry point that include/da.h
declares, and rejects invalid problems on the host (no GPU needed)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    with open(os.path.join(ROOT, "include", "da.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(da_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2602_14016_gb300 import _native, build

    if shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc"):
        build.build()
    if not os.path.exists(_native.LIB_PATH):
        pytest.fail("libda_gb300.so is not built and nvcc is unavailable")
    return _native.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("da_create", "da_forward", "da_cost_grad", "da_assimilate", "da_set_observations",
                 "da_control_from_omega", "da_omega_from_control", "da_last_error", "da_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2602_14016_gb300 import _native

    names = declared_functions()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) == set(_native.EXPORTS)


def _create(lib, n=64, nsteps=10, dt=1e-3, batch=1, px=8, every=5, nf=4, force=0, kind=0, param=0.0, ckpt=0, L=0.0):
    from paper_2602_14016_gb300 import _native as N

    g = N.Grid(n, L, dt, nsteps, ckpt, batch)
    f = N.Forcing(force, 1.0, nf)
    o = N.ObsOperator(px, px, every, 0)
    ks = (N.Kernel * batch)(*[N.Kernel(kind, param, None) for _ in range(batch)])
    ctx = ctypes.c_void_p()
    st = lib.da_create(ctypes.byref(ctx), ctypes.byref(g), 1e-3, ctypes.byref(f), ctypes.byref(o), ks)
    return st, lib.da_last_error(None).decode()


@pytest.mark.parametrize("kw,frag", [
    (dict(n=100), "power of two"),
    (dict(n=2048), "power of two"),
    (dict(L=1.0), "2 pi"),
    (dict(dt=-1.0), "dt"),
    (dict(nsteps=0), "nsteps"),
    (dict(batch=0), "batch"),
    (dict(px=7), "px"),
    (dict(px=128, n=128), "px"),
    (dict(every=3), "every"),
    (dict(force=1, nf=40), "forcing"),
    (dict(kind=9), "kernel"),
    (dict(kind=1, param=float("nan")), "finite"),
    (dict(ckpt=-2), "ckpt_every"),
])
def test_invalid_problems_are_rejected_on_the_host(lib, kw, frag):
    from paper_2602_14016_gb300 import _native as N

    st, msg = _create(lib, **kw)
    assert st == N.DA_EINVAL
    assert frag in msg


def test_plan_variant_queries_on_the_host(lib):
    """Plan counts per supported size, 0 elsewhere; NULL contexts are rejected
    before any device work."""
    counts = {16: 1, 32: 2, 64: 3, 128: 4, 256: 3, 512: 3, 1024: 3}
    for n, c in counts.items():
        assert lib.da_plan_count(n) == c
    for n in (0, 8, 48, 100, 2048):
        assert lib.da_plan_count(n) == 0
    assert lib.da_get_plan(None) == -1
    assert lib.da_set_plan(None, 0) == 1  # DA_EINVAL
    chosen = ctypes.c_int(-7)
    assert lib.da_autotune(None, 4, ctypes.byref(chosen), None) == 1
    assert chosen.value == -7


@pytest.mark.parametrize("n,kind,param,frag", [
    (512, 0, 0.0, b"256"),
    (64, 4, 0.0, b"table"),
    (64, 1, -800.0, b"finite"),   # exp(800 |k|) overflows on the retained set
    (256, 2, -400.0, b"finite"),  # |k|^800 overflows at |k| = sqrt(2) 85
    (64, 1, float("inf"), b"finite"),
])
def test_static_control_map_rejects_on_the_host(lib, n, kind, param, frag):
    """da_omega_from_control_static validates sizes and kernels before any
    device work, so it answers DA_EINVAL here without a GPU."""
    from paper_2602_14016_gb300 import _native as N

    k = N.Kernel(kind, param, None)
    msg = ctypes.c_char_p()
    dummy = ctypes.c_void_p(16)
    st = lib.da_omega_from_control_static(n, 1e-2, ctypes.byref(k), dummy, dummy, None, ctypes.byref(msg))
    assert st == N.DA_EINVAL and frag in msg.value, msg.value
