"""The allocation-free control map, for callers that cannot call cudaMalloc.

da_omega_from_control_static computes the control map of one member with
its scratch in a static device array instead of context buffers, so a
caller whose device memory is owned by someone else (a host framework's
pool, a serving loop that must not allocate once running) can still use
it.  This file is collected last so that a failure here leaves every other
test already run.  Each case calls the entry point twice in a row, with
different inputs, and compares both results with the context entry point
da_omega_from_control within the control-map tolerance of the parity tests.
"""
import ctypes

import numpy as np
import pytest

from paper_2602_14016_gb300 import synthetic

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-13


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a GPU")
    from paper_2602_14016_gb300 import _native, build

    build.build()
    return _native.load()


def static_map(lib, n, nu, kind, param, s):
    from paper_2602_14016_gb300 import _native as N

    out = torch.empty((n, n // 2 + 1), dtype=torch.complex128, device="cuda")
    k = N.Kernel(N.KERNEL_KINDS[kind], param, None)
    msg = ctypes.c_char_p()
    st = lib.da_omega_from_control_static(n, nu, ctypes.byref(k), ctypes.c_void_p(s.data_ptr()),
                                          ctypes.c_void_p(torch.view_as_real(out).data_ptr()),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(msg))
    assert st == N.DA_OK, msg.value
    return out


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("n,kind,param", [(16, "identity", 0.0), (64, "exp_abs", 0.5), (128, "frac", 0.5),
                                          (256, "exp_sq", 0.7), (256, "frac", 1.5)])
def test_static_control_map_matches_context_path(lib, n, kind, param):
    from paper_2602_14016_gb300 import api

    nu = 1e-2
    cfg = api.Config(n=n, nsteps=1, dt=1e-3, nu=nu, px=8, every=1, kernels=[api.KernelSpec(kind, param)],
                     store=False)
    ctx = api.Context(cfg)
    for call in range(2):  # two calls in a row, different inputs
        s = torch.from_numpy(synthetic.random_field(n, 100 + call)).cuda()
        ref = ctx.omega_from_control(s[None])[0]
        out = static_map(lib, n, nu, kind, param, s)
        torch.cuda.synchronize()
        assert rel(out, ref) < TOL, (call, rel(out, ref))
    ctx.close()


def test_static_control_map_rejects_sizes_beyond_its_scratch(lib):
    from paper_2602_14016_gb300 import _native as N

    k = N.Kernel(0, 0.0, None)
    msg = ctypes.c_char_p()
    dummy = ctypes.c_void_p(1)
    st = lib.da_omega_from_control_static(512, 1e-2, ctypes.byref(k), dummy, dummy, None, ctypes.byref(msg))
    assert st == N.DA_EINVAL and b"256" in msg.value


def test_static_control_map_from_two_threads(lib):
    """Two host threads, each on its own stream, take turns (calls that
    overlap on the GPU would race on the shared scratch); every result
    matches the context entry point."""
    import threading

    from paper_2602_14016_gb300 import api

    n, nu, kind, param = 64, 1e-2, "exp_abs", 0.5
    lock = threading.Lock()
    fields = {i: torch.from_numpy(synthetic.random_field(n, 200 + i)).cuda() for i in range(2)}
    out = {}

    def work(i):
        st = torch.cuda.Stream()
        for rep in range(3):
            with lock:
                with torch.cuda.stream(st):
                    r = static_map(lib, n, nu, kind, param, fields[i])
                st.synchronize()
            out[(i, rep)] = r

    th = [threading.Thread(target=work, args=(i,)) for i in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    ctx = api.Context(api.Config(n=n, nsteps=1, dt=1e-3, nu=nu, px=8, every=1,
                                 kernels=[api.KernelSpec(kind, param)], store=False))
    for i in range(2):
        ref = ctx.omega_from_control(fields[i][None])[0]
        torch.cuda.synchronize()
        for rep in range(3):
            assert rel(out[(i, rep)], ref) < TOL
    ctx.close()
