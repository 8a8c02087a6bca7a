"""PyTorch-facing wrapper of the C ABI (device memory and streams only).

Every method marshals torch tensors into the library's entry points; all
arithmetic runs in the library's CUDA kernels.  Shapes follow include/da.h:
controls and gradients (B, n, n) float64, spectra (B, n, n//2+1) complex128,
observations (B, nt, px*px, 2) float64, all on the context's CUDA device.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field
from typing import NamedTuple

import torch

from . import _native as N


@dataclass
class KernelSpec:
    """Fourier kernel W(k) of the preconditioner (Sec. III.B)."""

    kind: str = "identity"  # identity | exp_abs | frac | exp_sq | table
    param: float = 0.0
    table: "object | None" = None  # numpy float64 [n][n/2+1] for kind "table"


@dataclass
class Config:
    n: int
    nsteps: int
    dt: float
    nu: float
    forcing: str = "none"  # none | kolmogorov
    amp: float = 1.0
    nf: int = 4
    px: int = 8
    every: int = 10
    include_t0: bool = False
    kernels: list = field(default_factory=lambda: [KernelSpec()])
    store: bool = True  # keep the trajectory for the adjoint (False: forward only)
    ckpt_every: int = 0  # 0: stage fields of every step; K > 0: checkpoint every K steps

    @property
    def batch(self) -> int:
        return len(self.kernels)

    @property
    def nt(self) -> int:
        return self.nsteps // self.every + (1 if self.include_t0 else 0)


def _stream(stream=None) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor | None) -> ctypes.c_void_p | None:
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("tensors must be contiguous CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


def plan_flops(n: int, variant: int = 0) -> tuple[float, float]:
    """Nominal flops of one band-limited (inverse, forward) transform of n
    points as the pass kernels run it under plan `variant` (da_plan_flops)."""
    lib = N.load()
    inv, fwd = ctypes.c_double(), ctypes.c_double()
    st = lib.da_plan_flops(int(n), int(variant), ctypes.byref(inv), ctypes.byref(fwd))
    if st != N.DA_OK:
        raise N.DAError(st, (lib.da_last_error(None) or b"").decode())
    return inv.value, fwd.value


class AssimResult(NamedTuple):
    J_hist: "object"  # numpy [B, max_iter+1]
    iters: "object"  # numpy int32 [B]
    status: int  # status of the call (worst over members)
    member_status: "object"  # numpy int32 [B]


class Context:
    """One da_ctx: a batch of assimilation windows sharing grid and physics."""

    def __init__(self, cfg: Config, device: int | torch.device | None = None):
        self.cfg = cfg
        self.lib = N.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        g = N.Grid(cfg.n, 0.0, cfg.dt, cfg.nsteps, cfg.ckpt_every if cfg.store else -1, cfg.batch)
        f = N.Forcing(1 if cfg.forcing == "kolmogorov" else 0, cfg.amp, cfg.nf)
        o = N.ObsOperator(cfg.px, cfg.px, cfg.every, int(cfg.include_t0))
        ks = (N.Kernel * cfg.batch)()
        self._tables = []
        for i, k in enumerate(cfg.kernels):
            tab = None
            if k.kind == "table":
                import numpy as np

                tab = np.ascontiguousarray(k.table, dtype=np.float64)
                self._tables.append(tab)
            ks[i] = N.Kernel(N.KERNEL_KINDS[k.kind], float(k.param), tab.ctypes.data if tab is not None else None)
        ctx = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = self.lib.da_create(ctypes.byref(ctx), ctypes.byref(g), cfg.nu, ctypes.byref(f), ctypes.byref(o), ks)
        N.check(st, None)
        self.ctx = ctx
        self.nt = self.lib.da_num_obs_times(ctx)

    # -- helpers ------------------------------------------------------------
    def _phys(self):
        return torch.empty((self.cfg.batch, self.cfg.n, self.cfg.n), dtype=torch.float64, device=self.device)

    def _spec(self):
        n = self.cfg.n
        return torch.empty((self.cfg.batch, n, n // 2 + 1), dtype=torch.complex128, device=self.device)

    def _obs(self):
        return torch.empty((self.cfg.batch, self.nt, self.cfg.px * self.cfg.px, 2), dtype=torch.float64,
                           device=self.device)

    def _check(self, st):
        N.check(st, self.ctx)

    # -- entry points ---------------------------------------------------------
    def set_sobolev(self, lam: float):
        """Regularisation lambda/2 sum |grad u0|^2 of Eq. (4) (0: off)."""
        self._check(self.lib.da_set_sobolev(self.ctx, float(lam)))

    def set_graphs(self, enable: bool = True):
        """Replay da_cost_grad as a captured CUDA graph."""
        self._check(self.lib.da_set_graphs(self.ctx, int(enable)))

    def set_observations(self, m: torch.Tensor, stream=None):
        m = m.to(self.device, torch.float64).contiguous()
        assert m.numel() == self.cfg.batch * self.nt * self.cfg.px ** 2 * 2
        self._m = m
        self._check(self.lib.da_set_observations(self.ctx, _ptr(m), _stream(stream)))

    def forward(self, s: torch.Tensor, stream=None):
        """(omega_T half spectrum, model observations)."""
        s = s.contiguous()
        wT, obs = self._spec(), self._obs()
        self._check(self.lib.da_forward(self.ctx, _ptr(s), _ptr(torch.view_as_real(wT)), _ptr(obs), _stream(stream)))
        return wT, obs

    @property
    def plan(self) -> int:
        """Current FFT plan variant of the pass kernels."""
        return int(self.lib.da_get_plan(self.ctx))

    def set_plan(self, variant: int) -> None:
        self._check(self.lib.da_set_plan(self.ctx, int(variant)))

    def autotune(self, steps: int = 8):
        """Time every FFT plan variant of this grid on this batch and keep the
        fastest (also for later contexts of the same grid and batch).
        Returns (chosen variant, [ms per RK step of each variant])."""
        nv = int(self.lib.da_plan_count(self.cfg.n))
        chosen = ctypes.c_int(-1)
        ms = (ctypes.c_double * nv)()
        self._check(self.lib.da_autotune(self.ctx, int(steps), ctypes.byref(chosen), ms))
        return chosen.value, [float(x) for x in ms]

    def cost_grad(self, s: torch.Tensor, stream=None, J_on_device: bool = True):
        """(J [B], grad_s [B, n, n])."""
        s = s.contiguous()
        g = self._phys()
        J = torch.empty(self.cfg.batch, dtype=torch.float64, device=self.device)
        self._check(self.lib.da_cost_grad(self.ctx, _ptr(s), _ptr(J), _ptr(g), _stream(stream)))
        return J, g

    def cost_grad_host(self, s_host: torch.Tensor, stream=None):
        """End-to-end call from host memory: copies s in, returns (J, grad) on the host."""
        s = s_host.to(self.device, non_blocking=True)
        J, g = self.cost_grad(s, stream)
        return J.cpu(), g.cpu()

    def vjp(self, dobs: torch.Tensor | None = None, dwT: torch.Tensor | None = None, stream=None):
        """Gradient in s of <dobs, obs> + <dwT, omega_T> at the last forward."""
        g = self._phys()
        if dobs is not None:
            dobs = dobs.to(self.device, torch.float64).contiguous()
        dw = None
        if dwT is not None:
            dw = torch.view_as_real(dwT.to(self.device, torch.complex128).contiguous())
        self._check(self.lib.da_vjp(self.ctx, _ptr(dobs), _ptr(dw), _ptr(g), _stream(stream)))
        return g

    def last_adjoint(self, stream=None):
        """(lambda_0 half spectrum, G-metric gradient) of the last adjoint run."""
        lam0, filt = self._spec(), self._phys()
        self._check(self.lib.da_last_adjoint(self.ctx, _ptr(torch.view_as_real(lam0)), _ptr(filt), _stream(stream)))
        return lam0, filt

    def adjoint_terminal(self, s: torch.Tensor, lamT: torch.Tensor, stream=None):
        s = s.contiguous()
        lamT = lamT.to(self.device, torch.complex128).contiguous()
        g = self._phys()
        self._check(self.lib.da_adjoint_terminal(self.ctx, _ptr(s), _ptr(torch.view_as_real(lamT)), _ptr(g),
                                                 _stream(stream)))
        return g

    def adjoint_spectra(self, s: torch.Tensor, lamT: torch.Tensor, save_every: int, stream=None):
        """Shell energies of the adjoint velocity every save_every steps of
        backward time: (per member [B, nsave, nshell], ensemble mean [nsave, nshell])."""
        nshell = self.lib.da_num_shells(self.ctx)
        nsave = self.cfg.nsteps // save_every + 1
        member = torch.empty((self.cfg.batch, nsave, nshell), dtype=torch.float64, device=self.device)
        mean = torch.empty((nsave, nshell), dtype=torch.float64, device=self.device)
        lamT = torch.view_as_real(lamT.to(self.device, torch.complex128).contiguous())
        self._check(self.lib.da_adjoint_spectra(self.ctx, _ptr(s.contiguous()), _ptr(lamT), save_every, _ptr(member),
                                                _ptr(mean), _stream(stream)))
        return member, mean

    def assimilate(self, s: torch.Tensor, max_iter: int, memory: int = 10, c1: float = 1e-4, c2: float = 0.9,
                   gtol_rel: float = 1e-10, max_ls_evals: int = 20, stream=None, raise_on_notconv: bool = False,
                   raise_on_diverged: bool = False):
        """L-BFGS on s (updated in place).  Returns an AssimResult: J_hist
        [B, max_iter+1], iters [B], the call's status and member_status [B]
        (DA_OK, DA_ENOTCONV or DA_EDIVERGED per member).  A member that
        diverges or whose line search fails does not discard the others'
        results; raise_on_* turn those statuses into a DAError."""
        import numpy as np

        assert s.is_contiguous() and s.dtype == torch.float64
        J = np.zeros((self.cfg.batch, max_iter + 1), np.float64)
        it = np.zeros(self.cfg.batch, np.int32)
        ms = np.zeros(self.cfg.batch, np.int32)
        o = N.LbfgsOpts(memory, c1, c2, gtol_rel, max_ls_evals)
        st = self.lib.da_assimilate(self.ctx, _ptr(s), max_iter, ctypes.byref(o), J.ctypes.data, it.ctypes.data,
                                    ms.ctypes.data, _stream(stream))
        if (st not in (N.DA_OK, N.DA_ENOTCONV, N.DA_EDIVERGED) or (raise_on_notconv and st == N.DA_ENOTCONV)
                or (raise_on_diverged and st == N.DA_EDIVERGED)):
            self._check(st)
        return AssimResult(J, it, st, ms)

    # -- ragged batches and the stepwise optimiser -------------------------
    def set_member(self, member: int, nsteps: int, px: int = 8, nu: float = 1e-3, forcing: bool = False,
                   kernel: "KernelSpec | None" = None, m: "torch.Tensor | None" = None, stream=None):
        """Gives member slot `member` its own window (nsteps 0: idle), kernel and
        observations m [nt, px*px, 2]; the context becomes a ragged batch."""
        import numpy as np

        w = N.MemberWindow(int(nsteps), int(px), float(nu), int(bool(forcing)))
        kernel = kernel or KernelSpec()
        tab = None
        if kernel.kind == "table":
            tab = np.ascontiguousarray(kernel.table, dtype=np.float64)
        k = N.Kernel(N.KERNEL_KINDS[kernel.kind], float(kernel.param), tab.ctypes.data if tab is not None else None)
        mp = None
        if nsteps > 0:
            m = m.to(self.device, torch.float64).contiguous()
            self._keep = m  # the copy is asynchronous
            mp = _ptr(m)
        self._check(self.lib.da_set_member(self.ctx, int(member), ctypes.byref(w), ctypes.byref(k), mp,
                                           _stream(stream)))

    def lbfgs_start(self, member: int, s0: torch.Tensor, max_iter: int, memory: int = 10, c1: float = 1e-4,
                    c2: float = 0.9, gtol_rel: float = 1e-10, max_ls_evals: int = 20, stream=None):
        """Starts the optimiser of member slot `member` at s0 [n, n]."""
        s0 = s0.contiguous()
        o = N.LbfgsOpts(memory, c1, c2, gtol_rel, max_ls_evals)
        self._check(self.lib.da_lbfgs_start(self.ctx, int(member), _ptr(s0), int(max_iter), ctypes.byref(o),
                                            _stream(stream)))

    def lbfgs_iterate(self, stream=None) -> int:
        """One step (one shared evaluation); returns the number of members still running."""
        running = ctypes.c_int(0)
        self._check(self.lib.da_lbfgs_iterate(self.ctx, ctypes.byref(running), _stream(stream)))
        return running.value

    def lbfgs_member(self, member: int, hist_len: int = 0, control: bool = False, stream=None):
        """(report dict, J history [hist_len] or None, control [n, n] or None)."""
        import numpy as np

        rep = N.LbfgsReport()
        hist = np.zeros(hist_len, np.float64) if hist_len > 0 else None
        s = torch.empty((self.cfg.n, self.cfg.n), dtype=torch.float64, device=self.device) if control else None
        self._check(self.lib.da_lbfgs_member(self.ctx, int(member), ctypes.byref(rep),
                                             hist.ctypes.data if hist is not None else None, int(hist_len),
                                             _ptr(s), _stream(stream)))
        report = {"phase": rep.phase, "status": rep.status, "iters": rep.iters, "J0": rep.J0, "J": rep.J}
        return report, hist, s

    def lbfgs_release(self, member: int):
        self._check(self.lib.da_lbfgs_release(self.ctx, int(member)))

    def omega_from_control(self, s: torch.Tensor, stream=None):
        w = self._spec()
        self._check(self.lib.da_omega_from_control(self.ctx, _ptr(s.contiguous()), _ptr(torch.view_as_real(w)),
                                                   _stream(stream)))
        return w

    def control_from_omega(self, w0: torch.Tensor, stream=None):
        s = self._phys()
        w0 = w0.to(self.device, torch.complex128).contiguous()
        self._check(self.lib.da_control_from_omega(self.ctx, _ptr(torch.view_as_real(w0)), _ptr(s), _stream(stream)))
        return s

    KERNEL_CLASSES = {"off": 0, "fwd_rows": 1, "fwd_cols": 2, "adj_rows": 3, "adj_cols": 4}

    def time_kernels(self, kernel_class: str):
        """Bracket every launch of one pass-kernel class with CUDA events."""
        self._check(self.lib.da_time_kernels(self.ctx, self.KERNEL_CLASSES[kernel_class]))

    def kernel_time(self):
        """(total ms, launches) of the timed class since the last call."""
        ms = ctypes.c_double()
        cnt = ctypes.c_ulonglong()
        self._check(self.lib.da_kernel_time(self.ctx, ctypes.byref(ms), ctypes.byref(cnt)))
        return ms.value, int(cnt.value)

    @property
    def device_bytes(self) -> int:
        return int(self.lib.da_device_bytes(self.ctx))

    @property
    def launches(self) -> int:
        return int(self.lib.da_launch_count(self.ctx))

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.da_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
