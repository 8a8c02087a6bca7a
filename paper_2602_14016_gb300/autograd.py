"""Differentiation through the window: a torch.autograd.Function whose
forward is the CUDA forward solve (da_forward, which keeps the stage fields
or checkpoints) and whose backward is the hand-written discrete adjoint
(da_vjp), i.e. the adjoint equations of Eq. (11) driven by whatever
cotangents the caller's loss produces.

Outputs of `solve(s)`:
  obs      (B, nt, P*P, 2) float64  model velocities at the probes (Eq. 3)
  omega_T  (B, n, n//2+1) complex128 final vorticity half spectrum
Both are differentiable with respect to the control s (B, n, n).
"""
from __future__ import annotations

import torch

from .api import Context


def _cotangent_of_half_spectrum(g: torch.Tensor, n: int) -> torch.Tensor:
    """Converts torch's gradient of a real loss with respect to half-spectrum
    entries z (g = dL/dRe z + i dL/dIm z) into the DFT of the gradient with
    respect to the grid values, the convention of da_vjp.

    L depends on the grid field w through z_k = sum_x w(x) e^{-i k.x} for k in
    the half spectrum H, so dL/dw(x) = Re sum_{k in H} g_k e^{i k.x}, whose DFT
    is (n^2/2) (g_k + conj g_{-k} [-k in H]).  Only the kx = 0 and kx = n/2
    columns hold both k and -k."""
    out = g * (n * n / 2.0)
    for p in (0, n // 2):
        col = g[..., :, p]
        refl = torch.conj(torch.roll(torch.flip(col, dims=[-1]), shifts=1, dims=-1))
        out[..., :, p] = (col + refl) * (n * n / 2.0)
    return out


class _Window(torch.autograd.Function):
    @staticmethod
    def forward(ctx, s: torch.Tensor, context: Context):
        wT, obs = context.forward(s.contiguous())
        ctx.context = context
        return obs, wT

    @staticmethod
    def backward(ctx, g_obs, g_wT):
        context: Context = ctx.context
        n = context.cfg.n
        dobs = g_obs.contiguous() if g_obs is not None else None
        dwT = _cotangent_of_half_spectrum(g_wT, n).contiguous() if g_wT is not None else None
        if dobs is None and dwT is None:
            return None, None
        return context.vjp(dobs=dobs, dwT=dwT), None


def solve(s: torch.Tensor, context: Context):
    """Differentiable forward window: returns (obs, omega_T) of controls s.

    The context must keep its trajectory (Config.store = True; any
    ckpt_every).  One backward per forward."""
    return _Window.apply(s, context)


def misfit(obs: torch.Tensor, m: torch.Tensor) -> torch.Tensor:
    """J = 1/2 sum |obs - m|^2 per member (Eq. 2-3), as a torch expression."""
    r = obs - m
    return 0.5 * (r * r).sum(dim=tuple(range(1, r.dim())))
