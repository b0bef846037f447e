"""torch.autograd form of one stage: f = -div(tau_IB) with tau_IB the stress after
the wall model of Sec. 3.3 (band nodes from the velocity and the per-cell
roughness s = ln z0, solid nodes zero, fluid nodes the given stress).

Differentiable inputs: u, v, w and ln z0.  The given (fluid) stress is data: it
passes through the stage unchanged and receives no gradient.  Both directions
run in the CUDA library (wmibm_wall_stress_force, wmibm_backward).
"""
from __future__ import annotations

import torch


class WallStressForce(torch.autograd.Function):
    @staticmethod
    def forward(ctx, handle, u, v, w, logz0, txx, txy, tyy, tzz, txz, tyz):
        handle.set_log_z0(logz0)
        tau = [t.detach().clone() for t in (txx, txy, tyy, tzz, txz, tyz)]
        f = [torch.empty(handle.shape, dtype=handle.torch_dtype, device=handle.device) for _ in range(3)]
        handle.wall_stress_force(u.detach(), v.detach(), w.detach(), tau, f)
        ctx.handle = handle
        ctx.save_for_backward(u, v, w, logz0)
        return f[0], f[1], f[2]

    @staticmethod
    def backward(ctx, gx, gy, gz):
        u, v, w, logz0 = ctx.saved_tensors
        h = ctx.handle
        g = [torch.zeros(h.shape, dtype=h.torch_dtype, device=h.device) if t is None else t.contiguous()
             for t in (gx, gy, gz)]
        h.set_log_z0(logz0)
        du, dv, dw, ds = (torch.empty(h.shape, dtype=h.torch_dtype, device=h.device) for _ in range(4))
        h.backward(g, (u.detach(), v.detach(), w.detach()), du, dv, dw, ds)
        cast = lambda d, x: d if d.dtype == x.dtype else d.to(x.dtype)
        return (None, cast(du, u), cast(dv, v), cast(dw, w), ds) + (None,) * 6


def wall_stress_force(handle, u, v, w, logz0, tau):
    """(fx, fy, fz) of one stage, differentiable in u, v, w and logz0 (ln z0 per cell).
    tau: the six given stresses (txx, txy, tyy, tzz, txz, tyz); they are not modified."""
    return WallStressForce.apply(handle, u, v, w, logz0, *tau)
