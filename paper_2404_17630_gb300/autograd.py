"""torch.autograd.Function over one RT step (forward: rt_step; backward:
rt_adjoint with checkpoints every k subcycles).

Differentiable inputs: the source rates Q [n_src, B] (photons/s) and the
hydrogen densities n_H [C] (cm^-3).  Outputs: N [B, C], F [B, 3, C],
x5 [5, C], T [C] after the step.  The initial radiation and abundances are
held fixed (passed as plain tensors).  The backward pass restores the
initial state and calls the library's reverse mode, which recomputes the
forward segment by segment; nothing of the forward is kept on the device
between the two passes beyond the inputs.
"""
from __future__ import annotations

import torch

from . import rt as rtb


class RTStepFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Q, nH, rt, cells, N0, F0, x50, T0, dt, n_sub, checkpoint_every):
        dev = Q.device
        B, C = rt.B, rt.C
        rt.set_sources(cells, Q.detach().double())
        rt.set_gas(nH.detach().double(), x50, T0)
        rt.set_radiation(N0, F0)
        rt.step(dt, n_sub)
        rt.sync()
        N = torch.empty((B, C), dtype=torch.float64, device=dev)
        F = torch.empty((B, 3, C), dtype=torch.float64, device=dev)
        x5 = torch.empty((5, C), dtype=torch.float64, device=dev)
        T = torch.empty((C,), dtype=torch.float64, device=dev)
        rtb.rt_get_fields(rt.ctx, rtb.RT_FIELD_N | rtb.RT_FIELD_F | rtb.RT_FIELD_X | rtb.RT_FIELD_T, [N, F, x5, T])
        ctx.rt, ctx.cells, ctx.dt, ctx.n_sub, ctx.k = rt, cells, dt, n_sub, checkpoint_every
        ctx.save_for_backward(Q, nH, N0, F0, x50, T0)
        return N, F, x5, T

    @staticmethod
    def backward(ctx, gN, gF, gx5, gT):
        Q, nH, N0, F0, x50, T0 = ctx.saved_tensors
        rt = ctx.rt
        rt.set_sources(ctx.cells, Q.detach().double())
        rt.set_gas(nH.detach().double(), x50, T0)
        rt.set_radiation(N0, F0)
        dQ = torch.empty(Q.shape, dtype=torch.float64, device=Q.device)
        dnH = torch.empty(nH.shape, dtype=torch.float64, device=nH.device)
        z = lambda g: None if g is None else g.contiguous().double()
        rtb.rt_adjoint(rt.ctx, ctx.dt, ctx.n_sub, ctx.k, z(gN), z(gF), z(gx5), z(gT), dQ, dnH)
        return dQ.to(Q.dtype), dnH.to(nH.dtype), None, None, None, None, None, None, None, None, None


def rt_step_autograd(rt, cells, Q, nH, N0, F0, x50, T0, dt, n_sub, checkpoint_every):
    """Differentiable RT step; see RTStepFunction."""
    return RTStepFunction.apply(Q, nH, rt, cells, N0, F0, x50, T0, dt, n_sub, checkpoint_every)
