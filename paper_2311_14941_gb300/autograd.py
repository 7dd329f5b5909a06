"""torch.autograd integration of the chemistry integrator.

``integrate(mech, T0, p, Y0, dt, dlnA, dEa)`` advances every cell over its own dt (chem_integrate) and
returns the final (T, Y).  Its backward pass is the discrete adjoint (chem_adjoint): gradients with
respect to the initial state and to per-reaction shifts of ln A and Ea (description order, the same for
all cells), with the accepted step sizes frozen.  The backward pass integrates again with a tape
(checkpoints every ``ckpt_every`` accepted steps) and walks it back; nothing is kept between the two
passes but the inputs.

All tensors are float64 on the mechanism's CUDA device; Y is species-major [n, N].
"""
from __future__ import annotations

import torch


class ChemIntegrate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mech, T0, p, Y0, dt, dlnA, dEa, rtol, atol, ckpt_every, tape_steps):
        N = T0.numel()
        dev = T0.device
        T = T0.detach().clone().contiguous()
        Y = Y0.detach().clone().contiguous()
        mech.set_params(dlnA.detach().contiguous(), dEa.detach().contiguous())
        hio = torch.zeros(N, dtype=torch.float64, device=dev)
        ns = torch.zeros(N, dtype=torch.int32, device=dev)
        st = torch.zeros(N, dtype=torch.int32, device=dev)
        # the map chem_adjoint differentiates: one warp per cell, plain launch (same arithmetic, so the
        # returned state is bit for bit the one whose gradients backward gives)
        mech.integrate(T, p, Y, dt, hio, ns, st, rtol=rtol, atol=atol, mode=0, warps_per_cell=1, cells_per_warp=1)
        mech.set_params()
        ctx.mech = mech
        ctx.opts = (rtol, atol, ckpt_every, tape_steps)
        ctx.save_for_backward(T0.detach(), p, Y0.detach(), dt, dlnA.detach(), dEa.detach())
        ctx.mark_non_differentiable(st)
        return T, Y, st

    @staticmethod
    def backward(ctx, gT, gY, _gst):
        T0, p, Y0, dt, dlnA, dEa = ctx.saved_tensors
        mech = ctx.mech
        rtol, atol, ckpt_every, tape_steps = ctx.opts
        N = T0.numel()
        dev = T0.device
        gT = torch.zeros(N, dtype=torch.float64, device=dev) if gT is None else gT.contiguous()
        gY = torch.zeros_like(Y0) if gY is None else gY.contiguous()
        T = T0.clone().contiguous()
        Y = Y0.clone().contiguous()
        gA = torch.zeros(mech.R, dtype=torch.float64, device=dev)
        gE = torch.zeros(mech.R, dtype=torch.float64, device=dev)
        gT0 = torch.zeros(N, dtype=torch.float64, device=dev)
        gY0 = torch.zeros_like(Y0)
        st = torch.zeros(N, dtype=torch.int32, device=dev)
        mech.set_params(dlnA.contiguous(), dEa.contiguous())
        mech.adjoint(T, p, Y, dt, gT, gY, gA, gE, st, gT0=gT0, gY0=gY0, rtol=rtol, atol=atol,
                     ckpt_every=ckpt_every, tape_steps=tape_steps)
        mech.set_params()
        return None, gT0, None, gY0, None, gA, gE, None, None, None, None


def integrate(mech, T0, p, Y0, dt, dlnA=None, dEa=None, rtol=1e-6, atol=1e-12, ckpt_every=16, tape_steps=4096):
    """Differentiable chem_integrate.  Returns (T, Y, status)."""
    dev = T0.device
    if dlnA is None:
        dlnA = torch.zeros(mech.R, dtype=torch.float64, device=dev)
    if dEa is None:
        dEa = torch.zeros(mech.R, dtype=torch.float64, device=dev)
    return ChemIntegrate.apply(mech, T0, p, Y0, dt, dlnA, dEa, rtol, atol, ckpt_every, tape_steps)
