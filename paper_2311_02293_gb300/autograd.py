"""torch.autograd.Function around the library's forward modelling and its
exact discrete adjoint (SMIwiz, arXiv 2311.02293, Secs. 2.2 and 4.2).

``seismograms(vp, rho, prob, srcs, recs, stf)`` returns the flat seismogram
tensor of all shots (shot s occupies nt * nrec_s samples, receiver fastest).
Its backward pass calls ``smi_forward_vjp``: the forward modelling is run
again saving the boundaries, and the adjoint field driven by the upstream
gradient accumulates dL/dVp -- the saved boundaries are the checkpoint
(Sec. 4.2), no wavefield history is stored.  The density is held fixed (no
gradient).  Inputs must be CUDA tensors.
"""
from __future__ import annotations

import torch

from . import smi


class SeismogramFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vp, rho, prob, srcs, recs, stf):
        seis = smi.smi_forward(vp, rho, prob, srcs, recs, stf, flat=True)
        ctx.save_for_backward(vp, rho, stf)
        ctx.prob, ctx.srcs, ctx.recs = prob, srcs, recs
        return seis

    @staticmethod
    def backward(ctx, grad_seis):
        vp, rho, stf = ctx.saved_tensors
        grad_vp = None
        if ctx.needs_input_grad[0]:
            g = grad_seis.detach().contiguous().float()
            grad_vp = smi.smi_forward_vjp(vp.detach(), rho.detach(), ctx.prob, ctx.srcs, ctx.recs,
                                          stf.detach(), g).to(vp.dtype)
        return grad_vp, None, None, None, None, None


def seismograms(vp, rho, prob, srcs, recs, stf):
    """Differentiable (w.r.t. vp) seismograms of every shot, flat."""
    return SeismogramFn.apply(vp, rho, prob, srcs, recs, stf)


def misfit(vp, rho, prob, srcs, recs, stf, dobs_flat):
    """J = 1/2 sum (u - d)^2 in FP64 (Eq. objfwi), differentiable w.r.t. vp."""
    u = seismograms(vp, rho, prob, srcs, recs, stf)
    r = u.double() - dobs_flat.double()
    return 0.5 * torch.sum(r * r)
