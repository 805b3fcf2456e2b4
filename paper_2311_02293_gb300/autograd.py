"""torch.autograd.Function around the library's forward modelling and its
exact discrete adjoint (SMIwiz, arXiv 2311.02293, Secs. 2.2 and 4.2).

``seismograms(vp, rho, prob, srcs, recs, stf)`` returns the flat seismogram
tensor of all shots (shot s occupies nt * nrec_s samples, receiver fastest).
The forward pass runs ``smi_forward_tape``, which keeps the saved boundaries
and the final wavefield state on the device (the boundary-saving strategy of
Sec. 4.2 is the checkpoint; no wavefield history is stored); the backward
pass runs only the reverse loop from that tape (``Tape.vjp``: adjoint field
driven by the upstream gradient, source field reconstructed backwards,
dL/dVp accumulated) -- three modellings per gradient, no forward re-run.
The density is held fixed (no gradient).  Inputs must be CUDA tensors.
"""
from __future__ import annotations

import torch

from . import smi


class SeismogramFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vp, rho, prob, srcs, recs, stf):
        if ctx.needs_input_grad[0]:
            seis, ctx.tape = smi.smi_forward_tape(vp.detach(), rho.detach(), prob, srcs, recs, stf.detach())
        else:
            seis, ctx.tape = smi.smi_forward(vp, rho, prob, srcs, recs, stf, flat=True), None
        return seis

    @staticmethod
    def backward(ctx, grad_seis):
        grad_vp = None
        if ctx.tape is not None:
            g = grad_seis.detach().contiguous().float()
            grad_vp = ctx.tape.vjp(g)
            ctx.tape.free()
            ctx.tape = None
        return grad_vp, None, None, None, None, None


def seismograms(vp, rho, prob, srcs, recs, stf):
    """Differentiable (w.r.t. vp) seismograms of every shot, flat."""
    return SeismogramFn.apply(vp, rho, prob, srcs, recs, stf)


def misfit(vp, rho, prob, srcs, recs, stf, dobs_flat):
    """J = 1/2 sum (u - d)^2 in FP64 (Eq. objfwi), differentiable w.r.t. vp."""
    u = seismograms(vp, rho, prob, srcs, recs, stf)
    r = u.double() - dobs_flat.double()
    return 0.5 * torch.sum(r * r)
