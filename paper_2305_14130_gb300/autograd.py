"""torch.autograd bindings of the extended objective (eq. 8).

``DataMisfit.apply(vp, vs, rho, plan, d_obs, mask)`` returns phi_data (a float64
scalar on the device) and backpropagates through the adjoint-state gradient
computed by the CUDA kernels (eq. 6 for every extended component).  The
gradient is computed eagerly in forward(), because phi is a scalar: the
adjoint needs only the residual, and backward() then scales the stored
gradients by the incoming grad_output.

``Consistency.apply(m, plan, b, bp, sink, eta)`` returns phi_reg of one
parameter field and backpropagates eta^2 W^T P^T P W m (eqs. 8, 11, 12).

``ExtendedFWI.apply(vp, vs, rho, plan, d_obs, eta, b, bp, sink, mask)`` is the
whole extended objective of eq. 8 in one Function: the data term of every
component plus the consistency term of each parameter field with its eta
(b, bp, sink None: the zone-of-influence weights the plan holds).

``extended_objective(...)`` adds both terms for (Vp, Vs, rho) from the two
Functions above.
"""
from __future__ import annotations

import torch


class DataMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vp, vs, rho, plan, d_obs, mask=None):
        phi, gvp, gvs, grho = plan.gradient(vp.detach().contiguous(), vs.detach().contiguous(),
                                            rho.detach().contiguous(), d_obs, mask=mask)
        ctx.save_for_backward(gvp, gvs, grho)
        return phi

    @staticmethod
    def backward(ctx, grad_phi):
        gvp, gvs, grho = ctx.saved_tensors
        s = grad_phi.to(torch.float32)
        return s * gvp, s * gvs, s * grho, None, None, None


class Consistency(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, plan, b, bp, sink, eta):
        g = torch.zeros_like(m)
        phi, g = plan.regularization_grad(m.detach().contiguous(), b, bp, sink, eta, g=g)
        ctx.save_for_backward(g)
        return phi

    @staticmethod
    def backward(ctx, grad_phi):
        (g,) = ctx.saved_tensors
        return grad_phi.to(torch.float32) * g, None, None, None, None, None


def extended_objective(plan, vp, vs, rho, d_obs, eta, b, bp, sink, mask=None):
    """phi_ext = phi_data + sum over (Vp, Vs, rho) of 1/2 eta_p^2 ||(I - S^T S_w) W m~_p||^2."""
    phi = DataMisfit.apply(vp, vs, rho, plan, d_obs, mask)
    for m, e in zip((vp, vs, rho), eta):
        phi = phi + Consistency.apply(m, plan, b, bp, sink, float(e))
    return phi


class ExtendedFWI(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vp, vs, rho, plan, d_obs, eta, b=None, bp=None, sink=None, mask=None):
        ms = [t.detach().contiguous() for t in (vp, vs, rho)]
        phi, gvp, gvs, grho = plan.gradient(*ms, d_obs, mask=mask)
        grads = (gvp, gvs, grho)
        for m, gm, e in zip(ms, grads, eta):
            phi_r, _ = plan.regularization_grad(m, b, bp, sink, float(e), g=gm)
            phi = phi + phi_r
        ctx.save_for_backward(*grads)
        return phi

    @staticmethod
    def backward(ctx, grad_phi):
        s = grad_phi.to(torch.float32)
        gvp, gvs, grho = ctx.saved_tensors
        return s * gvp, s * gvs, s * grho, None, None, None, None, None, None, None
