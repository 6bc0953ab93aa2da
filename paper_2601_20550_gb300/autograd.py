"""torch.autograd wrapper of the 2D-spectrum misfit gradient.

``SpectrumMisfit.apply(theta, model, grid, S_ref, ckpt_every)`` returns the
scalar misfit sum (S_C(theta) - S_ref)^2 of the model description with its
twelve gradient parameters (see ``heom.theta_of``) set from ``theta``; its
backward pass returns the gradient that heom_response_2d_grad computed in the
same call (discrete adjoint on the GPU).  Every call rebuilds the hierarchy and
the equilibrium for the given theta in FP64.
"""
import numpy as np
import torch

from . import heom as H


class SpectrumMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, model, grid, S_ref, ckpt_every=64):
        m = H.with_theta(model, theta.detach().cpu().double().numpy())
        h = H.heom_build_hierarchy(m, H.FP64)
        eq = H.heom_equilibrate(h, grid["dt_fs"], grid["t_eq_fs"], 0.0)
        loss, g = H.heom_response_2d_grad(h, eq, grid, np.asarray(S_ref), ckpt_every)
        ctx.save_for_backward(torch.as_tensor(g, dtype=theta.dtype, device=theta.device))
        return theta.new_tensor(loss)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None, None, None
