"""Trial-parameter gradients as a torch.autograd.Function, and variance-minimising
tuning with Adam (the paper's VQMC step: trial functions whose parameters are
adjusted to minimise the variance of the local energy).

GFKLoss.apply(theta, ...) runs the walk and its adjoint through the C ABI
(gfk_grad): the forward returns the loss, the backward the stored gradient.
Only argument handling lives here; the walk and the adjoint run in the CUDA
kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import gfk

THETA_NAMES = ("Z", "a", "beta", "c1", "c2", "c3", "c4")


class GFKLoss(torch.autograd.Function):
    """loss(theta) of one instance's walk; theta = [Z, a, beta, c1, c2, c3, c4]."""

    @staticmethod
    def forward(ctx, theta, handle, inst, loss_kind, n_steps, ckpt_every):
        th = theta.detach().to(torch.float64).cpu().numpy()
        gfk.gfk_reset(handle)
        gfk.gfk_set_trial(handle, inst, gfk.GFK_TRIAL_JASTROW_PRODUCT, th)
        loss, grad = gfk.gfk_grad(handle, inst, loss_kind, n_steps, ckpt_every)
        ctx.save_for_backward(torch.from_numpy(grad).to(theta.dtype))
        return theta.new_tensor(loss)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None, None, None, None


def tune(handle, inst, theta0, *, steps=50, lr=1e-2, loss_kind=1, n_steps=2000,
         ckpt_every=64, free=(0, 2, 3, 4, 5, 6)):
    """Adam on the free parameters (default: all but a, which keeps the e-e cusp).
    Returns the history [(loss, theta), ...] and the final theta."""
    theta = torch.tensor(np.asarray(theta0, dtype=np.float64), requires_grad=True)
    mask = torch.zeros(7, dtype=torch.float64)
    mask[list(free)] = 1.0
    opt = torch.optim.Adam([theta], lr=lr)
    history = []
    for _ in range(steps):
        opt.zero_grad()
        loss = GFKLoss.apply(theta, handle, inst, loss_kind, n_steps, ckpt_every)
        loss.backward()
        theta.grad.mul_(mask)
        history.append((float(loss.detach()), theta.detach().numpy().copy()))
        opt.step()
    return history, theta.detach().numpy().copy()
