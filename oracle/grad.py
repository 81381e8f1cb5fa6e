"""Gradient oracle: the GFK walk in plain PyTorch (CPU, FP64) with autograd.

TEST INFRASTRUCTURE ONLY (tests and the smoke check call it).  It shares no
code with the CUDA library.  Everything follows the definitions:
  ln psi = -Z (r1 + r2) + u(r12),  u(r) = a rho + sum_k c_k rho^{k+1},
  rho = r / (1 + beta r)                      (the Jastrow-product trial function)
  b = grad ln psi,  E_L = -(lap ln psi + |grad ln psi|^2) / 2 + V
  (the GFK split before Eq. 4: V_P = E_L - E_T), V = -2/r1 - 2/r2 + 1/r12,
with the drift and the Laplacian taken by autograd from ln psi itself; the walk
X_{n+1} = X_n + b(X_n) dt + sqrt(dt) xi_n (the SDE under Eq. 4), log-weights
by the right-point rule, and the space-averaged loss at the last step.  The
normals are the C oracle's Philox / Box-Muller stream (pinned separately), so
the trajectories are the C oracle's; with noise = 1 the increments are the C
oracle's Bernoulli +-1 steps from each walker's Superduper generator.
d(loss)/d(theta) is autograd's.

Parity status: pinned by tests/test_oracle_pins.py (drift and E_L equal the C
oracle's at random points; the loss equals the C oracle walk's E(t_S); the
autograd gradient equals central finite differences of this loss).
"""
from __future__ import annotations

import numpy as np
import torch

from . import init_normals, move_bernoulli, move_normals

THETA_NAMES = ("Z", "a", "beta", "c1", "c2", "c3", "c4")


def lnpsi(X: torch.Tensor, theta: torch.Tensor) -> torch.Tensor:
    theta = theta.to(torch.float64)            # all arithmetic in FP64
    Z, a, beta = theta[0], theta[1], theta[2]
    r1 = torch.linalg.norm(X[:, :3], dim=1)
    r2 = torch.linalg.norm(X[:, 3:], dim=1)
    r12 = torch.linalg.norm(X[:, :3] - X[:, 3:], dim=1)
    rho = r12 / (1.0 + beta * r12)
    u = a * rho
    for k in range(4):
        u = u + theta[3 + k] * rho ** (k + 2)
    return -Z * (r1 + r2) + u


def drift_and_local_energy(X: torch.Tensor, theta: torch.Tensor, ee_on: bool = True):
    """b = grad ln psi and E_L = -(lap ln psi + |b|^2)/2 + V, by autograd (graph kept)."""
    if not X.requires_grad:
        X = X.requires_grad_(True)
    lp = lnpsi(X, theta).sum()
    b = torch.autograd.grad(lp, X, create_graph=True)[0]
    lap = torch.zeros(X.shape[0], dtype=X.dtype)
    for d in range(6):
        lap = lap + torch.autograd.grad(b[:, d].sum(), X, create_graph=True)[0][:, d]
    r1 = torch.linalg.norm(X[:, :3], dim=1)
    r2 = torch.linalg.norm(X[:, 3:], dim=1)
    r12 = torch.linalg.norm(X[:, :3] - X[:, 3:], dim=1)
    V = -2.0 / r1 - 2.0 / r2 + (1.0 / r12 if ee_on else 0.0)
    el = -0.5 * (lap + (b * b).sum(dim=1)) + V
    return b, el


def walk_loss(theta, *, n_walkers, n_steps, dt, e_trial, seed, inst=0, sigma=0.5,
              loss_kind=0, ee_on=True, noise=0):
    """The walk from a fresh population and its loss at the last step (differentiable
    in theta): loss 0 = sum w E_L / sum w, loss 1 = the weighted variance of E_L."""
    n = int(n_walkers)
    X = torch.tensor(np.array([sigma * init_normals(seed, i, inst) for i in range(n)]),
                     dtype=torch.float64)
    logw = torch.zeros(n, dtype=torch.float64)
    b, el = drift_and_local_energy(X, theta, ee_on)
    sdt = float(np.sqrt(dt))
    for step in range(n_steps):
        draw = move_bernoulli if noise == 1 else move_normals
        xi = torch.tensor(np.array([draw(seed, i, step, inst) for i in range(n)]),
                          dtype=torch.float64)
        X = X + b * dt + sdt * xi
        b, el = drift_and_local_energy(X, theta, ee_on)
        logw = logw - (el - e_trial) * dt
    w = torch.exp(logw - logw.max().detach())
    W = w.sum()
    L = (w * el).sum() / W
    if loss_kind == 0:
        return L
    return (w * el * el).sum() / W - L * L


def gradient(theta0, **kw):
    """(loss, d loss / d theta) with theta = [Z, a, beta, c1, c2, c3, c4]."""
    theta = torch.tensor(np.asarray(theta0, dtype=np.float64), requires_grad=True)
    loss = walk_loss(theta, **kw)
    (g,) = torch.autograd.grad(loss, theta)
    return float(loss.detach()), g.numpy()
