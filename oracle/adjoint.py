"""Float64 torch (CPU) restatement of the force sum and the shared-step Hermite
trajectory, differentiated by torch.autograd -- the oracle's own gradient.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Dense (N, N) pair tensors,
so it is meant for N <= a few hundred.

The force law is the one of sp2_oracle.c (Plummer-softened Newtonian gravity,
G = 1, self pair excluded):
    A_ij = m_j s^3 r,  J_ij = m_j s^3 v - 3 alpha A_ij,  phi_ij = -m_j s,
    s = (r.r + eps^2)^-1/2,  alpha = (r.v) s^2,  r = x_j - x_i,  v = v_j - v_i.
"""
from __future__ import annotations

import torch


def forces(x, v, m, eps2: float):
    """acc, jerk, pot of every particle on every other one (all active)."""
    n = x.shape[0]
    r = x[None, :, :] - x[:, None, :]          # r[i, j] = x_j - x_i
    u = v[None, :, :] - v[:, None, :]
    eye = torch.eye(n, dtype=torch.bool, device=x.device)
    d2 = (r * r).sum(-1) + eps2
    d2 = torch.where(eye, torch.ones_like(d2), d2)  # keep the masked diagonal finite
    s = d2.rsqrt()
    s = torch.where(eye, torch.zeros_like(s), s)
    s2 = s * s
    ms3 = m[None, :] * s * s2
    alpha = (r * u).sum(-1) * s2
    A = ms3[..., None] * r
    J = ms3[..., None] * u - 3.0 * alpha[..., None] * A
    pot = -(m[None, :] * s).sum(1)
    return A.sum(1), J.sum(1), pot


def hermite4_trajectory(x0, v0, m, eps2: float, dt: float, n_steps: int):
    """Shared-step Hermite-4 trajectory; returns (x, v) after n_steps."""
    x, v = x0, v0
    a0, j0, _ = forces(x, v, m, eps2)
    for _ in range(n_steps):
        xp = x + v * dt + a0 * (dt * dt * 0.5) + j0 * (dt * dt * dt / 6.0)
        vp = v + a0 * dt + j0 * (dt * dt * 0.5)
        a1, j1, _ = forces(xp, vp, m, eps2)
        v1 = v + (a0 + a1) * (dt / 2) + (j0 - j1) * (dt * dt / 12)
        x1 = x + (v + v1) * (dt / 2) + (a0 - a1) * (dt * dt / 12)
        x, v, a0, j0 = x1, v1, a1, j1
    return x, v


def loss_and_grad(x0, v0, m, w, eps2: float, dt: float, n_steps: int):
    """L = sum w . x_final and its gradient w.r.t. (x0, v0, m) by autograd."""
    x0 = torch.as_tensor(x0, dtype=torch.float64).clone().requires_grad_(True)
    v0 = torch.as_tensor(v0, dtype=torch.float64).clone().requires_grad_(True)
    m = torch.as_tensor(m, dtype=torch.float64).clone().requires_grad_(True)
    w = torch.as_tensor(w, dtype=torch.float64)
    xf, _ = hermite4_trajectory(x0, v0, m, eps2, dt, n_steps)
    L = (w * xf).sum()
    gx, gv, gm = torch.autograd.grad(L, (x0, v0, m))
    return float(L.detach()), gx.numpy(), gv.numpy(), gm.numpy()


def force_vjp(x, v, m, abar, jbar, pbar, eps2: float):
    """VJP of (acc, jerk, pot) w.r.t. (x, v, m) for given cotangents, by autograd."""
    x = torch.as_tensor(x, dtype=torch.float64).clone().requires_grad_(True)
    v = torch.as_tensor(v, dtype=torch.float64).clone().requires_grad_(True)
    m = torch.as_tensor(m, dtype=torch.float64).clone().requires_grad_(True)
    A, J, P = forces(x, v, m, eps2)
    s = (A * torch.as_tensor(abar)).sum() + (J * torch.as_tensor(jbar)).sum() \
        + (P * torch.as_tensor(pbar)).sum()
    gx, gv, gm = torch.autograd.grad(s, (x, v, m))
    return gx.numpy(), gv.numpy(), gm.numpy()
