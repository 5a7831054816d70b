"""FP64 oracle of the differentiable unrolled PnP-ADMM (plain PyTorch CPU ops).

TEST INFRASTRUCTURE ONLY (like the rest of oracle/).  It states, in float64
with whole-array torch operations, the unrolled map that the CUDA library
differentiates by hand, and takes its gradient with torch.autograd (a library
primitive), so that the hand-written reverse pass can be compared with it.

The map is Algorithm 1 with two relaxations used for learning masks and
parameters end to end:
  m = sigmoid(logits)  (continuous DMD patterns; diag(Phi Phi^T) = sum_r m_r^2),
  Huber-smoothed TV   h_eps(x) = |x| - eps/2 for |x| > eps, |x|^2/(2 eps) else,
whose prox at h with weight theta (Eq. u-update: theta = lambda / (rho + 2 gamma))
is taken by T projected-gradient steps on its dual from p = 0:
  q = div p - h/theta,  a = p + tau (grad q - (eps/theta) p),  p <- a / max(1, |a|),
  u = h - theta div p.
grad: forward differences, zero on the last row / column; div = -grad^T.
"""
from __future__ import annotations

import torch


def grad2(u: torch.Tensor):
    """Forward differences of [..., H, W]: (along rows, along columns), zero at the end."""
    gx = torch.zeros_like(u)
    gy = torch.zeros_like(u)
    gx[..., :-1, :] = u[..., 1:, :] - u[..., :-1, :]
    gy[..., :, :-1] = u[..., :, 1:] - u[..., :, :-1]
    return gx, gy


def div2(p1: torch.Tensor, p2: torch.Tensor) -> torch.Tensor:
    """div = -grad^T with the same boundary (Chambolle's discretisation)."""
    H, W = p1.shape[-2:]
    a = torch.zeros_like(p1)
    c = torch.zeros_like(p2)
    if H > 1:
        a[..., 0, :] = p1[..., 0, :]
        a[..., 1:H - 1, :] = p1[..., 1:H - 1, :] - p1[..., 0:H - 2, :]
        a[..., H - 1, :] = -p1[..., H - 2, :]
    if W > 1:
        c[..., :, 0] = p2[..., :, 0]
        c[..., :, 1:W - 1] = p2[..., :, 1:W - 1] - p2[..., :, 0:W - 2]
        c[..., :, W - 1] = -p2[..., :, W - 2]
    return a + c


def huber_tv_prox(h: torch.Tensor, theta, T: int, tau: float, eps: float) -> torch.Tensor:
    """T dual projected-gradient steps for min theta*sum h_eps(|grad u|) + 1/2||u-h||^2."""
    p1 = torch.zeros_like(h)
    p2 = torch.zeros_like(h)
    kappa = eps / theta
    for _ in range(T):
        q = div2(p1, p2) - h / theta
        gx, gy = grad2(q)
        a1 = p1 + tau * (gx - kappa * p1)
        a2 = p2 + tau * (gy - kappa * p2)
        nrm = torch.sqrt(torch.clamp(a1 * a1 + a2 * a2, min=1.0))  # max(1, |a|)
        p1, p2 = a1 / nrm, a2 / nrm
    return h - theta * div2(p1, p2)


def unrolled_admm(logits, b, rho, lam, gamma, *, iters: int, T: int, tau: float, eps: float):
    """v^K of the unrolled map.  logits [B,Z,H,W], b [B,H,W]; rho, lam, gamma scalars
    (0-dim tensors when their gradients are wanted)."""
    B, Z, H, W = logits.shape
    m = torch.sigmoid(logits)
    D = (m * m).sum(1)
    u = torch.zeros_like(logits)
    d = torch.zeros_like(logits)
    gam = gamma if Z > 1 else 0.0 * gamma
    theta = lam / (rho + 2 * gam)
    v = None
    for _ in range(iters):
        g = u - d
        e = (b - (m * g).sum(1)) / (rho + D)
        v = g + m * e[:, None]
        w = v + d
        us = [u[:, n] for n in range(Z)]
        for n in range(Z):
            nb = us[(n - 1) % Z] + us[(n + 1) % Z]  # newest values (in-place sweep)
            h = (rho * w[:, n] + gam * nb) / (rho + 2 * gam)
            us[n] = huber_tv_prox(h, theta, T, tau, eps)
        u = torch.stack(us, 1)
        d = w - u
    return v
