"""Dense-matrix statements of the operators, for pinning the oracle on tiny sizes.

These build the matrices straight from their definitions (pixel by pixel), so
that a checked identity does not reuse the oracle's own loops.
"""
from __future__ import annotations

import numpy as np


def phi_matrix(masks: np.ndarray, Z: int, n_shots: int) -> np.ndarray:
    """Phi as an (N*H*W) x (Z*H*W) matrix: shot j sees slices j*R..j*R+R-1 (Sec. III-A)."""
    R = Z // n_shots
    per_slice = masks.shape[0] == Z
    H, W = masks.shape[1:]
    HW = H * W
    P = np.zeros((n_shots * HW, Z * HW))
    for j in range(n_shots):
        for r in range(R):
            m = masks[j * R + r] if per_slice else masks[r]
            for p in range(HW):
                P[j * HW + p, (j * R + r) * HW + p] = m.flat[p]
    return P


def grad_matrix(H: int, W: int) -> np.ndarray:
    """Forward-difference gradient, (2*H*W) x (H*W); zero rows on the last row/column.

    Rows 0..HW-1: component along i (rows); rows HW..2HW-1: along j (columns).
    """
    HW = H * W
    K = np.zeros((2 * HW, HW))
    for i in range(H):
        for j in range(W):
            p = i * W + j
            if i < H - 1:
                K[p, p] = -1.0
                K[p, p + W] = 1.0
            if j < W - 1:
                K[HW + p, p] = -1.0
                K[HW + p, p + 1] = 1.0
    return K


def cyclic_laplacian(Z: int) -> np.ndarray:
    """Graph Laplacian of the cyclic z chain with one edge (n, n-1 mod Z) per slice n."""
    L = np.zeros((Z, Z))
    if Z < 2:
        return L
    for n in range(Z):
        m = (n - 1) % Z
        L[n, n] += 1
        L[m, m] += 1
        L[n, m] -= 1
        L[m, n] -= 1
    return L


def tv_value(u: np.ndarray) -> float:
    """Isotropic TV of one slice with the same forward differences as grad_matrix."""
    H, W = u.shape
    K = grad_matrix(H, W)
    gu = K @ u.ravel()
    return float(np.sum(np.hypot(gu[: H * W], gu[H * W:])))


def chambolle_pock_tv(g: np.ndarray, theta: float, iters: int = 20000) -> np.ndarray:
    """Independent TV-prox solver: primal-dual (Chambolle-Pock 2011) on
    min_u theta*||K u||_{2,1} + 1/2 ||u - g||^2, with the dense K above."""
    H, W = g.shape
    HW = H * W
    K = grad_matrix(H, W)
    L = np.linalg.norm(K, 2)
    sig = tau = 0.99 / L
    u = g.ravel().copy()
    ub = u.copy()
    y = np.zeros(2 * HW)
    gg = g.ravel()
    for _ in range(iters):
        y = y + sig * (K @ ub)
        nrm = np.maximum(1.0, np.hypot(y[:HW], y[HW:]) / theta)
        y = y / np.concatenate([nrm, nrm])
        un = (u - tau * (K.T @ y) + tau * gg) / (1.0 + tau)
        ub = 2 * un - u
        u = un
    return u.reshape(H, W)
