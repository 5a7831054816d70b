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


# ---- BM3D restated with numpy (dense transform matrices, brute-force search) ----

def bm3d_codes(img: np.ndarray) -> np.ndarray:
    """8-bit matching codes, computed in float32 with round-half-to-even."""
    return np.clip(np.rint(img.astype(np.float32) * np.float32(255.0)), 0, 255).astype(np.int64)


def bm3d_refs(n: int) -> list[int]:
    r = list(range(0, n - 8, 3))
    return r + [n - 8]


def bm3d_brute_force_match(img: np.ndarray, tau: int):
    """Every reference's group by exhaustive search: reference first, then up to 15
    positions of the 39x39 window with SSD <= 64 tau in (SSD, linear index) order."""
    H, W = img.shape
    q = bm3d_codes(img)
    groups = []
    for ri in bm3d_refs(H):
        for rj in bm3d_refs(W):
            ref = q[ri:ri + 8, rj:rj + 8]
            cands = []
            for ci in range(max(0, ri - 19), min(H - 8, ri + 19) + 1):
                for cj in range(max(0, rj - 19), min(W - 8, rj + 19) + 1):
                    if (ci, cj) == (ri, rj):
                        continue
                    ssd = int(np.sum((ref - q[ci:ci + 8, cj:cj + 8]) ** 2))
                    if ssd <= 64 * tau:
                        cands.append((ssd, ci * W + cj))
            cands.sort()
            groups.append([ri * W + rj] + [lin for _, lin in cands[:15]])
    return groups


def haar_matrix(L: int) -> np.ndarray:
    """Orthonormal Haar matrix: sums of pairs first (recursively), differences last."""
    if L == 1:
        return np.ones((1, 1))
    Hh = haar_matrix(L // 2)
    top = np.kron(Hh, np.array([[1.0, 1.0]]))
    bot = np.kron(np.eye(L // 2), np.array([[1.0, -1.0]]))
    return np.vstack([top, bot]) / np.sqrt(2.0)


def dct_matrix() -> np.ndarray:
    import scipy.fft

    return scipy.fft.dct(np.eye(8), norm="ortho", axis=0)


def bm3d_stage_dense(noisy: np.ndarray, sigma: float, guide=None, lambda3d: float = 2.7):
    """One BM3D stage with the group transform as a dense matrix kron(Haar, C (x) C)."""
    H, W = noisy.shape
    C = dct_matrix()
    C2 = np.kron(C, C)  # acts on a row-major flattened 8x8 patch
    k = np.kaiser(8, 2.0)
    K = np.outer(k, k).ravel()
    groups = bm3d_brute_force_match(guide if guide is not None else noisy,
                                    400 if guide is not None else 2500)
    num = np.zeros(H * W)
    den = np.zeros(H * W)
    for grp in groups:
        L = 1
        while 2 * L <= len(grp):
            L *= 2
        pos = grp[:L]
        T3 = np.kron(haar_matrix(L), C2)

        def stack(img):
            return np.concatenate([img[p // W:p // W + 8, p % W:p % W + 8].ravel() for p in pos])

        tn = T3 @ stack(noisy)
        if guide is None:
            keep = np.abs(tn) > lambda3d * sigma
            tn = np.where(keep, tn, 0.0)
            wgt = 1.0 / (sigma ** 2 * max(1, int(keep.sum())))
        else:
            tb = T3 @ stack(guide)
            wie = tb ** 2 / (tb ** 2 + sigma ** 2)
            tn = wie * tn
            s = float(np.sum(wie ** 2))
            wgt = 1.0 / (sigma ** 2 * s) if s > 0 else 1.0 / sigma ** 2
        est = T3.T @ tn
        for kk, p in enumerate(pos):
            i, j = p // W, p % W
            flat = (np.arange(8)[:, None] + i) * W + (np.arange(8)[None, :] + j)
            np.add.at(num, flat.ravel(), wgt * K * est[kk * 64:(kk + 1) * 64])
            np.add.at(den, flat.ravel(), wgt * K)
    return (num / den).reshape(H, W)
