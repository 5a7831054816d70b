"""FP64 oracle of the WNNM u-step denoiser (plain numpy).  TEST INFRASTRUCTURE ONLY.

Weighted nuclear norm minimisation is one of the plug-in denoisers the paper lists
for the u-subproblem (Eq. u-sub, Sec. III-B); Sec. II describes it as stacking
similar patches into a matrix and shrinking it towards low rank with a weighted
nuclear norm.  The paper states none of its internals.  The variant stated here,
applied to each 2-D slice on its own:

  - groups: the hard-stage block matching of the BM3D oracle (8 x 8 patches on
    the 8-bit codes, reference grid step 3 plus the last position, 39 x 39
    window, mean-SSD threshold 2500 / 255^2, up to 16 positions in increasing
    (SSD, index), the reference first); all m matches are used;
  - Y: 64 x m, column k = patch k in row-major order; mu = the mean patch;
    Yc = Y - mu 1^T = U diag(s) V^T (the SVD, a library routine);
  - sigma_hat_i = sqrt(max(s_i^2 - 64 sigma^2, 0)) estimates the clean singular
    value (a 64 x m Gaussian noise matrix with m <= 16 carries about
    max(64, m) sigma^2 = 64 sigma^2 per singular value; WNNM's own estimate
    subtracts m sigma^2 for groups with more patches than pixels per patch);
    weight w_i = c sqrt(m) / (sigma_hat_i + eps), c = 2 sqrt(2), eps = 1e-8;
  - x_i = max(s_i - sigma^2 w_i, 0): with weights that grow as s_i shrinks this
    weighted soft threshold minimises 1/2 ||Yc - X||_F^2 + sigma^2 sum_i w_i s_i(X);
  - Xhat = U diag(x) V^T + mu 1^T; every estimated patch is added with weight 1
    into numerator and count images, and the slice is their ratio (the reference
    grid reaches every pixel);
  - one pass per u-step (no inner iterative regularisation: PnP-ADMM iterates);
    slices smaller than a patch are returned unchanged.
"""
from __future__ import annotations

import numpy as np

from . import bm3d_match, vupdate

C_WNNM = 2.0 * np.sqrt(2.0)
EPS = 1e-8
PS = 8


def wnnm_group(Y: np.ndarray, sigma: float) -> np.ndarray:
    """The WNNM estimate of one group matrix Y (64 x m)."""
    Y = np.asarray(Y, dtype=np.float64)
    m = Y.shape[1]
    mu = Y.mean(axis=1, keepdims=True)
    U, s, Vt = np.linalg.svd(Y - mu, full_matrices=False)
    sh = np.sqrt(np.maximum(s * s - max(64, m) * sigma * sigma, 0.0))
    w = C_WNNM * np.sqrt(m) / (sh + EPS)
    x = np.maximum(s - sigma * sigma * w, 0.0)
    return (U * x) @ Vt + mu


def wnnm_slice(img: np.ndarray, sigma: float) -> np.ndarray:
    img = np.asarray(img, dtype=np.float64)
    H, W = img.shape
    if H < PS or W < PS:
        return img.copy()
    idx, cnt = bm3d_match(img, 1)
    num = np.zeros_like(img)
    den = np.zeros_like(img)
    for r in range(idx.shape[0]):
        pos = idx[r, :cnt[r]]
        ys, xs = pos // W, pos % W
        Y = np.stack([img[y:y + PS, x:x + PS].reshape(-1) for y, x in zip(ys, xs)], axis=1)
        X = wnnm_group(Y, sigma)
        for k, (y, x) in enumerate(zip(ys, xs)):
            num[y:y + PS, x:x + PS] += X[:, k].reshape(PS, PS)
            den[y:y + PS, x:x + PS] += 1.0
    return num / den


def wnnm(g, sigma: float) -> np.ndarray:
    """WNNM of each slice of g ([Z, H, W] or [H, W])."""
    g = np.asarray(g, dtype=np.float64)
    if g.ndim == 2:
        return wnnm_slice(g, sigma)
    return np.stack([wnnm_slice(g[z], sigma) for z in range(g.shape[0])])


def admm_wnnm(b, masks, Z: int, *, rho: float, gamma: float, sigma: float, iters: int,
              u0=None, d0=None):
    """Algorithm 1 with the WNNM u-step (Eq. u-update: the slice's g from w and its
    z neighbours, newest values first, cyclic), one shot (N = 1, R = Z).
    Returns (v^K, u^K, d^K)."""
    b = np.asarray(b, dtype=np.float64)
    u = np.zeros((Z,) + b.shape[1:]) if u0 is None else np.array(u0, dtype=np.float64)
    d = np.zeros_like(u) if d0 is None else np.array(d0, dtype=np.float64)
    gam = gamma if Z > 1 else 0.0
    v = np.zeros_like(u)
    for _ in range(iters):
        v = vupdate(b, u, d, masks, rho)
        w = v + d
        for n in range(Z):
            g = (rho * w[n] + gam * (u[(n - 1) % Z] + u[(n + 1) % Z])) / (rho + 2 * gam) \
                if gam > 0 else w[n]
            u[n] = wnnm_slice(g, sigma)
        d = w - u
    return v, u, d
