"""FP64 CPU oracle for the PnP-ADMM light-sheet reconstruction (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  The oracle is a plain double-precision C
implementation of what the method computes (forward model of Sec. III-A, the
Woodbury v-update of Sec. III-B, the Tikhonov / TV / BM3D u-steps, the
Gauss-Seidel z-sweep of Sec. III-C and Algorithm 1).  Only the tests, the
package smoke check and the benchmark's CPU-baseline leg use it; the CUDA
product path never imports it, and it imports nothing from the product.

Every array argument is converted to C-contiguous float64; masks are given as
{0,1} (or relaxed real) arrays of shape [R,H,W] (shared) or [Z,H,W] (per slice).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SOURCES = ["oracle.c", "bm3d.c"]

OR_TIKHONOV, OR_TV, OR_BM3D = 0, 1, 2
_DENOISERS = {"tikhonov": OR_TIKHONOV, "tv": OR_TV, "bm3d": OR_BM3D}


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C11, OpenMP, no fast-math, no FMA contraction)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    if not force and os.path.exists(_LIB_PATH):
        lib_m = os.path.getmtime(_LIB_PATH)
        deps = srcs + [os.path.join(_HERE, "oracle.h")]
        if all(os.path.getmtime(s) <= lib_m for s in deps):
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        i, d, P = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        L.or_forward.argtypes = [i, i, i, i, P, i, P, P]
        L.or_forward.restype = None
        L.or_adjoint.argtypes = [i, i, i, i, P, i, P, P]
        L.or_adjoint.restype = None
        L.or_phiphit.argtypes = [i, i, i, i, P, i, P]
        L.or_phiphit.restype = None
        L.or_vupdate.argtypes = [i, i, i, i, P, i, P, P, P, d, P]
        L.or_vupdate.restype = None
        L.or_tv_prox.argtypes = [i, i, P, d, i, d, P]
        L.or_tv_prox.restype = i
        L.or_psnr.argtypes = [ctypes.c_size_t, P, P]
        L.or_psnr.restype = d
        L.or_ssim3d.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P]
        L.or_ssim3d.restype = d
        L.or_bm3d.argtypes = [i, i, P, d, P]
        L.or_bm3d.restype = i
        L.or_bm3d_stage.argtypes = [i, i, P, P, d, d, P]
        L.or_bm3d_stage.restype = i
        L.or_bm3d_match.argtypes = [i, i, P, i, P, P]
        L.or_bm3d_match.restype = i
        L.or_bm3d_ref_positions.argtypes = [i, P]
        L.or_bm3d_ref_positions.restype = i
        L.or_bm3d_dct8.argtypes = [P]
        L.or_bm3d_dct8.restype = None
        L.or_bm3d_transform.argtypes = [i, P, i]
        L.or_bm3d_transform.restype = None
        L.or_bm3d_kaiser.argtypes = [P]
        L.or_bm3d_kaiser.restype = None
        L.or_admm.argtypes = [i, i, i, i, P, i, P, d, d, d, i, d, i, i, d, d, i, P, P, P,
                              ctypes.POINTER(ctypes.c_int)]
        L.or_admm.restype = i
        _lib = L
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _geom(masks: np.ndarray, Z: int, n_shots: int):
    masks = _f64(masks)
    R = Z // n_shots
    if R * n_shots != Z:
        raise ValueError("Z must equal n_shots * R")
    per_slice = {Z: 1, R: 0}.get(masks.shape[0])
    if per_slice is None:
        raise ValueError("masks must have R or Z planes")
    if Z == R:
        per_slice = 1
    return masks, R, per_slice


def forward(v, masks, n_shots: int = 1) -> np.ndarray:
    """b = Phi v (Sec. III-A).  v [Z,H,W] -> b [N,H,W]."""
    v = _f64(v)
    Z, H, W = v.shape
    m, R, ps = _geom(masks, Z, n_shots)
    b = np.empty((n_shots, H, W))
    lib().or_forward(n_shots, R, H, W, _p(m), ps, _p(v), _p(b))
    return b


def adjoint(b, masks, Z: int) -> np.ndarray:
    """v = Phi^T b.  b [N,H,W] -> v [Z,H,W]."""
    b = _f64(b)
    N, H, W = b.shape
    m, R, ps = _geom(masks, Z, N)
    v = np.empty((Z, H, W))
    lib().or_adjoint(N, R, H, W, _p(m), ps, _p(b), _p(v))
    return v


def phiphit(masks, Z: int, n_shots: int = 1) -> np.ndarray:
    """D = diag(Phi Phi^T) per shot, [N,H,W]."""
    m, R, ps = _geom(masks, Z, n_shots)
    H, W = m.shape[1:]
    D = np.empty((n_shots, H, W))
    lib().or_phiphit(n_shots, R, H, W, _p(m), ps, _p(D))
    return D


def vupdate(b, u, d, masks, rho: float) -> np.ndarray:
    """Closed-form v-subproblem solution (Eq. v-update, Woodbury form)."""
    b, u, d = _f64(b), _f64(u), _f64(d)
    N, H, W = b.shape
    Z = u.shape[0]
    m, R, ps = _geom(masks, Z, N)
    v = np.empty_like(u)
    lib().or_vupdate(N, R, H, W, _p(m), ps, _p(b), _p(u), _p(d), float(rho), _p(v))
    return v


def tv_prox(g, theta: float, T: int, tau: float = 0.125) -> np.ndarray:
    """Chambolle prox of theta*TV on one slice [H,W] or each slice of [Z,H,W]."""
    g = _f64(g)
    squeeze = g.ndim == 2
    g3 = g[None] if squeeze else g
    out = np.empty_like(g3)
    Z, H, W = g3.shape
    for z in range(Z):
        gz = np.ascontiguousarray(g3[z])
        oz = np.empty_like(gz)
        if lib().or_tv_prox(H, W, _p(gz), float(theta), int(T), float(tau), _p(oz)) != 0:
            raise MemoryError("or_tv_prox failed")
        out[z] = oz
    return out[0] if squeeze else out


def bm3d(g, sigma: float) -> np.ndarray:
    """BM3D denoise of each slice with noise level sigma."""
    g = _f64(g)
    squeeze = g.ndim == 2
    g3 = g[None] if squeeze else g
    out = np.empty_like(g3)
    Z, H, W = g3.shape
    for z in range(Z):
        gz = np.ascontiguousarray(g3[z])
        oz = np.empty_like(gz)
        rc = lib().or_bm3d(H, W, _p(gz), float(sigma), _p(oz))
        if rc != 0:
            raise RuntimeError(f"or_bm3d failed ({rc})")
        out[z] = oz
    return out[0] if squeeze else out


def bm3d_stage(noisy, sigma: float, guide=None, lambda3d: float = 2.7) -> np.ndarray:
    """One BM3D stage on one slice [H,W]: hard threshold (guide None) or Wiener."""
    noisy = _f64(noisy)
    H, W = noisy.shape
    out = np.empty_like(noisy)
    g = _f64(guide) if guide is not None else None
    rc = lib().or_bm3d_stage(H, W, _p(noisy), _p(g) if g is not None else None, float(sigma),
                             float(lambda3d), _p(out))
    if rc != 0:
        raise RuntimeError(f"or_bm3d_stage failed ({rc})")
    return out


def bm3d_ref_positions(n: int) -> list[int]:
    buf = np.zeros(n + 2, dtype=np.int32)
    k = lib().or_bm3d_ref_positions(int(n), _p(buf))
    return buf[:k].tolist()


def bm3d_match(img, stage: int):
    """Match lists of one slice: (idx [nref,16] int64 with -1 padding, counts [nref])."""
    img = _f64(img)
    H, W = img.shape
    nref = max(1, len(bm3d_ref_positions(H)) * len(bm3d_ref_positions(W)))
    idx = np.full((nref, 16), -1, dtype=np.int64)
    cnt = np.zeros(nref, dtype=np.int32)
    k = lib().or_bm3d_match(H, W, _p(img), int(stage), _p(idx), _p(cnt))
    if k < 0:
        raise MemoryError("or_bm3d_match failed")
    return idx[:k], cnt[:k]


def bm3d_dct8() -> np.ndarray:
    C = np.empty((8, 8))
    lib().or_bm3d_dct8(_p(C))
    return C


def bm3d_transform(group, inverse: bool = False) -> np.ndarray:
    g = _f64(group).copy()
    lib().or_bm3d_transform(g.shape[0], _p(g), int(bool(inverse)))
    return g


def bm3d_kaiser() -> np.ndarray:
    K = np.empty((8, 8))
    lib().or_bm3d_kaiser(_p(K))
    return K


def psnr(x, ref) -> float:
    """3D PSNR (Sec. IV): 10 log10(n V^2 / ||x-ref||^2), V = max(ref)."""
    x, ref = _f64(x), _f64(ref)
    return float(lib().or_psnr(x.size, _p(x), _p(ref)))


def ssim3d(x, ref, return_map: bool = False):
    """3-D SSIM (Sec. IV): mean over all voxels of the local ssim with an
    11^3 Gaussian window (sigma 1.5) clipped to the volume and renormalised,
    c1 = 0.01^2, c2 = 0.03^2.  x, ref: [Z, H, W] (or [H, W])."""
    x, ref = _f64(x), _f64(ref)
    if x.ndim == 2:
        x, ref = x[None], ref[None]
    Z, H, W = x.shape
    m = np.empty_like(x) if return_map else None
    s = float(lib().or_ssim3d(Z, H, W, _p(x), _p(ref), _p(m) if m is not None else None))
    return (s, m) if return_map else s


def admm(b, masks, Z: int, *, rho: float, lam: float, gamma: float = 0.0, iters: int,
         denoiser: str = "tv", tol: float = 0.0, tv_inner: int = 20, tv_tau: float = 0.125,
         bm3d_sigma: float = 0.05, u0=None, d0=None):
    """Algorithm 1.  Returns (v^K, u^K, d^K, iterations run)."""
    b = _f64(b)
    N, H, W = b.shape
    m, R, ps = _geom(masks, Z, N)
    user = u0 is not None
    u = _f64(u0).copy() if user else np.zeros((Z, H, W))
    d = _f64(d0).copy() if user else np.zeros((Z, H, W))
    v = np.empty((Z, H, W))
    done = ctypes.c_int(0)
    rc = lib().or_admm(N, R, H, W, _p(m), ps, _p(b), float(rho), float(lam), float(gamma),
                       int(iters), float(tol), _DENOISERS[denoiser], int(tv_inner),
                       float(tv_tau), float(bm3d_sigma), int(user), _p(v), _p(u), _p(d),
                       ctypes.byref(done))
    if rc != 0:
        raise RuntimeError(f"or_admm failed ({rc})")
    return v, u, d, done.value
