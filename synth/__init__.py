"""Seeded synthetic inputs for the compressive light-sheet reconstruction.

This module is shared by the oracle tests, the CUDA parity tests and the
benchmark.  It draws ground-truth volumes, binary DMD masks and camera noise;
it holds none of the reconstruction method's arithmetic (no Phi^T, no
x-update, no denoiser).  The one operator it applies is the acquisition
itself (the physical camera exposure of Sec. III-A: each coded image is the
sum of R mask-modulated z-planes), followed by Poisson + Gaussian camera noise,
so that both sides of every parity test receive the same measurement.

The paper's zebrafish-heart dataset (Sec. IV-A) is not available; the
Gaussian-blob volumes below stand in for it: sparse round nuclei (sigma 1.5-4
px, amplitudes U[0.2, 1]) on a smooth low-frequency background, optionally
drifting laterally from slice to slice like a contracting heart.

One numpy PCG64 stream per workload, drawn in a fixed order: blob parameters,
background phases, masks, noise.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Workload",
    "WORKLOADS",
    "batch_workloads",
    "blob_count",
    "make_volume",
    "make_masks",
    "acquire",
    "generate",
    "random_fields",
]


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic acquisition: a Z x H x W volume seen through N coded shots.

    Z = n_shots * R slices; mask_p is the Bernoulli probability of an "on"
    DMD mirror; (peak, sigma_g) set the Poisson photon peak and the Gaussian
    read-noise level relative to the measurement maximum (peak=None: noise free).
    """

    name: str
    Z: int
    H: int
    W: int
    n_shots: int = 1
    drift: bool = False
    mask_p: float = 0.5
    per_slice_masks: bool = True
    peak: float | None = 200.0
    sigma_g: float = 0.01
    seed: int = 1001
    n_blobs: int | None = None

    @property
    def R(self) -> int:
        return self.Z // self.n_shots


# The workloads every test and benchmark refers to by name.
WORKLOADS: dict[str, Workload] = {
    # 128x128x8, 200 blobs, Bernoulli(0.5), Poisson peak 200 + Gaussian 0.01
    "tv_128x128x8": Workload("tv_128x128x8", 8, 128, 128, mask_p=0.5, peak=200.0,
                             sigma_g=0.01, seed=1001, n_blobs=200),
    # 512x512x16 drifting blobs, Bernoulli(0.3), Poisson peak 50 + Gaussian 0.02
    "tvz_512x512x16": Workload("tvz_512x512x16", 16, 512, 512, drift=True, mask_p=0.3,
                               peak=50.0, sigma_g=0.02, seed=1002),
    # 1024x1024x32, Bernoulli(0.5)
    "bm3d_1024x1024x32": Workload("bm3d_1024x1024x32", 32, 1024, 1024, mask_p=0.5,
                                  peak=200.0, sigma_g=0.01, seed=1003),
}


def batch_workloads(n: int = 64, seed: int = 4000, max_blobs: int = 2000) -> list[Workload]:
    """The batch of independent measurements: item i has H = W drawn uniformly
    from {256, 512, 768, 1024} and Z from {8, 16, 32} (one numpy stream seeded
    with `seed`, Z first), drifting blobs (at most `max_blobs` per item, to keep
    the host-side generation of the 64-item batch to seconds), Bernoulli(0.3)
    patterns, Poisson peak 50 + Gaussian sigma 0.02, and seed `seed` + i."""
    rng = np.random.default_rng(seed)
    sizes = [(int(rng.choice([8, 16, 32])), int(rng.choice([256, 512, 768, 1024])))
             for _ in range(n)]
    return [Workload(f"b{i}", Z, S, S, drift=True, mask_p=0.3, peak=50.0, sigma_g=0.02,
                     seed=seed + i, n_blobs=min(max_blobs, blob_count(Z, S, S)))
            for i, (Z, S) in enumerate(sizes)]


def blob_count(Z: int, H: int, W: int) -> int:
    """200 blobs per 128x128x8 voxels, capped at 20000 (density kept constant)."""
    return int(min(20000, max(1, round(200.0 * Z * H * W / (128 * 128 * 8)))))


def make_volume(rng: np.random.Generator, Z: int, H: int, W: int, n_blobs: int,
                drift: bool) -> np.ndarray:
    """Ground-truth volume in [0, 1], float64 [Z, H, W], max exactly 1."""
    cz = rng.uniform(0.0, Z, n_blobs)
    cy = rng.uniform(0.0, H, n_blobs)
    cx = rng.uniform(0.0, W, n_blobs)
    sig = rng.uniform(1.5, 4.0, n_blobs)
    amp = rng.uniform(0.2, 1.0, n_blobs)
    if drift:
        mag = rng.uniform(0.0, 2.0, n_blobs)
        ang = rng.uniform(0.0, 2.0 * math.pi, n_blobs)
        dy, dx = mag * np.sin(ang), mag * np.cos(ang)
    else:
        dy = dx = np.zeros(n_blobs)
    ph = rng.uniform(0.0, 2.0 * math.pi, 3)

    vol = np.zeros((Z, H, W), dtype=np.float64)
    for k in range(n_blobs):
        s = sig[k]
        rad = 4.0 * s
        z0, z1 = max(0, int(math.floor(cz[k] - rad))), min(Z, int(math.ceil(cz[k] + rad)) + 1)
        for z in range(z0, z1):
            gz = math.exp(-((z - cz[k]) ** 2) / (2 * s * s))
            yc = cy[k] + (z - cz[k]) * dy[k]
            xc = cx[k] + (z - cz[k]) * dx[k]
            y0, y1 = max(0, int(math.floor(yc - rad))), min(H, int(math.ceil(yc + rad)) + 1)
            x0, x1 = max(0, int(math.floor(xc - rad))), min(W, int(math.ceil(xc + rad)) + 1)
            if y0 >= y1 or x0 >= x1:
                continue
            gy = np.exp(-((np.arange(y0, y1) - yc) ** 2) / (2 * s * s))
            gx = np.exp(-((np.arange(x0, x1) - xc) ** 2) / (2 * s * s))
            vol[z, y0:y1, x0:x1] += (amp[k] * gz) * np.outer(gy, gx)

    zz = np.arange(Z, dtype=np.float64)[:, None, None]
    yy = np.arange(H, dtype=np.float64)[None, :, None]
    xx = np.arange(W, dtype=np.float64)[None, None, :]
    bg = 0.05 + 0.05 * (np.cos(2 * math.pi * xx / W + ph[0])
                        * np.cos(2 * math.pi * yy / H + ph[1])
                        * np.cos(math.pi * zz / Z + ph[2]))
    vol += bg
    vol /= vol.max()
    return vol


def make_masks(rng: np.random.Generator, n_masks: int, H: int, W: int, p: float) -> np.ndarray:
    """Binary DMD patterns, uint8 {0,1} [n_masks, H, W], i.i.d. Bernoulli(p)."""
    return (rng.random((n_masks, H, W)) < p).astype(np.uint8)


def acquire(rng: np.random.Generator, vol: np.ndarray, masks: np.ndarray, n_shots: int,
            per_slice: bool, peak: float | None, sigma_g: float) -> np.ndarray:
    """Simulated camera exposures, float64 [n_shots, H, W].

    Shot j integrates the R slices (j*R .. j*R+R-1) of the volume, each
    modulated by its DMD pattern (the DMD/scanner hardware of Sec. III-A),
    then Poisson photon noise at the given peak count and Gaussian read
    noise with std sigma_g * max are added.
    """
    Z, H, W = vol.shape
    R = Z // n_shots
    y = np.zeros((n_shots, H, W), dtype=np.float64)
    for j in range(n_shots):
        for r in range(R):
            m = masks[j * R + r] if per_slice else masks[r]
            y[j] += m * vol[j * R + r]
    if peak is None:
        return y
    s = float(y.max())
    y = s * rng.poisson(peak * y / s).astype(np.float64) / peak
    y += rng.normal(0.0, sigma_g * s, size=y.shape)
    return y


def generate(w: Workload | str) -> dict:
    """Draw one workload: ground truth x, masks, measurement b (float32) and b64.

    b64 is float64(b): both the oracle and the CUDA path see exactly the same
    float32 measurement values.
    """
    if isinstance(w, str):
        w = WORKLOADS[w]
    rng = np.random.default_rng(w.seed)
    nb = w.n_blobs if w.n_blobs is not None else blob_count(w.Z, w.H, w.W)
    x = make_volume(rng, w.Z, w.H, w.W, nb, w.drift)
    n_masks = w.Z if w.per_slice_masks else w.R
    masks = make_masks(rng, n_masks, w.H, w.W, w.mask_p)
    b64 = acquire(rng, x, masks, w.n_shots, w.per_slice_masks, w.peak, w.sigma_g)
    b = b64.astype(np.float32)
    return {"workload": w, "x": x, "masks": masks, "b": b, "b64": b.astype(np.float64)}


def random_fields(seed: int, shape, n: int, scale: float = 1.0) -> list[np.ndarray]:
    """n float32 arrays of standard-normal values (iterate states for one-step tests)."""
    rng = np.random.default_rng(seed)
    return [(scale * rng.standard_normal(shape)).astype(np.float32) for _ in range(n)]
