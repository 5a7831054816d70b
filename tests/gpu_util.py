"""Helpers shared by the GPU parity tests (marshalling and error metrics only)."""
from __future__ import annotations

import numpy as np


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def to_dev(x, dtype=None):
    import torch

    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def to_np(t) -> np.ndarray:
    return t.detach().double().cpu().numpy()


# Parity bar for one FP32 ADMM iteration against the FP64 oracle.
REL_ITER = 1e-5
# Full-run bar: reconstruction PSNR within this many dB of the oracle's.
DPSNR = 0.05
