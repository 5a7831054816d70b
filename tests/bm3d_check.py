"""Element-wise BM3D parity with counted decision flips (test helpers).

A hard-threshold decision |c| > 2.7 sigma taken on a coefficient a few FP32
roundings from the threshold, or an 8-bit matching code rint(255 x) a few
roundings from a half-integer, can go the other way on the GPU than in the FP64
oracle; either changes one group's estimate, and so the pixels its patches
cover, and nothing else.  These helpers find every such group (hard stage: the
kept-coefficient count the GPU reports against the oracle's count on the same
group; Wiener stage: match lists that differ, or a guide that differs under the
group's patches) and return the pixels outside their footprints, where the GPU
must agree with the oracle to the FP32 bar.
"""
from __future__ import annotations

import numpy as np

import oracle
from tests.gpu_util import to_dev, to_np

PS = 8
LAMBDA_3D = 2.7


def pow2(m: int) -> int:
    L = 1
    while 2 * L <= m:
        L *= 2
    return L


def oracle_kept(img: np.ndarray, lists: np.ndarray, counts: np.ndarray, sigma: float):
    """Per group, the coefficients the oracle's hard threshold keeps on img (FP64)."""
    W = img.shape[1]
    thr = LAMBDA_3D * sigma
    kept = np.empty(len(counts), np.int64)
    for r in range(len(counts)):
        L = pow2(int(counts[r]))
        g = np.stack([img[p // W:p // W + PS, p % W:p % W + PS] for p in lists[r][:L]])
        kept[r] = int(np.count_nonzero(np.abs(oracle.bm3d_transform(g)) > thr))
    return kept


def footprint(shape, lists: np.ndarray, counts: np.ndarray, groups) -> np.ndarray:
    """Pixels covered by the patches of the given groups."""
    H, W = shape
    m = np.zeros((H, W), bool)
    for r in groups:
        for p in lists[r][:pow2(int(counts[r]))]:
            y, x = divmod(int(p), W)
            m[y:y + PS, x:x + PS] = True
    return m


def touches(shape, lists, counts, mask: np.ndarray) -> np.ndarray:
    """Groups any of whose patches overlaps mask."""
    W = shape[1]
    out = []
    for r in range(len(counts)):
        for p in lists[r][:pow2(int(counts[r]))]:
            y, x = divmod(int(p), W)
            if mask[y:y + PS, x:x + PS].any():
                out.append(r)
                break
    return np.array(out, np.int64)


def rel_on(a, b, keep) -> float:
    a, b = np.asarray(a, np.float64)[keep], np.asarray(b, np.float64)[keep]
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


class Check:
    """Accumulates flipped groups and the pixels kept for the element-wise bar."""

    def __init__(self):
        self.groups = 0
        self.flipped = 0
        self.pixels = 0
        self.kept_pixels = 0


def hard_stage(cs, img: np.ndarray, sigma: float, chk: Check):
    """GPU stage 1 of every slice of img [Z,H,W] (float32) with its decisions, the
    oracle's stage 1 on the same slices, and the mask of unflipped pixels.
    Returns (gpu_out, oracle_out, keep) as arrays [Z,H,W]."""
    Z, H, W = img.shape
    out, lists, counts, stat = cs.bm3d_stage_groups(1, to_dev(img), sigma)
    out, lists, counts = to_np(out), lists.cpu().numpy(), counts.cpu().numpy()
    stat = stat.cpu().numpy()
    refs, keeps = [], []
    for z in range(Z):
        x = img[z].astype(np.float64)
        idx, cnt = oracle.bm3d_match(x, 1)
        np.testing.assert_array_equal(lists[z], idx)
        np.testing.assert_array_equal(counts[z], cnt)
        kept = oracle_kept(x, idx, cnt, sigma)
        flipped = np.nonzero(kept != np.rint(stat[z]).astype(np.int64))[0]
        keeps.append(~footprint((H, W), idx, cnt, flipped))
        refs.append(oracle.bm3d_stage(x, sigma))
        chk.groups += len(cnt)
        chk.flipped += len(flipped)
    keep = np.stack(keeps)
    chk.pixels += keep.size
    chk.kept_pixels += int(keep.sum())
    return out, np.stack(refs), keep


def wiener_mask(cs, noisy, guide_gpu, guide_ref, changed, sigma, chk: Check):
    """Pixels of the Wiener stage outside the footprints of groups whose lists
    differ between the GPU (matched on guide_gpu) and the oracle (matched on
    guide_ref), or whose patches cover a pixel where the two guides differ
    (`changed`).  Returns the keep mask [Z,H,W]."""
    Z, H, W = noisy.shape
    _, lg, cg, _ = cs.bm3d_stage_groups(2, to_dev(noisy), sigma, guide=to_dev(guide_gpu))
    lg, cg = lg.cpu().numpy(), cg.cpu().numpy()
    keeps = []
    for z in range(Z):
        idx, cnt = oracle.bm3d_match(guide_ref[z].astype(np.float64), 2)
        differ = np.nonzero((cnt != cg[z]) | np.any(idx != lg[z], axis=1))[0]
        bad = footprint((H, W), idx, cnt, differ) | footprint((H, W), lg[z], cg[z], differ)
        for lst, c in ((idx, cnt), (lg[z], cg[z])):
            bad |= footprint((H, W), lst, c, touches((H, W), lst, c, changed[z]))
        chk.groups += len(cnt)
        chk.flipped += len(differ)
        keeps.append(~bad)
    return np.stack(keeps)


def denoise(cs, g: np.ndarray, sigma: float, chk: Check):
    """BM3D (both stages) of every slice of g [Z,H,W] float32 against the oracle,
    element-wise outside flipped footprints.  Returns (oracle_out, keep)."""
    basic_g, basic_r, keep1 = hard_stage(cs, g, sigma, chk)
    basic_g32 = basic_g.astype(np.float32)
    keep2 = wiener_mask(cs, g, basic_g32, basic_r, ~keep1, sigma, chk)
    ref = np.stack([oracle.bm3d_stage(g[z].astype(np.float64), sigma, guide=basic_r[z])
                    for z in range(g.shape[0])])
    keep = keep1 & keep2
    chk.pixels += keep.size
    chk.kept_pixels += int(keep.sum())
    return ref, keep
