"""BM3D u-step: CUDA path vs the FP64 oracle through the C ABI.

Bars: match lists bit-exact (integer work on identical float32 inputs); every
stage element-wise within relative L2 1e-5 of the oracle outside the footprints
of the groups whose decisions flipped (a hard-threshold decision on a
coefficient a few FP32 roundings from 2.7 sigma, found by comparing each
group's kept-coefficient count with the oracle's; a Wiener group whose match
list or guide differs), with the flipped groups counted and held to a small
fraction; full ADMM runs with BM3D within 0.05 dB PSNR of the oracle.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import bm3d_check as bc
from tests.gpu_util import DPSNR, REL_ITER, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cs():
    import torch

    from paper_2511_03093_gb300 import build as b

    b.build()
    import paper_2511_03093_gb300 as m

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return m


def _blobs(seed, Z, H, W, noise=0.04):
    w = synth.Workload("b", Z, H, W, seed=seed, peak=None, n_blobs=max(4, Z * H * W // 300))
    rng = np.random.default_rng(seed + 1)
    x = synth.generate(w)["x"]
    return (x + noise * rng.standard_normal(x.shape)).astype(np.float32)


SHAPES = [(2, 37, 53), (1, 64, 70), (1, 100, 41), (1, 8, 8), (2, 9, 20), (1, 46, 46)]


@pytest.mark.parametrize("Z,H,W", SHAPES)
@pytest.mark.parametrize("stage", [1, 2])
def test_match_lists_bit_exact(cs, Z, H, W, stage):
    img = _blobs(Z * 100 + H, Z, H, W, noise=0.02 if stage == 1 else 0.005)
    lists, counts = cs.bm3d_match(to_dev(img), stage)
    lists, counts = lists.cpu().numpy(), counts.cpu().numpy()
    for z in range(Z):
        idx, cnt = oracle.bm3d_match(img[z], stage)
        np.testing.assert_array_equal(counts[z], cnt)
        np.testing.assert_array_equal(lists[z], idx)


@pytest.mark.parametrize("stage", [1, 2])
def test_match_lists_bit_exact_outside_unit_range(cs, stage):
    """ADMM iterates leave [0, 1]: the 8-bit matching codes saturate at 0 and 255
    there; lists must still equal the oracle's bit for bit."""
    img = _blobs(77, 2, 64, 70, noise=0.02 if stage == 1 else 0.005)
    img = (1.8 * img - 0.4).astype(np.float32)  # about [-0.4, 1.4]
    assert img.min() < 0.0 and img.max() > 1.0
    lists, counts = cs.bm3d_match(to_dev(img), stage)
    lists, counts = lists.cpu().numpy(), counts.cpu().numpy()
    for z in range(2):
        idx, cnt = oracle.bm3d_match(img[z], stage)
        np.testing.assert_array_equal(counts[z], cnt)
        np.testing.assert_array_equal(lists[z], idx)


def test_match_ties_on_constant_image(cs):
    img = np.full((1, 40, 44), 0.25, dtype=np.float32)
    lists, counts = cs.bm3d_match(to_dev(img), 1)
    idx, cnt = oracle.bm3d_match(img[0], 1)
    np.testing.assert_array_equal(lists.cpu().numpy()[0], idx)
    assert np.all(counts.cpu().numpy() == 16)


@pytest.mark.parametrize("Z,H,W", [(2, 37, 53), (1, 64, 70), (1, 96, 96)])
def test_wiener_stage_on_identical_guide(cs, Z, H, W):
    noisy = _blobs(7 + H, Z, H, W)
    sigma = 0.04
    basic = np.stack([oracle.bm3d_stage(noisy[z], sigma) for z in range(Z)]).astype(np.float32)
    out = to_np(cs.bm3d_stage(2, to_dev(noisy), sigma, guide=to_dev(basic)))
    ref = np.stack([oracle.bm3d_stage(noisy[z], sigma, guide=basic[z]) for z in range(Z)])
    assert rel_l2(out, ref) <= REL_ITER


def _flip_bounds(chk, max_frac=0.01):
    """Flips are rare (coefficients within FP32 rounding of the threshold): a
    systematic error would flip many groups and leave few pixels to compare."""
    assert chk.flipped <= max(2, max_frac * chk.groups), (chk.flipped, chk.groups)
    assert chk.kept_pixels >= 0.5 * chk.pixels, (chk.kept_pixels, chk.pixels)


@pytest.mark.parametrize("Z,H,W", [(2, 37, 53), (1, 96, 96), (1, 130, 70)])
def test_hard_stage(cs, Z, H, W):
    noisy = _blobs(11 + H, Z, H, W)
    chk = bc.Check()
    out, ref, keep = bc.hard_stage(cs, noisy, 0.04, chk)
    assert bc.rel_on(out, ref, keep) <= REL_ITER, (bc.rel_on(out, ref, keep), chk.flipped)
    _flip_bounds(chk)
    # the plain stage entry point gives the same result as the diagnostic one
    np.testing.assert_allclose(to_np(cs.bm3d_stage(1, to_dev(noisy), 0.04)), out, rtol=0,
                               atol=1e-6)


def test_hard_stage_zero_threshold_limit(cs):
    """Tiny sigma: nothing is thresholded away, the stage reproduces its input."""
    noisy = _blobs(3, 1, 40, 40)
    out = to_np(cs.bm3d_stage(1, to_dev(noisy), 1e-6))
    assert rel_l2(out, noisy) <= 1e-6


@pytest.mark.parametrize("Z,H,W", [(2, 48, 40), (1, 128, 128)])
def test_denoise_bm3d(cs, Z, H, W):
    noisy = _blobs(5 + W, Z, H, W)
    out = to_np(cs.denoise(to_dev(noisy), cs.Params(denoiser="bm3d", bm3d_sigma=0.04)))
    chk = bc.Check()
    ref, keep = bc.denoise(cs, noisy, 0.04, chk)
    assert bc.rel_on(out, ref, keep) <= REL_ITER, (bc.rel_on(out, ref, keep), chk.flipped)
    _flip_bounds(chk)
    clean = synth.generate(synth.Workload("b", Z, H, W, seed=5 + W, peak=None,
                                          n_blobs=max(4, Z * H * W // 300)))["x"]
    assert abs(oracle.psnr(out, clean) - oracle.psnr(oracle.bm3d(noisy, 0.04), clean)) <= DPSNR


@pytest.mark.parametrize("gamma", [0.0, 0.5])
def test_one_iteration_bm3d(cs, gamma):
    """One ADMM iteration (Algorithm 1) with the BM3D u-step from a given state.
    v against the oracle; every slice's u against the oracle's BM3D of the prox
    input the sweep formed for it (from the GPU's own newer neighbour, so a flip
    in one slice is not carried into the check of the next), element-wise
    outside flipped groups.  rho = 1, gamma = 0.5 make the prox input's FP32
    arithmetic exact to restate: g = (w + (u_prev + u_next) / 2) / 2."""
    import torch

    Z, H, W = 4, 40, 48
    rng = np.random.default_rng(21)
    masks = (rng.random((Z, H, W)) < 0.5).astype(np.uint8)
    x = _blobs(9, Z, H, W, noise=0.0)
    b = oracle.forward(x, masks, 1).astype(np.float32)
    u0 = _blobs(10, Z, H, W, noise=0.05)
    d0 = (0.01 * rng.standard_normal((Z, H, W))).astype(np.float32)
    prm = cs.Params(rho=1.0, lam=0.0, gamma=gamma, iters=1, denoiser="bm3d", bm3d_sigma=0.04)
    plan = cs.Plan(H, W, 1, Z, to_dev(masks))
    u, d = to_dev(u0), to_dev(d0)
    v = plan.solve(to_dev(b), prm, u=u, d=d, init_user=True)
    torch.cuda.synchronize()
    v_r, *_ = oracle.admm(b, masks, Z, rho=1.0, lam=0.0, gamma=gamma, iters=1,
                          denoiser="bm3d", bm3d_sigma=0.04, u0=u0, d0=d0)
    vg = to_np(v).astype(np.float32)
    assert rel_l2(vg, v_r) <= REL_ITER
    ug, dg = to_np(u).astype(np.float32), to_np(d).astype(np.float32)
    w = vg + d0  # the workspace w = v + d the x-update wrote (FP32)
    np.testing.assert_array_equal(dg, w - ug)  # dual update d = w - u
    chk = bc.Check()
    for n in range(Z):  # sweep order: slice n sees u_{n-1} new and u_{n+1} old
        if gamma > 0.0:
            um = ug[n - 1] if n > 0 else u0[Z - 1]
            up = u0[n + 1] if n < Z - 1 else ug[0]
            g = ((w[n] + np.float32(0.5) * (um + up)) * np.float32(0.5)).astype(np.float32)
        else:
            g = w[n]
        ref, keep = bc.denoise(cs, g[None], 0.04, chk)
        assert bc.rel_on(ug[n][None], ref, keep) <= REL_ITER, (n, chk.flipped)
    _flip_bounds(chk)
    plan.close()


@pytest.mark.parametrize("gamma", [0.0, 0.1])
def test_full_run_bm3d(cs, gamma):
    import torch

    w = synth.Workload("bm3d_small", 8, 64, 72, mask_p=0.5, seed=31, n_blobs=60)
    data = synth.generate(w)
    prm = cs.Params(rho=1.0, lam=0.0, gamma=gamma, iters=10, denoiser="bm3d", bm3d_sigma=0.05)
    plan = cs.Plan(w.H, w.W, 1, w.Z, to_dev(data["masks"]))
    v = plan.solve(to_dev(data["b"]), prm)
    torch.cuda.synchronize()
    v_r, *_ = oracle.admm(data["b64"], data["masks"], w.Z, rho=1.0, lam=0.0, gamma=gamma,
                          iters=10, denoiser="bm3d", bm3d_sigma=0.05)
    p_gpu, p_ref = oracle.psnr(to_np(v), data["x"]), oracle.psnr(v_r, data["x"])
    assert abs(p_gpu - p_ref) <= DPSNR, (p_gpu, p_ref)
    plan.close()
