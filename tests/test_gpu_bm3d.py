"""BM3D u-step: CUDA path vs the FP64 oracle through the C ABI.

Bars: match lists bit-exact (integer work on identical float32 inputs); the
Wiener stage on an identical basic estimate within relative L2 1e-5 (no
discontinuous decision); the hard stage and the whole denoiser, whose hard
threshold can flip on 1-ulp differences between FP32 and FP64 coefficients,
within relative L2 1e-4 and with at most 0.1 % of pixels off by more than 1e-4;
full ADMM runs with BM3D within 0.05 dB PSNR of the oracle.
"""
import numpy as np
import pytest

import oracle
import synth
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


def _close_with_flips(out, ref):
    diff = np.abs(out - ref)
    return rel_l2(out, ref) <= 1e-4 and np.mean(diff > 1e-4) <= 1e-3


@pytest.mark.parametrize("Z,H,W", [(2, 37, 53), (1, 96, 96)])
def test_hard_stage(cs, Z, H, W):
    noisy = _blobs(11 + H, Z, H, W)
    out = to_np(cs.bm3d_stage(1, to_dev(noisy), 0.04))
    ref = np.stack([oracle.bm3d_stage(noisy[z], 0.04) for z in range(Z)])
    assert _close_with_flips(out, ref), (rel_l2(out, ref), np.mean(np.abs(out - ref) > 1e-4))


def test_hard_stage_zero_threshold_limit(cs):
    """Tiny sigma: nothing is thresholded away, the stage reproduces its input."""
    noisy = _blobs(3, 1, 40, 40)
    out = to_np(cs.bm3d_stage(1, to_dev(noisy), 1e-6))
    assert rel_l2(out, noisy) <= 1e-6


@pytest.mark.parametrize("Z,H,W", [(2, 48, 40), (1, 128, 128)])
def test_denoise_bm3d(cs, Z, H, W):
    noisy = _blobs(5 + W, Z, H, W)
    out = to_np(cs.denoise(to_dev(noisy), cs.Params(denoiser="bm3d", bm3d_sigma=0.04)))
    ref = oracle.bm3d(noisy, 0.04)
    assert rel_l2(out, ref) <= 1e-3
    clean = synth.generate(synth.Workload("b", Z, H, W, seed=5 + W, peak=None,
                                          n_blobs=max(4, Z * H * W // 300)))["x"]
    assert abs(oracle.psnr(out, clean) - oracle.psnr(ref, clean)) <= DPSNR


@pytest.mark.parametrize("gamma", [0.0, 0.2])
def test_one_iteration_bm3d(cs, gamma):
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
    v_r, u_r, d_r, _ = oracle.admm(b, masks, Z, rho=1.0, lam=0.0, gamma=gamma, iters=1,
                                   denoiser="bm3d", bm3d_sigma=0.04, u0=u0, d0=d0)
    assert rel_l2(to_np(v), v_r) <= REL_ITER
    ug = to_np(u)
    if gamma == 0.0:
        assert _close_with_flips(ug, u_r)
    else:
        # The first slice of the sweep sees the same inputs as the oracle up to
        # rounding.  Later slices take the previous slice's output as input, and
        # a hard-threshold or matching decision flipped by one FP32 rounding
        # changes whole groups (up to 27 pixels away) that the next slice then
        # sees: the sweep spreads such local changes, so the later slices are
        # held to the volume-level bar only.
        assert _close_with_flips(ug[0], u_r[0])
        assert rel_l2(ug, u_r) <= 1e-2, rel_l2(ug, u_r)
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
