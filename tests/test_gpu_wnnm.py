"""WNNM u-step: CUDA path (one-sided Jacobi per group in FP32) vs the FP64 oracle
(library SVD) through the C ABI.  The groups come from the same bit-exact block
matching as BM3D; the weighted soft threshold is continuous in the singular
values, so the denoiser agrees to FP32 accuracy (bar: relative L2 2e-4); ADMM runs
within 0.05 dB PSNR of the oracle; repeated calls are bit-identical."""
import numpy as np
import pytest

import oracle
import synth
from oracle import wnnm as wn
from tests.gpu_util import DPSNR, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

BAR = 2e-4


@pytest.fixture(scope="module")
def cs():
    import torch

    from paper_2511_03093_gb300 import build as b

    b.build()
    import paper_2511_03093_gb300 as m

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return m


def _noisy(seed, Z, H, W, noise=0.05):
    w = synth.Workload("w", Z, H, W, seed=seed, peak=None, n_blobs=max(4, Z * H * W // 300))
    rng = np.random.default_rng(seed + 1)
    x = synth.generate(w)["x"]
    return x, (x + noise * rng.standard_normal(x.shape)).astype(np.float32)


@pytest.mark.parametrize("Z,H,W", [(2, 37, 53), (1, 64, 70), (1, 8, 8), (2, 9, 20), (1, 7, 30)])
def test_denoise_matches_oracle(cs, Z, H, W):
    _, noisy = _noisy(H + W, Z, H, W)
    out = to_np(cs.denoise(to_dev(noisy), cs.Params(denoiser="wnnm", bm3d_sigma=0.05)))
    ref = wn.wnnm(noisy.astype(np.float64), 0.05)
    assert rel_l2(out, ref) <= BAR, rel_l2(out, ref)


def test_denoises_and_is_deterministic(cs):
    clean, noisy = _noisy(3, 2, 96, 80)
    p = cs.Params(denoiser="wnnm", bm3d_sigma=0.05)
    a = to_np(cs.denoise(to_dev(noisy), p))
    b = to_np(cs.denoise(to_dev(noisy), p))
    np.testing.assert_array_equal(a, b)
    assert np.linalg.norm(a - clean) < 0.8 * np.linalg.norm(noisy - clean)


@pytest.mark.parametrize("gamma", [0.0, 0.2])
def test_full_run_psnr_matches_oracle(cs, gamma):
    import torch

    w = synth.Workload("wa", 6, 48, 40, drift=True, mask_p=0.5, peak=200.0, sigma_g=0.01,
                       seed=77, n_blobs=40)
    data = synth.generate(w)
    plan = cs.Plan(w.H, w.W, 1, w.Z, to_dev(data["masks"]))
    prm = cs.Params(rho=1.0, lam=0.0, gamma=gamma, iters=8, denoiser="wnnm", bm3d_sigma=0.05)
    v = to_np(plan.solve(to_dev(data["b"]), prm))
    torch.cuda.synchronize()
    v_r, *_ = wn.admm_wnnm(data["b64"], data["masks"], w.Z, rho=1.0, gamma=gamma, sigma=0.05,
                           iters=8)
    p_gpu, p_ref = oracle.psnr(v, data["x"]), oracle.psnr(v_r, data["x"])
    assert abs(p_gpu - p_ref) <= DPSNR, (p_gpu, p_ref)
    assert rel_l2(v, v_r) <= 1e-2
    plan.close()
