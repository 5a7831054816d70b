"""3-D SSIM (Sec. IV) on the GPU through cslsm_ssim3d against the FP64 oracle:
ragged shapes, Z below / above the window, a single slice, identical volumes,
and the 512 x 512 x 16 benchmark reconstruction against its ground truth."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu

# FP32 window moments (E[x^2] - mean^2) against FP64: the mean over the volume
# agrees to a few 1e-7; the bar leaves an order of magnitude.
BAR = 5e-6


@pytest.fixture(scope="module")
def cs():
    import torch

    from paper_2511_03093_gb300 import build as b

    b.build()
    import paper_2511_03093_gb300 as m

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return m


def _pair(seed, shape):
    rng = np.random.default_rng(seed)
    w = synth.Workload("s", shape[0], shape[1], shape[2], seed=seed, peak=None,
                       n_blobs=max(4, int(np.prod(shape)) // 300))
    x = synth.generate(w)["x"].astype(np.float32)
    y = np.clip(x + 0.05 * rng.standard_normal(shape), 0, 1).astype(np.float32)
    return x, y


@pytest.mark.parametrize("shape", [(7, 33, 50), (16, 128, 128), (1, 64, 64), (20, 17, 300),
                                   (3, 5, 4), (11, 70, 65)])
def test_matches_oracle(cs, shape):
    x, y = _pair(sum(shape), shape)
    got = float(cs.ssim3d(to_dev(y), to_dev(x)))
    ref = oracle.ssim3d(y, x)
    assert abs(got - ref) <= BAR, (got, ref)


def test_identical_volumes(cs):
    x, _ = _pair(5, (9, 40, 70))
    assert abs(float(cs.ssim3d(to_dev(x), to_dev(x))) - 1.0) <= 1e-6


def test_deterministic(cs):
    x, y = _pair(6, (8, 96, 80))
    a = float(cs.ssim3d(to_dev(y), to_dev(x)))
    b = float(cs.ssim3d(to_dev(y), to_dev(x)))
    assert a == b


def test_benchmark_reconstruction(cs):
    """SSIM of a 10-iteration TV + z reconstruction of the 512 x 512 x 16
    benchmark workload against its ground truth, GPU vs oracle."""
    import torch

    wk = synth.WORKLOADS["tvz_512x512x16"]
    data = synth.generate(wk)
    plan = cs.Plan(wk.H, wk.W, 1, wk.Z, to_dev(data["masks"]))
    v = plan.solve(to_dev(data["b"]), cs.Params(rho=1.0, lam=0.05, gamma=0.2, iters=10,
                                                denoiser="tv", tv_inner=20))
    torch.cuda.synchronize()
    x = data["x"].astype(np.float32)
    got = float(cs.ssim3d(v, to_dev(x)))
    ref = oracle.ssim3d(v.cpu().numpy(), x)
    assert abs(got - ref) <= BAR, (got, ref)
    assert 0.0 < got < 1.0
    plan.close()
