"""Parity at the full size of the 1024 x 1024 x 32 configuration (Bernoulli(0.5)
patterns, Poisson peak 200 + Gaussian 0.01), in the launch configurations the
benchmark's secondary workloads time: one whole ADMM iteration with the Tikhonov
prior and with the TV prior (gamma = 0) against the FP64 oracle's iteration, and
the BM3D match lists of one full 1024 x 1024 slice, bit for bit.  The smaller
parity tests cover ragged shapes; these cover the sizes where tiles, grids and
reductions run at their largest.  Both BM3D stages are also checked on one full
1024 x 1024 slice."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import REL_ITER, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cs():
    import torch

    from paper_2511_03093_gb300 import build as b

    b.build()
    import paper_2511_03093_gb300 as m

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return m


@pytest.fixture(scope="module")
def cfg3():
    wk = synth.WORKLOADS["bm3d_1024x1024x32"]
    return wk, synth.generate(wk)


@pytest.mark.parametrize("den", ["tikhonov", "tv"])
def test_one_iteration_full_size(cs, cfg3, den):
    """One GPU iteration from u = d = 0 (x-update, the prior's u-step over all 32
    slices, dual update) against the oracle's first iteration."""
    import torch

    wk, data = cfg3
    kw = dict(rho=1.0, lam=0.05, gamma=0.0, denoiser=den, tv_inner=20)
    v_r, u_r, d_r, _ = oracle.admm(data["b64"], data["masks"], wk.Z, iters=1, **kw)
    plan = cs.Plan(wk.H, wk.W, 1, wk.Z, to_dev(data["masks"]))
    zeros = np.zeros((wk.Z, wk.H, wk.W), dtype=np.float32)
    u, d = to_dev(zeros), to_dev(zeros)
    v = plan.solve(to_dev(data["b"]), cs.Params(iters=1, **kw), u=u, d=d, init_user=True)
    torch.cuda.synchronize()
    assert rel_l2(to_np(v), v_r) <= REL_ITER
    assert rel_l2(to_np(u), u_r) <= REL_ITER
    assert rel_l2(to_np(d), d_r) <= REL_ITER
    plan.close()


def test_bm3d_match_full_slice(cs, cfg3):
    """Hard-stage block matching of one full 1024 x 1024 slice of noisy data (115,600
    references): lists and counts equal the oracle's exactly."""
    wk, data = cfg3
    rng = np.random.default_rng(1003)
    img = np.clip(data["x"][5] + 0.05 * rng.standard_normal((wk.H, wk.W)), -0.2, 1.2)
    img = img.astype(np.float32)[None]
    lists, counts = cs.bm3d_match(to_dev(img), 1)
    idx, cnt = oracle.bm3d_match(img[0], 1)
    np.testing.assert_array_equal(counts.cpu().numpy()[0], cnt)
    np.testing.assert_array_equal(lists.cpu().numpy()[0], idx)


def test_bm3d_stages_full_slice(cs):
    """Both BM3D stages on one full 1024 x 1024 slice of noisy data (sigma 0.05):
    the hard stage element-wise within relative L2 1e-5 outside the footprints of
    the groups whose kept-coefficient count differs from the oracle's (counted,
    a small fraction); the Wiener stage on the oracle's basic estimate within
    1e-5."""
    from tests import bm3d_check as bc

    w = synth.Workload("s", 1, 1024, 1024, seed=1003, peak=None,
                       n_blobs=synth.blob_count(1, 1024, 1024))
    x = synth.generate(w)["x"][0]
    img = (x + 0.05 * np.random.default_rng(3).standard_normal(x.shape)).astype(np.float32)
    chk = bc.Check()
    basic, basic_r, keep = bc.hard_stage(cs, img[None], 0.05, chk)
    assert bc.rel_on(basic, basic_r, keep) <= REL_ITER, (bc.rel_on(basic, basic_r, keep),
                                                        chk.flipped)
    assert chk.flipped <= 0.01 * chk.groups and chk.kept_pixels >= 0.5 * chk.pixels
    guide = basic_r[0].astype(np.float32)
    wien_r = oracle.bm3d_stage(img, 0.05, guide=guide)
    wien = to_np(cs.bm3d_stage(2, to_dev(img[None]), 0.05, guide=to_dev(guide[None])))[0]
    assert rel_l2(wien, wien_r) <= REL_ITER
