"""Tolerance-stopped solves (Sec. IV-B stopping rule) checked on the device: the
iteration count agrees with the FP64 oracle's, and the stopped state equals a
fixed-count solve of that many iterations bit for bit (every kernel after the
stop returns at once), for the TV + z sweep, TV, Tikhonov and BM3D paths, with the
paper's caps (100 iterations / 1e-3, 200 iterations / 1e-2)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cs():
    from paper_2511_03093_gb300 import build as b

    b.build()
    import paper_2511_03093_gb300 as m

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return m


def _solve(cs, plan, b, **kw):
    prm = cs.Params(**kw)
    u = torch.empty(plan.vol_shape, dtype=torch.float32, device="cuda")
    d = torch.empty(plan.vol_shape, dtype=torch.float32, device="cuda")
    v, st = plan.solve(b, prm, u=u, d=d, stats=True)
    torch.cuda.synchronize()
    return v.cpu(), u.cpu(), d.cpu(), st


@pytest.mark.parametrize("den,gamma,iters,tol,every", [
    ("tv", 0.2, 100, 1e-3, 1), ("tv", 0.2, 200, 1e-2, 1), ("tv", 0.0, 100, 1e-2, 2),
    ("tikhonov", 0.3, 200, 1e-3, 3), ("bm3d", 0.0, 40, 2e-2, 2)])
def test_stopped_state_equals_fixed_count_solve(cs, den, gamma, iters, tol, every):
    w = synth.Workload("tol", 8, 64, 56, drift=True, mask_p=0.3, peak=50.0, sigma_g=0.02,
                       seed=31, n_blobs=40)
    data = synth.generate(w)
    plan = cs.Plan(w.H, w.W, 1, w.Z, to_dev(data["masks"]))
    b = to_dev(data["b"])
    kw = dict(rho=1.0, lam=0.0 if den == "bm3d" else 0.05, gamma=gamma, denoiser=den,
              tv_inner=20, bm3d_sigma=0.05)
    v, u, d, st = _solve(cs, plan, b, iters=iters, tol=tol, check_every=every, **kw)
    k = st["iters_done"]
    assert 1 <= k <= iters
    if k < iters:
        assert 0 < st["rel_change"] < tol
    v2, u2, d2, st2 = _solve(cs, plan, b, iters=k, **kw)
    assert st2["iters_done"] == k
    assert torch.equal(v, v2) and torch.equal(u, u2) and torch.equal(d, d2)
    plan.close()


@pytest.mark.parametrize("iters,tol", [(100, 1e-3), (200, 1e-2)])
def test_iteration_count_matches_oracle(cs, iters, tol):
    """TV + z at the paper's caps: the GPU stops within one check of the oracle."""
    w = synth.Workload("tolz", 6, 48, 40, drift=True, mask_p=0.3, peak=50.0, sigma_g=0.02,
                       seed=41, n_blobs=30)
    data = synth.generate(w)
    plan = cs.Plan(w.H, w.W, 1, w.Z, to_dev(data["masks"]))
    kw = dict(rho=1.0, lam=0.05, gamma=0.2, denoiser="tv", tv_inner=20)
    v, _, _, st = _solve(cs, plan, to_dev(data["b"]), iters=iters, tol=tol, check_every=1, **kw)
    v_r, _, _, k = oracle.admm(data["b64"], data["masks"], w.Z, iters=iters, tol=tol, **{
        "rho": 1.0, "lam": 0.05, "gamma": 0.2, "denoiser": "tv", "tv_inner": 20})
    assert abs(st["iters_done"] - k) <= 1, (st["iters_done"], k)
    if st["iters_done"] == k:
        rel = np.linalg.norm(to_np(v) - v_r) / np.linalg.norm(v_r)
        assert rel <= 1e-4
    plan.close()
