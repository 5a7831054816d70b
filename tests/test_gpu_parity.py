"""CUDA path vs the FP64 oracle, through the C ABI, on identical seeded inputs.

Bars (from the FP32 arithmetic of the path):
  - adjoint and mask packing: bit-exact;
  - forward, denoisers, one ADMM iteration: relative L2 <= 1e-5;
  - full runs: reconstruction PSNR within 0.05 dB of the oracle's.
Sizes span several 32 x 32 tiles with ragged edges; the bench workload
(512 x 512 x 16, TV + z) is covered by one-iteration parity from oracle states.
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


GEOMS = [
    # N, R, H, W, per_slice
    (1, 8, 37, 53, True),
    (2, 3, 40, 33, True),
    (3, 4, 29, 64, False),
    (1, 32, 64, 70, True),
    (1, 1, 17, 19, True),
    (1, 16, 1, 45, True),
    (2, 5, 33, 1, False),
]


def _geom_inputs(seed, N, R, H, W, per_slice, p=0.5):
    rng = np.random.default_rng(seed)
    Z = N * R
    masks = (rng.random((Z if per_slice else R, H, W)) < p).astype(np.uint8)
    v = rng.standard_normal((Z, H, W)).astype(np.float32)
    b = (rng.random((N, H, W)) * 2).astype(np.float32)
    return masks, v, b


@pytest.mark.parametrize("N,R,H,W,per_slice", GEOMS)
def test_forward_adjoint(cs, N, R, H, W, per_slice):
    masks, v, b = _geom_inputs(1, N, R, H, W, per_slice)
    plan = cs.Plan(H, W, N, R, to_dev(masks), per_slice)
    bg = plan.forward(to_dev(v))
    vg = plan.adjoint(to_dev(b))
    b_ref = oracle.forward(v, masks, N)
    v_ref = oracle.adjoint(b, masks, N * R)
    assert rel_l2(to_np(bg), b_ref) <= 1e-6
    np.testing.assert_array_equal(to_np(vg), v_ref)  # products with {0,1}: exact
    plan.close()


def test_set_masks_repacks(cs):
    N, R, H, W = 1, 6, 35, 41
    m1, v, _ = _geom_inputs(2, N, R, H, W, True)
    m2, _, _ = _geom_inputs(3, N, R, H, W, True)
    plan = cs.Plan(H, W, N, R, to_dev(m1))
    plan.set_masks(to_dev(m2))
    assert rel_l2(to_np(plan.forward(to_dev(v))), oracle.forward(v, m2, N)) <= 1e-6
    plan.close()


@pytest.mark.parametrize("shape", [(3, 70, 45), (1, 1, 50), (2, 33, 1), (1, 128, 128),
                                   (2, 97, 131)])
@pytest.mark.parametrize("T,lam", [(1, 0.05), (5, 0.3), (20, 0.05), (40, 0.1), (41, 0.05),
                                   (100, 0.2)])
def test_denoise_tv(cs, shape, T, lam):
    rng = np.random.default_rng(T * 7 + shape[1])
    x = rng.random(shape).astype(np.float32)
    prm = cs.Params(rho=1.0, lam=lam, tv_inner=T, denoiser="tv")
    out = to_np(cs.denoise(to_dev(x), prm))
    ref = oracle.tv_prox(x, lam / 1.0, T)
    assert rel_l2(out, ref) <= REL_ITER


@pytest.mark.parametrize("mode", [2, 3, 4, 5, 1])
@pytest.mark.parametrize("shape,T", [((3, 70, 45), 20), ((1, 131, 97), 7), ((2, 256, 200), 24)])
def test_tv_kernel_variants(cs, mode, shape, T):
    """Every TV kernel variant (forced) and the timed autotuner give the oracle's prox."""
    rng = np.random.default_rng(T + shape[1])
    x = rng.random(shape).astype(np.float32)
    prm = cs.Params(rho=1.0, lam=0.1, tv_inner=T, denoiser="tv")
    try:
        cs.set_autotune(mode)
        out = to_np(cs.denoise(to_dev(x), prm))
        out2 = to_np(cs.denoise(to_dev(x), prm))  # the tuned (cached) choice
    finally:
        cs.set_autotune(0)
    ref = oracle.tv_prox(x, 0.1, T)
    assert rel_l2(out, ref) <= REL_ITER
    np.testing.assert_array_equal(out, out2) if mode >= 2 else None
    assert rel_l2(out2, ref) <= REL_ITER


def test_denoise_tv_zero_weight_is_identity(cs):
    x = np.random.default_rng(0).random((2, 40, 50)).astype(np.float32)
    out = to_np(cs.denoise(to_dev(x), cs.Params(lam=0.0, denoiser="tv")))
    np.testing.assert_array_equal(out, x)


def test_denoise_tikhonov(cs):
    x = np.random.default_rng(0).standard_normal((3, 20, 30)).astype(np.float32)
    prm = cs.Params(rho=0.7, lam=0.2, denoiser="tikhonov")
    out = to_np(cs.denoise(to_dev(x), prm))
    assert rel_l2(out, 0.7 * x.astype(np.float64) / (0.4 + 0.7)) <= 1e-7


ITER_CASES = [
    # denoiser, gamma, geometry
    ("tikhonov", 0.0, (1, 8, 37, 53, True)),
    ("tikhonov", 0.3, (1, 8, 37, 53, True)),
    ("tikhonov", 0.3, (3, 4, 29, 64, False)),
    ("tikhonov", 0.5, (1, 2, 20, 24, True)),
    ("tikhonov", 0.3, (1, 32, 33, 40, True)),
    ("tv", 0.0, (1, 8, 37, 53, True)),
    ("tv", 0.0, (2, 3, 40, 33, True)),
    ("tv", 0.2, (1, 8, 37, 53, True)),
    ("tv", 0.2, (3, 4, 29, 64, False)),
    ("tv", 0.4, (1, 2, 36, 30, True)),
    ("tv", 0.2, (1, 16, 70, 66, True)),
    # degenerate geometries: one slice with gamma > 0 (no z term), a single pixel,
    # single-row and single-column slices, two one-plane shots (the cyclic z
    # neighbours of each slice are the same slice)
    ("tv", 0.2, (1, 1, 37, 53, True)),
    ("tikhonov", 0.3, (1, 1, 5, 5, True)),
    ("tv", 0.0, (1, 1, 1, 1, True)),
    ("tv", 0.2, (1, 3, 1, 70, True)),
    ("tv", 0.2, (1, 3, 70, 1, True)),
    ("tv", 0.2, (2, 1, 17, 19, True)),
    ("tikhonov", 0.3, (2, 1, 17, 19, True)),
]


@pytest.mark.parametrize("den,gamma,geom", ITER_CASES)
def test_one_iteration_from_state(cs, den, gamma, geom):
    """One Algorithm-1 iteration from a random (u, d) state."""
    import torch

    N, R, H, W, per_slice = geom
    Z = N * R
    rng = np.random.default_rng(11)
    masks = (rng.random((Z if per_slice else R, H, W)) < 0.5).astype(np.uint8)
    b = (rng.random((N, H, W)) * 3).astype(np.float32)
    u0 = rng.random((Z, H, W)).astype(np.float32)
    d0 = (0.1 * rng.standard_normal((Z, H, W))).astype(np.float32)
    prm = cs.Params(rho=0.8, lam=0.07, gamma=gamma, iters=1, denoiser=den, tv_inner=20)
    plan = cs.Plan(H, W, N, R, to_dev(masks), per_slice)
    u = to_dev(u0)
    d = to_dev(d0)
    v = plan.solve(to_dev(b), prm, u=u, d=d, init_user=True)
    torch.cuda.synchronize()
    v_r, u_r, d_r, _ = oracle.admm(b, masks, Z, rho=0.8, lam=0.07, gamma=gamma, iters=1,
                                   denoiser=den, tv_inner=20, u0=u0, d0=d0)
    assert rel_l2(to_np(v), v_r) <= REL_ITER
    assert rel_l2(to_np(u), u_r) <= REL_ITER
    assert rel_l2(to_np(d), d_r) <= REL_ITER
    plan.close()


@pytest.mark.parametrize("fill", [0, 1])
@pytest.mark.parametrize("den", ["tv", "tikhonov"])
def test_one_iteration_constant_patterns(cs, fill, den):
    """Every DMD pattern closed (D = 0: the x-update keeps g) or open (D = R)."""
    import torch

    N, R, H, W = 1, 5, 33, 41
    rng = np.random.default_rng(30 + fill)
    masks = np.full((R, H, W), fill, dtype=np.uint8)
    b = (rng.random((N, H, W)) * 3).astype(np.float32)
    u0 = rng.random((R, H, W)).astype(np.float32)
    d0 = (0.1 * rng.standard_normal((R, H, W))).astype(np.float32)
    kw = dict(rho=0.8, lam=0.07, gamma=0.2, iters=1, denoiser=den, tv_inner=20)
    plan = cs.Plan(H, W, N, R, to_dev(masks))
    u, d = to_dev(u0), to_dev(d0)
    v = plan.solve(to_dev(b), cs.Params(**kw), u=u, d=d, init_user=True)
    torch.cuda.synchronize()
    v_r, u_r, d_r, _ = oracle.admm(b, masks, R, u0=u0, d0=d0, **kw)
    assert rel_l2(to_np(v), v_r) <= REL_ITER
    assert rel_l2(to_np(u), u_r) <= REL_ITER
    assert rel_l2(to_np(d), d_r) <= REL_ITER
    if fill == 0:  # nothing measured: v = u - d exactly
        np.testing.assert_array_equal(to_np(v), u0 - d0)
    plan.close()


@pytest.mark.parametrize("T", [1, 2, 3])
def test_one_iteration_few_tv_steps(cs, T):
    """The TV + z u-step with one to three Chambolle steps (a phase shorter than the
    halo logic's usual k) against the oracle."""
    import torch

    N, R, H, W = 1, 6, 45, 77
    rng = np.random.default_rng(20 + T)
    masks = (rng.random((R, H, W)) < 0.5).astype(np.uint8)
    b = (rng.random((N, H, W)) * 3).astype(np.float32)
    u0 = rng.random((R, H, W)).astype(np.float32)
    d0 = (0.1 * rng.standard_normal((R, H, W))).astype(np.float32)
    prm = cs.Params(rho=0.8, lam=0.07, gamma=0.2, iters=1, denoiser="tv", tv_inner=T)
    plan = cs.Plan(H, W, N, R, to_dev(masks))
    u, d = to_dev(u0), to_dev(d0)
    v = plan.solve(to_dev(b), prm, u=u, d=d, init_user=True)
    torch.cuda.synchronize()
    v_r, u_r, d_r, _ = oracle.admm(b, masks, R, rho=0.8, lam=0.07, gamma=0.2, iters=1,
                                   denoiser="tv", tv_inner=T, u0=u0, d0=d0)
    assert rel_l2(to_np(v), v_r) <= REL_ITER
    assert rel_l2(to_np(u), u_r) <= REL_ITER
    assert rel_l2(to_np(d), d_r) <= REL_ITER
    plan.close()


def _full_run(cs, w, prm, iters_oracle=None):
    import torch

    data = synth.generate(w)
    plan = cs.Plan(w.H, w.W, w.n_shots, w.R, to_dev(data["masks"]), w.per_slice_masks)
    v = plan.solve(to_dev(data["b"]), prm)
    torch.cuda.synchronize()
    v_r, *_ = oracle.admm(data["b64"], data["masks"], w.Z, rho=prm.rho, lam=prm.lam,
                          gamma=prm.gamma, iters=prm.iters, denoiser=prm.denoiser,
                          tv_inner=prm.tv_inner)
    vg = to_np(v)
    p_gpu = oracle.psnr(vg, data["x"])
    p_ref = oracle.psnr(v_r, data["x"])
    # the GPU PSNR kernel agrees with the oracle's definition
    p_kernel = float(cs.psnr(v, to_dev(data["x"].astype(np.float32))).item())
    plan.close()
    return p_gpu, p_ref, p_kernel, rel_l2(vg, v_r), oracle.psnr(vg, data["x"].astype(np.float32))


def test_full_run_tv_128x128x8(cs):
    """50 iterations, 20 inner TV steps, rho = 1, lambda = 0.05 on the 128 x 128 x 8 workload."""
    w = synth.WORKLOADS["tv_128x128x8"]
    prm = cs.Params(rho=1.0, lam=0.05, gamma=0.0, iters=50, denoiser="tv", tv_inner=20)
    p_gpu, p_ref, p_kernel, rel, p32 = _full_run(cs, w, prm)
    assert abs(p_gpu - p_ref) <= DPSNR, (p_gpu, p_ref)
    assert abs(p_kernel - p32) <= 1e-6
    assert rel <= 1e-3


@pytest.mark.parametrize("den,gamma", [("tv", 0.2), ("tikhonov", 0.0), ("tikhonov", 0.3)])
def test_full_run_small_drifting(cs, den, gamma):
    w = synth.Workload("drift_small", 12, 96, 112, drift=True, mask_p=0.3, peak=50.0,
                       sigma_g=0.02, seed=77)
    prm = cs.Params(rho=1.0, lam=0.05, gamma=gamma, iters=40, denoiser=den, tv_inner=20)
    p_gpu, p_ref, _, rel, _ = _full_run(cs, w, prm)
    assert abs(p_gpu - p_ref) <= DPSNR, (p_gpu, p_ref)
    assert rel <= 1e-3


def test_full_run_multi_shot_shared_masks(cs):
    w = synth.Workload("shots", 12, 64, 48, n_shots=3, per_slice_masks=False, mask_p=0.5,
                       seed=5, n_blobs=60)
    prm = cs.Params(rho=1.0, lam=0.05, gamma=0.1, iters=30, denoiser="tv", tv_inner=10)
    p_gpu, p_ref, _, rel, _ = _full_run(cs, w, prm)
    assert abs(p_gpu - p_ref) <= DPSNR
    assert rel <= 1e-3


def test_tolerance_stop_matches_oracle(cs):
    import torch

    w = synth.Workload("tol", 8, 48, 40, seed=9, n_blobs=30)
    data = synth.generate(w)
    plan = cs.Plan(w.H, w.W, 1, w.Z, to_dev(data["masks"]))
    prm = cs.Params(rho=1.0, lam=0.05, iters=300, tol=1e-3, check_every=1, denoiser="tikhonov")
    v, st = plan.solve(to_dev(data["b"]), prm, stats=True)
    torch.cuda.synchronize()
    v_r, _, _, k = oracle.admm(data["b64"], data["masks"], w.Z, rho=1.0, lam=0.05, iters=300,
                               tol=1e-3, denoiser="tikhonov")
    assert abs(st["iters_done"] - k) <= 1
    assert st["iters_done"] < 300 and 0 < st["rel_change"] < 1e-3
    v_k, *_ = oracle.admm(data["b64"], data["masks"], w.Z, rho=1.0, lam=0.05,
                          iters=st["iters_done"], denoiser="tikhonov")
    assert rel_l2(to_np(v), v_k) <= 1e-5
    plan.close()


def test_psnr_kernel(cs):
    rng = np.random.default_rng(3)
    x = rng.random((5, 33, 47)).astype(np.float32)
    ref = rng.random((5, 33, 47)).astype(np.float32)
    got = float(cs.psnr(to_dev(x), to_dev(ref)).item())
    assert got == pytest.approx(oracle.psnr(x, ref), abs=1e-9)


@pytest.mark.parametrize("k_oracle", [0, 2])
def test_bench_workload_one_iteration(cs, k_oracle):
    """512 x 512 x 16 TV + z (the benchmark's launch configuration): one GPU iteration
    from the oracle's state after k_oracle iterations, against the oracle's next one."""
    import torch

    w = synth.WORKLOADS["tvz_512x512x16"]
    data = synth.generate(w)
    kw = dict(rho=1.0, lam=0.05, gamma=0.2, denoiser="tv", tv_inner=20)
    if k_oracle:
        _, u0, d0, _ = oracle.admm(data["b64"], data["masks"], w.Z, iters=k_oracle, **kw)
    else:
        u0 = d0 = np.zeros((w.Z, w.H, w.W))
    u0 = u0.astype(np.float32)
    d0 = d0.astype(np.float32)
    v_r, u_r, d_r, _ = oracle.admm(data["b64"], data["masks"], w.Z, iters=1, u0=u0, d0=d0, **kw)
    plan = cs.Plan(w.H, w.W, 1, w.Z, to_dev(data["masks"]))
    u, d = to_dev(u0), to_dev(d0)
    v = plan.solve(to_dev(data["b"]), cs.Params(iters=1, **kw), u=u, d=d, init_user=True)
    torch.cuda.synchronize()
    assert rel_l2(to_np(v), v_r) <= REL_ITER
    assert rel_l2(to_np(u), u_r) <= REL_ITER
    assert rel_l2(to_np(d), d_r) <= REL_ITER
    plan.close()


def test_bench_workload_full_run(cs):
    """The benchmark's whole 100-iteration TV + z solve at 512 x 512 x 16: the GPU
    reconstruction's PSNR is within 0.05 dB of the oracle's."""
    w = synth.WORKLOADS["tvz_512x512x16"]
    prm = cs.Params(rho=1.0, lam=0.05, gamma=0.2, iters=100, denoiser="tv", tv_inner=20)
    p_gpu, p_ref, p_kernel, rel, p32 = _full_run(cs, w, prm)
    assert abs(p_gpu - p_ref) <= DPSNR, (p_gpu, p_ref)
    assert abs(p_kernel - p32) <= 1e-6
    assert rel <= 1e-3
