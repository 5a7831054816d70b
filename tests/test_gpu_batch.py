"""Batched solver: one persistent launch under a CUDA graph over measurements of
uneven size and slice count.  Per measurement it must reproduce the plain
per-volume solve bit for bit (same FP32 / BF16 arithmetic, tiling does not
change any pixel's operations), replay identically, and report a device-side
wait that runs out as CSLSM_ERR_TIMEOUT without hanging."""
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


SIZES = [(8, 64, 64), (16, 96, 80), (4, 130, 101), (8, 40, 200), (1, 33, 47)]


@pytest.fixture(autouse=True)
def _per_launch_references(cs):
    """Per-volume reference solves take the per-launch TV tiles, never a batch."""
    cs.set_tv_route(1)
    yield
    cs.set_tv_route(0)


def _items(cs, seed0):
    import torch

    items, plans = [], []
    for k, (Z, H, W) in enumerate(SIZES):
        w = synth.Workload(f"b{k}", Z, H, W, drift=True, mask_p=0.3, peak=50.0, sigma_g=0.02,
                           seed=seed0 + k, n_blobs=max(4, Z * H * W // 400))
        data = synth.generate(w)
        plan = cs.Plan(H, W, 1, Z, to_dev(data["masks"]))
        b = to_dev(data["b"])
        v = torch.empty((Z, H, W), dtype=torch.float32, device="cuda")
        items.append((plan, b, v))
    return items


@pytest.mark.parametrize("gamma,storage,T", [(0.2, "fp32", 20), (0.0, "fp32", 20),
                                             (0.2, "bf16", 20), (0.2, "fp16", 7),
                                             (0.2, "fp32", 30), (0.0, "fp32", 3)])
def test_batch_equals_per_volume(cs, gamma, storage, T):
    import torch

    items = _items(cs, 500)
    prm = cs.Params(rho=1.0, lam=0.05, gamma=gamma, iters=12, denoiser="tv", tv_inner=T,
                    storage=storage)
    batch = cs.Batch(items, prm)
    batch.run()
    batch.wait()
    got = [to_np(v).copy() for _, _, v in items]
    batch.run()  # graph replay
    batch.wait()
    for (plan, b, v), g in zip(items, got):
        np.testing.assert_array_equal(to_np(v), g)
        ref = plan.solve(b, prm)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(g, to_np(ref))
    batch.close()


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_batch_equals_per_volume_benchmark_sizes(cs, storage):
    """Items of the 64-measurement benchmark's size distribution, including its
    largest (1024 x 1024 x 32), TV + z, 3 iterations: bit-identical to the plain
    per-volume solves."""
    import torch

    sizes = [(32, 1024, 1024), (8, 256, 256), (16, 768, 768)]
    items = []
    for k, (Z, S, _) in enumerate(sizes):
        w = synth.Workload(f"bb{k}", Z, S, S, drift=True, mask_p=0.3, peak=50.0, sigma_g=0.02,
                           seed=4100 + k, n_blobs=min(2000, synth.blob_count(Z, S, S)))
        data = synth.generate(w)
        plan = cs.Plan(S, S, 1, Z, to_dev(data["masks"]))
        items.append((plan, to_dev(data["b"]),
                      torch.empty((Z, S, S), dtype=torch.float32, device="cuda")))
    prm = cs.Params(rho=1.0, lam=0.05, gamma=0.2, iters=3, denoiser="tv", tv_inner=20,
                    storage=storage)
    batch = cs.Batch(items, prm)
    batch.run()
    batch.wait()
    for plan, b, v in items:
        ref = plan.solve(b, prm)
        torch.cuda.synchronize()
        assert torch.equal(v, ref)
    batch.close()
    for plan, _, _ in items:
        plan.close()


def test_batch_autotuned_tiles(cs):
    import torch

    items = _items(cs, 600)
    prm = cs.Params(rho=1.0, lam=0.05, gamma=0.2, iters=5, denoiser="tv", tv_inner=20)
    try:
        cs.set_autotune(1)
        batch = cs.Batch(items, prm)
    finally:
        cs.set_autotune(0)
    info = batch.info()
    assert info["steps_per_phase"] in (5, 7, 10, 20)  # ceil(20 / P), P = 1..4
    assert info["grid"] > 0 and info["grid"] % torch.cuda.get_device_properties(0).multi_processor_count == 0
    assert info["units_per_iteration"] > 0
    batch.run()
    batch.wait()
    for plan, b, v in items:
        ref = plan.solve(b, prm)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(to_np(v), to_np(ref))
    batch.close()


def test_batch_forced_steps_per_phase(cs):
    """A set phase length is used as given (clamped to T), with results equal to
    the per-volume solves."""
    import torch

    items = _items(cs, 650)[:3]
    prm = cs.Params(rho=1.0, lam=0.05, gamma=0.2, iters=4, denoiser="tv", tv_inner=20)
    try:
        cs.set_batch_steps_per_phase(3)
        batch = cs.Batch(items, prm)
        cs.set_batch_steps_per_phase(50)
        batch_t = cs.Batch(items, cs.Params(rho=1.0, lam=0.05, gamma=0.2, iters=4,
                                            denoiser="tv", tv_inner=7))
    finally:
        cs.set_batch_steps_per_phase(0)
    assert batch.info()["steps_per_phase"] == 3
    assert batch_t.info()["steps_per_phase"] == 7
    batch_t.close()
    batch.run()
    batch.wait()
    for plan, b, v in items:
        ref = plan.solve(b, prm)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(to_np(v), to_np(ref))
    batch.close()


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_routed_tv_solve_equals_per_launch(cs, storage):
    """Slice-independent TV solves routed through a one-item batch give the bits
    of the per-launch tiles: gamma = 0, and Z = 1 with gamma > 0; a stats request
    synchronises and reports; the kept batch is pointed at another measurement
    buffer, and at an output that plan.solve allocates."""
    import torch

    items = _items(cs, 900)
    for k, (plan, b, v) in enumerate(items):
        gamma = 0.2 if plan.vol_shape[0] == 1 else 0.0
        prm = cs.Params(rho=1.0, lam=0.05, gamma=gamma, iters=6, denoiser="tv", tv_inner=20,
                        storage=storage)
        cs.set_tv_route(1)
        ref = to_np(plan.solve(b, prm))
        cs.set_tv_route(2)
        out = plan.solve(b, prm, v_out=v)
        np.testing.assert_array_equal(to_np(out), ref)
        v.zero_()
        out, st = plan.solve(b, prm, v_out=v, stats=True)  # the kept batch, replayed
        assert st["iters_done"] == 6
        np.testing.assert_array_equal(to_np(out), ref)
        b2 = b.clone()  # another buffer, the same batch
        np.testing.assert_array_equal(to_np(plan.solve(b2, prm, v_out=v)), ref)
        np.testing.assert_array_equal(to_np(plan.solve(b2, prm)), ref)
        torch.cuda.synchronize()


@pytest.mark.parametrize("per_slice", [True, False])
def test_routed_tv_solve_multishot(cs, per_slice):
    """Several coded shots of R planes (patterns per slice, or shared by every
    shot): the routed solve and a batch of the item give the bits of the
    per-launch tiles."""
    import torch

    Z, H, W, N = 12, 72, 88, 3
    R = Z // N
    wk = synth.Workload("ms", Z, H, W, n_shots=N, per_slice_masks=per_slice, drift=True,
                        mask_p=0.5, peak=200.0, sigma_g=0.01, seed=1400 + int(per_slice),
                        n_blobs=40)
    data = synth.generate(wk)
    plan = cs.Plan(H, W, N, R, to_dev(data["masks"]), per_slice=per_slice)
    b = to_dev(data["b"])
    prm = cs.Params(rho=1.0, lam=0.05, gamma=0.0, iters=5, denoiser="tv", tv_inner=20)
    cs.set_tv_route(1)
    ref = to_np(plan.solve(b, prm))
    cs.set_tv_route(2)
    np.testing.assert_array_equal(to_np(plan.solve(b, prm)), ref)
    v = torch.empty(plan.vol_shape, dtype=torch.float32, device="cuda")
    batch = cs.Batch([(plan, b, v)], prm)
    batch.run()
    batch.wait()
    np.testing.assert_array_equal(to_np(v), ref)
    batch.close()
    plan.close()


def test_batch_wait_timeout_is_reported(cs):
    items = _items(cs, 700)[:2]
    prm = cs.Params(rho=1.0, lam=0.05, gamma=0.2, iters=3, denoiser="tv", tv_inner=10)
    batch = cs.Batch(items, prm)
    batch.set_wait_limit(0.05, test_stall=True)
    batch.run()
    with pytest.raises(cs.CslsmError) as ei:
        batch.wait()
    assert ei.value.status == 3  # CSLSM_ERR_TIMEOUT
    batch.set_wait_limit(4.0, test_stall=False)
    batch.run()
    batch.wait()  # the context is still usable and a normal run completes
    batch.close()


def test_batch_rejects_unsupported(cs):
    items = _items(cs, 800)[:1]
    for prm in (cs.Params(denoiser="bm3d"), cs.Params(denoiser="tv", tol=1e-3)):
        with pytest.raises(cs.CslsmError):
            cs.Batch(items, prm)


ORACLE_SIZES = [(8, 64, 64), (4, 130, 101), (16, 48, 72)]


def _oracle_items(cs, seed0):
    import torch

    items, datas = [], []
    for k, (Z, H, W) in enumerate(ORACLE_SIZES):
        w = synth.Workload(f"o{k}", Z, H, W, drift=True, mask_p=0.3, peak=50.0, sigma_g=0.02,
                           seed=seed0 + k, n_blobs=max(4, Z * H * W // 400))
        data = synth.generate(w)
        plan = cs.Plan(H, W, 1, Z, to_dev(data["masks"]))
        items.append((plan, to_dev(data["b"]), torch.empty((Z, H, W), dtype=torch.float32,
                                                           device="cuda")))
        datas.append(data)
    return items, datas


def test_batch_items_match_fp64_oracle_one_iteration(cs):
    """Every item of an uneven FP32 batch, one iteration of Algorithm 1 (TV + z),
    against the FP64 oracle run on the same measurement."""
    items, datas = _oracle_items(cs, 900)
    prm = cs.Params(rho=1.0, lam=0.05, gamma=0.2, iters=1, denoiser="tv", tv_inner=20)
    batch = cs.Batch(items, prm)
    batch.run()
    batch.wait()
    for (plan, b, v), data, (Z, H, W) in zip(items, datas, ORACLE_SIZES):
        ref, *_ = oracle.admm(data["b64"], data["masks"], Z, rho=1.0, lam=0.05, gamma=0.2,
                              iters=1, denoiser="tv", tv_inner=20)
        assert rel_l2(to_np(v), ref) <= REL_ITER, (Z, H, W)
    batch.close()


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_batch_items_full_run_psnr_matches_fp64_oracle(cs, storage):
    """Whole 40-iteration solves of every item: reconstruction PSNR within 0.05 dB
    of the FP64 oracle's, for FP32 and for BF16 state storage."""
    items, datas = _oracle_items(cs, 950)
    prm = cs.Params(rho=1.0, lam=0.05, gamma=0.2, iters=40, denoiser="tv", tv_inner=20,
                    storage=storage)
    batch = cs.Batch(items, prm)
    batch.run()
    batch.wait()
    for (plan, b, v), data, (Z, H, W) in zip(items, datas, ORACLE_SIZES):
        ref, *_ = oracle.admm(data["b64"], data["masks"], Z, rho=1.0, lam=0.05, gamma=0.2,
                              iters=40, denoiser="tv", tv_inner=20)
        p_gpu = oracle.psnr(to_np(v), data["x"])
        p_ref = oracle.psnr(ref, data["x"])
        assert abs(p_gpu - p_ref) <= DPSNR, (storage, Z, H, W, p_gpu, p_ref)
    batch.close()


@pytest.mark.parametrize("shift", [1, 2])
def test_batch_with_unaligned_caller_buffers(cs, shift):
    """Measurements and outputs that start `shift` floats past a 16-byte boundary
    (views into larger tensors): the x-update takes its one-pixel path for a
    4-byte offset and its two-pixel path for an 8-byte one (H W is a multiple of
    4, so aligned buffers would take the four-pixel path), and the batch still
    reproduces the per-volume solves bit for bit."""
    import torch

    items = []
    for k, (Z, H, W) in enumerate([(8, 64, 64), (4, 48, 40)]):
        w = synth.Workload(f"ua{k}", Z, H, W, drift=True, mask_p=0.3, peak=50.0, sigma_g=0.02,
                           seed=1300 + k, n_blobs=20)
        data = synth.generate(w)
        plan = cs.Plan(H, W, 1, Z, to_dev(data["masks"]))
        bbig = torch.zeros(H * W + shift, dtype=torch.float32, device="cuda")
        bbig[shift:] = to_dev(data["b"]).reshape(-1)
        b = bbig[shift:].view(1, H, W)
        vbig = torch.empty(Z * H * W + shift, dtype=torch.float32, device="cuda")
        v = vbig[shift:].view(Z, H, W)
        assert b.data_ptr() % 16 == 4 * shift and v.data_ptr() % 16 == 4 * shift
        items.append((plan, b, v))
    prm = cs.Params(rho=1.0, lam=0.05, gamma=0.2, iters=6, denoiser="tv", tv_inner=20,
                    storage="bf16")
    batch = cs.Batch(items, prm)
    batch.run()
    batch.wait()
    for plan, b, v in items:
        ref = plan.solve(b.contiguous(), prm)
        torch.cuda.synchronize()
        assert torch.equal(v, ref)
    batch.close()
