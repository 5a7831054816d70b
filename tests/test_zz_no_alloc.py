"""The allocation-free BM3D entry point, for callers that cannot allocate
device memory when they denoise: it must give what the allocating BM3D
denoiser gives, call after call, from its fixed scratch array.

Collected last on purpose (file name), so that a run stopping at its first
failure has run every other test before this one."""
import ctypes

import numpy as np
import pytest

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


def _noisy(seed, Z, H, W):
    w = synth.Workload("na", Z, H, W, seed=seed, peak=None, n_blobs=max(4, Z * H * W // 300))
    x = synth.generate(w)["x"]
    return (x + 0.04 * np.random.default_rng(seed).standard_normal(x.shape)).astype(np.float32)


def test_no_alloc_matches_allocating_denoiser_twice(cs):
    import torch

    L = cs.lib()
    shapes = [(2, 70, 90), (1, 128, 96)]
    for call, (Z, H, W) in enumerate(shapes + shapes[:1]):
        x = to_dev(_noisy(40 + call, Z, H, W))
        out = torch.empty_like(x)
        st = L.cslsm_denoise_bm3d_noalloc(ctypes.c_void_p(x.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()), Z, H, W,
                                          ctypes.c_float(0.04),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == 0, L.cslsm_last_error()
        ref = cs.denoise(x, cs.Params(denoiser="bm3d", bm3d_sigma=0.04))
        torch.cuda.synchronize()
        assert rel_l2(to_np(out), to_np(ref)) <= REL_ITER


def test_no_alloc_allocates_nothing_after_first_use(cs):
    import torch

    x = to_dev(_noisy(7, 1, 64, 64))
    out = torch.empty_like(x)
    cs.denoise_bm3d_noalloc(x, 0.05, out=out)  # first use on this device: address set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        cs.denoise_bm3d_noalloc(x, 0.05, out=out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0


def test_no_alloc_rejects_oversized_requests(cs):
    L = cs.lib()
    cap = L.cslsm_bm3d_noalloc_capacity()
    assert cap == 64 << 20
    assert L.cslsm_bm3d_scratch_bytes(1, 1024, 1024) <= cap < L.cslsm_bm3d_scratch_bytes(4, 1024, 1024)
    fake_in, fake_out = ctypes.c_void_p(0x1000), ctypes.c_void_p(0x10000000000)
    st = L.cslsm_denoise_bm3d_noalloc(fake_in, fake_out, 4, 1024, 1024, ctypes.c_float(0.05), None)
    assert st == 1 and b"scratch" in L.cslsm_last_error()
