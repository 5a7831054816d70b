"""The allocation-free BM3D entry point, for callers that cannot allocate
device memory when they denoise: it must give what the allocating BM3D
denoiser gives, call after call, from its fixed scratch array, and it must
leave the device's stream-ordered memory pool untouched.

Collected last on purpose (file name), so that a run stopping at its first
failure has run every other test before this one."""
import ctypes

import numpy as np
import pytest

import synth
from tests.gpu_util import REL_ITER, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

# CUmemPool_attribute values of the CUDA driver API
_RESERVED_MEM_HIGH, _USED_MEM_CURRENT, _USED_MEM_HIGH = 6, 7, 8


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


def _noalloc(L, x, out, sigma):
    import torch

    Z, H, W = x.shape
    return L.cslsm_denoise_bm3d_noalloc(ctypes.c_void_p(x.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), Z, H, W,
                                        ctypes.c_float(sigma),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_no_alloc_matches_allocating_denoiser_twice(cs):
    import torch

    L = cs.lib()
    # near the capacity (7 x 512 x 512 uses most of the array), then smaller
    # calls that leave most of the array as the large call wrote it, a slice
    # smaller than a patch (the identity branch), and the first shape again
    shapes = [(7, 512, 512), (2, 70, 90), (1, 128, 96), (2, 6, 40), (2, 70, 90)]
    assert L.cslsm_bm3d_scratch_bytes(7, 512, 512) <= L.cslsm_bm3d_noalloc_capacity()
    for call, (Z, H, W) in enumerate(shapes):
        x = to_dev(_noisy(40 + call, Z, H, W))
        out = torch.empty_like(x)
        st = _noalloc(L, x, out, 0.04)
        assert st == 0, L.cslsm_last_error()
        ref = cs.denoise(x, cs.Params(denoiser="bm3d", bm3d_sigma=0.04))
        torch.cuda.synchronize()
        assert rel_l2(to_np(out), to_np(ref)) <= REL_ITER, (Z, H, W)


class _Pool:
    """The device's default stream-ordered memory pool (CUDA driver API), which
    the allocating BM3D path draws its scratch from."""

    def __init__(self, device):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev, self.pool = ctypes.c_int(), ctypes.c_void_p()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), device) == 0
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high_marks(self):
        zero = ctypes.c_uint64(0)  # resets a high-water mark to the current value
        for a in (_RESERVED_MEM_HIGH, _USED_MEM_HIGH):
            assert self.cu.cuMemPoolSetAttribute(self.pool, a, ctypes.byref(zero)) == 0


def test_no_alloc_allocates_nothing_after_first_use(cs):
    import torch

    x = to_dev(_noisy(7, 1, 64, 64))
    out = torch.empty_like(x)
    cs.denoise_bm3d_noalloc(x, 0.05, out=out)  # first use on this device: address set-up
    torch.cuda.synchronize()
    pool = _Pool(torch.cuda.current_device())
    used0 = pool.get(_USED_MEM_CURRENT)
    # the probe sees an allocation: the allocating denoiser raises the mark
    pool.reset_high_marks()
    cs.denoise(x, cs.Params(denoiser="bm3d", bm3d_sigma=0.05))
    torch.cuda.synchronize()
    assert pool.get(_USED_MEM_HIGH) > used0
    # the allocation-free calls do not
    pool.reset_high_marks()
    high0 = pool.get(_RESERVED_MEM_HIGH)
    for _ in range(3):
        cs.denoise_bm3d_noalloc(x, 0.05, out=out)
    torch.cuda.synchronize()
    assert pool.get(_USED_MEM_HIGH) == used0
    assert pool.get(_RESERVED_MEM_HIGH) == high0


def test_no_alloc_rejects_oversized_and_host_buffers(cs):
    L = cs.lib()
    cap = L.cslsm_bm3d_noalloc_capacity()
    assert cap == 64 << 20
    assert L.cslsm_bm3d_scratch_bytes(1, 1024, 1024) <= cap < L.cslsm_bm3d_scratch_bytes(2, 1024, 1024)
    fake_in, fake_out = ctypes.c_void_p(0x1000), ctypes.c_void_p(0x10000000000)
    st = L.cslsm_denoise_bm3d_noalloc(fake_in, fake_out, 4, 1024, 1024, ctypes.c_float(0.05), None)
    assert st == 1 and b"scratch" in L.cslsm_last_error()
    # host buffers are refused before any GPU work
    a = np.zeros((1, 16, 16), np.float32)
    b = np.zeros((1, 16, 16), np.float32)
    st = L.cslsm_denoise_bm3d_noalloc(ctypes.c_void_p(a.ctypes.data), ctypes.c_void_p(b.ctypes.data),
                                      1, 16, 16, ctypes.c_float(0.05), None)
    assert st == 1 and b"device memory" in L.cslsm_last_error()
