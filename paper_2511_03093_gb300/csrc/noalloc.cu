// Allocation-free BM3D denoiser entry point.
//
// Some callers cannot allocate device memory at the moment they denoise: a
// host application that owns a fixed memory budget and forbids libraries from
// growing it, or a real-time loop where an allocation's latency or failure is
// not acceptable.  cslsm_denoise with BM3D takes its scratch (the basic
// estimate, the aggregation accumulators, the match lists) from
// cudaMallocAsync; this entry point takes it from a fixed array that is part
// of the library image instead.
//
// The array is a file-scope __device__ variable: every GPU on which the
// library is loaded holds its kScratchBytes until the process exits.  Host
// code must not use the array's name as a device address (on the host it only
// names a stand-in); its device address is obtained once per device with
// cudaGetSymbolAddress while that device is current.
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "internal.cuh"

namespace cslsm {
namespace {

constexpr size_t kScratchBytes = 64ull << 20;  // 64 MiB

static __device__ __align__(256) unsigned char g_bm3d_scratch[kScratchBytes];

std::mutex g_mu;
std::vector<void *> g_scratch_addr;  // per device, filled at first use

cslsm_status scratch_address(void **out)
{
    int dev = 0;
    CSLSM_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mu);
    if ((int)g_scratch_addr.size() <= dev) g_scratch_addr.resize(dev + 1, nullptr);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_bm3d_scratch);
        if (e != cudaSuccess || p == nullptr) {
            set_error("cudaGetSymbolAddress of the BM3D scratch array failed: %s",
                      cudaGetErrorString(e));
            return CSLSM_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return CSLSM_OK;
}

// The scratch address is per device, so in and out must be device (or
// managed) memory of the device that is current: a buffer of another GPU, or
// host memory, would otherwise reach this device's kernels.
cslsm_status check_device_buffer(const void *p, const char *name)
{
    int dev = 0;
    CSLSM_CUDA(cudaGetDevice(&dev));
    cudaPointerAttributes at{};
    const cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("%s: cudaPointerGetAttributes failed: %s", name, cudaGetErrorString(e));
        return CSLSM_ERR_INVALID_ARG;
    }
    const bool device_mem = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
    if (!device_mem || at.device != dev) {
        set_error("%s must be device memory of the current device %d (memory type %d, device %d)",
                  name, dev, (int)at.type, at.device);
        return CSLSM_ERR_INVALID_ARG;
    }
    return CSLSM_OK;
}

}  // namespace
}  // namespace cslsm

using namespace cslsm;

extern "C" {

size_t cslsm_bm3d_noalloc_capacity(void) { return kScratchBytes; }

size_t cslsm_bm3d_scratch_bytes(int Z, int H, int W)
{
    if (Z < 1 || H < 1 || W < 1) return 0;
    return bm3d_workspace_bytes(Z, H, W);
}

cslsm_status cslsm_denoise_bm3d_noalloc(const float *in, float *out, int Z, int H, int W,
                                        float sigma, void *stream)
{
    if (!in || !out) {
        set_error("in and out must be non-NULL");
        return CSLSM_ERR_INVALID_ARG;
    }
    if (Z < 1 || H < 1 || W < 1 || (long long)Z * H * W >= (1ll << 31)) {
        set_error("need Z, H, W >= 1 and Z*H*W < 2^31");
        return CSLSM_ERR_INVALID_ARG;
    }
    if (!(sigma > 0.f) || sigma != sigma || sigma > 3.0e38f) {
        set_error("sigma must be finite and > 0");
        return CSLSM_ERR_INVALID_ARG;
    }
    const size_t nv = (size_t)Z * H * W;
    const char *a = (const char *)in, *o = (const char *)out;
    if (!(o + nv * sizeof(float) <= a || a + nv * sizeof(float) <= o)) {
        set_error("in and out must not overlap");
        return CSLSM_ERR_INVALID_ARG;
    }
    const size_t need = bm3d_workspace_bytes(Z, H, W);
    if (need > kScratchBytes) {
        set_error("BM3D of %d x %d x %d needs %zu bytes of scratch; the fixed array holds %zu "
                  "(split the volume into fewer slices per call)",
                  Z, H, W, need, kScratchBytes);
        return CSLSM_ERR_INVALID_ARG;
    }
    cslsm_status st = check_device_buffer(in, "in");
    if (st) return st;
    if ((st = check_device_buffer(out, "out"))) return st;
    void *ws = nullptr;
    st = scratch_address(&ws);
    if (st) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the array keeps the previous call's contents: zero what must start at 0
    CSLSM_CUDA(cudaMemsetAsync(ws, 0, need, s));
    Bm3dSlices b{};
    b.storage = CSLSM_STORE_FP32;
    b.src = in;
    b.u = nullptr;
    b.out = out;
    b.dual = nullptr;
    b.Z = Z;
    b.H = H;
    b.W = W;
    b.n0 = 0;
    b.nslices = Z;
    b.rho = 1.f;
    b.gamma = 0.f;
    b.sigma = sigma;
    return bm3d_slices(b, ws, s);
}

}  // extern "C"
