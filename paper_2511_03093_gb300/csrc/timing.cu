// Launch accounting and sampled per-kernel event timing.
//
// Every kernel launch of the library goes through a LaunchScope: it counts
// the launch and, while timing is enabled with period p, brackets every p-th
// launch of each kernel with two CUDA events recorded on the launching
// stream.  Benchmarks read the summed device time per kernel afterwards.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace cslsm {
namespace {

const char *const kNames[K_COUNT] = {"pack_masks", "forward",  "adjoint",      "xupdate_w",
                                     "tikhonov_iter", "tikhonov_prox", "tv_tile",
                                     "psnr_partials", "reduce_finish", "bm3d_prep",
                                     "bm3d_match", "bm3d_filter", "bm3d_finish",
                                     "batch_persistent", "unrolled", "tvz_sweep", "ssim3d", "wnnm_filter"};

struct Rec {
    int kernel;
    cudaEvent_t a, b;
};

std::atomic<unsigned long long> g_launches{0};
std::atomic<int> g_period{0};
std::mutex g_mu;
unsigned long long g_seen[K_COUNT] = {};
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event()
{
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

}  // namespace

LaunchScope::LaunchScope(int kernel, cudaStream_t s) : rec_(-1), s_(s)
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    const int period = g_period.load(std::memory_order_relaxed);
    if (period <= 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_seen[kernel]++ % (unsigned long long)period != 0) return;
    cudaEvent_t a = take_event(), b = take_event();
    if (!a || !b) return;
    if (cudaEventRecord(a, s) != cudaSuccess) return;
    g_recs.push_back(Rec{kernel, a, b});
    rec_ = (int)g_recs.size() - 1;
}

LaunchScope::~LaunchScope()
{
    if (rec_ < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEventRecord(g_recs[rec_].b, s_);
}

}  // namespace cslsm

using namespace cslsm;

extern "C" {

unsigned long long cslsm_launch_count(void) { return g_launches.load(); }

cslsm_status cslsm_timing_enable(int period)
{
    if (period < 0) {
        set_error("timing period must be >= 0");
        return CSLSM_ERR_INVALID_ARG;
    }
    g_period.store(period);
    return CSLSM_OK;
}

cslsm_status cslsm_timing_read(const char *kernel, long long *launches_timed, double *total_ms,
                               int reset)
{
    if (!kernel || !launches_timed || !total_ms) {
        set_error("kernel, launches_timed and total_ms must be non-NULL");
        return CSLSM_ERR_INVALID_ARG;
    }
    int k = -1;
    for (int i = 0; i < K_COUNT; ++i)
        if (!strcmp(kernel, kNames[i])) k = i;
    if (k < 0) {
        set_error("unknown kernel name '%s'", kernel);
        return CSLSM_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    long long n = 0;
    double ms = 0.0;
    for (const Rec &r : g_recs) {
        if (r.kernel != k) continue;
        float t = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e != cudaSuccess) {
            set_error("timing read: %s", cudaGetErrorString(e));
            return CSLSM_ERR_CUDA;
        }
        ms += t;
        ++n;
    }
    *launches_timed = n;
    *total_ms = ms;
    if (reset) {
        for (const Rec &r : g_recs) {
            g_pool.push_back(r.a);
            g_pool.push_back(r.b);
        }
        g_recs.clear();
        memset(g_seen, 0, sizeof(g_seen));
    }
    return CSLSM_OK;
}

}  // extern "C"
