// Batched reconstruction: many independent measurements of uneven size and
// slice count solved by Algorithm 1 (TV prior, optional z smoothness) in ONE
// persistent kernel launch, captured once in a CUDA graph and replayed.
//
// Work decomposition.  For every item (measurement) an iteration is a chain of
// phases: the x-update (Eq. v-update, units of 1024 pixel columns), then the
// TV u-step (units = tiles of one slice; with gamma > 0 one phase per slice
// in Gauss-Seidel order, otherwise one phase holding every slice's tiles).
// Units of a phase are independent; a phase may start when every unit of the
// item's previous phase is done.  All units of all items and iterations are
// numbered in one global order: iteration-major, then phase level, then item
// - so every unit a unit waits for has a smaller number.
//
// Scheduling.  The grid is exactly as many CTAs as fit on the GPU at once.
// Each CTA takes the next unit number from a global ticket counter, waits
// until the item's completed-unit counter reaches the count the unit depends
// on, runs the unit and increments the counter.  Because units are taken in
// global order and every CTA is resident, the units waited for are already
// held by running CTAs: the schedule cannot deadlock.  Every wait is bounded
// (a wall-clock limit read from %globaltimer); on expiry the CTA raises the
// batch's error word, every CTA stops taking units, and the host reports
// CSLSM_ERR_TIMEOUT.  Data produced inside the launch is read with L2-only
// loads (__ldcg) after an acquire fence, never from a possibly stale L1.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <vector>

#include "internal.cuh"
#include "storage.cuh"
#include "tv_body.cuh"

namespace cslsm {
namespace {

constexpr int kBC = 2, kBB = 16;       // TV kernel variant used by the batch
constexpr int kBNT = kBC * kBB * 32;  // 1024 threads per CTA

struct BItem {
    void *u, *d, *w;
    const float *b;
    float *v_out;
    const uint32_t *words;
    int wstride;
    int H, W, N, R, Z;
    int TH, TW, RH, tiles_x, tiles;
    int units_x;
    long long units_iter;
};

struct BDesc {
    const BItem *items;
    int n, iters, levels;
    const long long *level_cum;  // [levels + 1] units before each level within an iteration
    const int *lvl_start;        // [levels + 1] first entry of each level
    const int *ent_item;         // entries: item of the entry
    const long long *ent_cum;    // entries: first unit of the entry within its level
    long long units_iter, total;
    unsigned long long *ticket;
    unsigned long long *done;  // [n]
    int *error;
    long long timeout_ns;
    int stall_test;
    float rho, lam, gam, tau;
    int T;
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Units of item it before phase p of an iteration.
__device__ __forceinline__ long long phase_prefix(const BItem &it, int p, bool zsweep)
{
    if (p == 0) return 0;
    return it.units_x + (zsweep ? (long long)(p - 1) * it.tiles : 0);
}

template <typename S>
__device__ void xupdate_unit(const BItem &it, int unit, float rho, bool last)
{
    const int HW = it.H * it.W;
    const int pix = unit * kBNT + threadIdx.x;
    if (pix >= HW) return;
    const S *u = (const S *)it.u, *d = (const S *)it.d;
    S *w = (S *)it.w;
    for (int j = 0; j < it.N; ++j) {
        const uint32_t word = __ldcg(it.words + (size_t)j * it.wstride + pix);
        const size_t base = (size_t)j * it.R * HW + pix;
        float s = 0.f;
        for (int r = 0; r < it.R; ++r) {
            if ((word >> r) & 1u) {
                const size_t o = base + (size_t)r * HW;
                s += ld_l2<S>(u + o) - ld_l2<S>(d + o);
            }
        }
        const float e = (__ldcg(it.b + (size_t)j * HW + pix) - s) / (rho + (float)__popc(word));
        for (int r = 0; r < it.R; ++r) {
            const size_t o = base + (size_t)r * HW;
            const float dr = ld_l2<S>(d + o);
            const float g = ld_l2<S>(u + o) - dr;
            const float v = ((word >> r) & 1u) ? g + e : g;
            st<S>(w + o, v + dr);
            if (last) it.v_out[o] = v;
        }
    }
}

template <typename S>
__global__ void __launch_bounds__(kBNT, 1) batch_persistent_kernel(const BDesc *__restrict__ dp)
{
    extern __shared__ float smem[];
    __shared__ long long s_t;
    __shared__ int s_abort;
    const BDesc D = *dp;
    const bool zsweep = D.gam > 0.f;
    for (;;) {
        if (threadIdx.x == 0) {
            s_abort = *(volatile int *)D.error;
            s_t = s_abort ? D.total : (long long)atomicAdd(D.ticket, 1ull);
        }
        __syncthreads();
        const long long t = s_t;
        if (t >= D.total) break;
        // decode the unit number
        const int k = (int)(t / D.units_iter);
        long long r = t - (long long)k * D.units_iter;
        int lo = 0, hi = D.levels - 1;
        while (lo < hi) {  // last level with level_cum <= r
            const int mid = (lo + hi + 1) / 2;
            if (D.level_cum[mid] <= r) lo = mid;
            else hi = mid - 1;
        }
        const int p = lo;
        r -= D.level_cum[p];
        int e0 = D.lvl_start[p], e1 = D.lvl_start[p + 1] - 1;
        while (e0 < e1) {
            const int mid = (e0 + e1 + 1) / 2;
            if (D.ent_cum[mid] <= r) e0 = mid;
            else e1 = mid - 1;
        }
        const int i = D.ent_item[e0];
        const int unit = (int)(r - D.ent_cum[e0]);
        const BItem &it = D.items[i];
        // wait for the item's previous phase (and iteration)
        if (threadIdx.x == 0) {
            const unsigned long long need =
                D.stall_test ? ~0ull
                             : (unsigned long long)((long long)k * it.units_iter +
                                                    phase_prefix(it, p, zsweep));
            const unsigned long long t0 = global_ns();
            while (*(volatile unsigned long long *)(D.done + i) < need) {
                if (*(volatile int *)D.error) {
                    s_abort = 1;
                    break;
                }
                if ((long long)(global_ns() - t0) > D.timeout_ns) {
                    atomicExch(D.error, 1);
                    s_abort = 1;
                    break;
                }
                __nanosleep(256);
            }
            __threadfence();
        }
        __syncthreads();
        if (s_abort) break;
        if (p == 0) {
            xupdate_unit<S>(it, unit, D.rho, k == D.iters - 1);
        } else {
            TvLaunch a{};
            a.w = it.w;
            a.u = it.u;
            a.d = it.d;
            a.H = it.H;
            a.W = it.W;
            a.Z = it.Z;
            a.T = D.lam > 0.f ? D.T : 0;
            a.TH = it.TH;
            a.TW = it.TW;
            a.RH = it.RH;
            a.rho = D.rho;
            a.gamma = it.Z > 1 ? D.gam : 0.f;
            a.inv_rho2g = 1.f / (D.rho + 2.f * a.gamma);
            a.theta = D.lam / (D.rho + 2.f * a.gamma);
            a.inv_theta = a.theta > 0.f ? 1.f / a.theta : 0.f;
            a.tau = D.tau;
            a.write_final = 1;
            a.n0 = 0;
            a.nslices = 1;
            int n, tile;
            if (zsweep) {
                n = p - 1;
                tile = unit;
            } else {
                n = unit / it.tiles;
                tile = unit - n * it.tiles;
            }
            tv_tile_body<kBC, kBB, S>(a, tile % it.tiles_x, tile / it.tiles_x, n, smem);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(D.done + i, 1ull);
        }
    }
}

template <typename S>
cslsm_status launch_persistent(const BDesc *dp, int grid, size_t smem, cudaStream_t s)
{
    LaunchScope ls(K_BATCH, s);
    batch_persistent_kernel<S><<<grid, kBNT, smem, s>>>(dp);
    CSLSM_LAUNCHED();
    return CSLSM_OK;
}

template <typename S>
cslsm_status occupancy(size_t smem, int &per_sm)
{
    CSLSM_CUDA(cudaFuncSetAttribute(batch_persistent_kernel<S>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    CSLSM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_persistent_kernel<S>,
                                                             kBNT, smem));
    return CSLSM_OK;
}

}  // namespace

int batch_max_tile_rows(int T)
{
    // the largest region that fits: 5 arrays of 64 C x RH floats in 227 KB
    const int rh = (int)((227 * 1024 / sizeof(float) / 5 - 4) / (64 * kBC));
    return std::max(0, rh - 2 * T - 2);
}

cslsm_status batch_build(const BatchSpec &spec, BatchRun &run)
{
    const int n = (int)spec.items.size();
    const bool zs = spec.gamma > 0.f;
    std::vector<BItem> items(n);
    int levels = 1, max_rh = 0;
    for (int i = 0; i < n; ++i) {
        const BatchItemSpec &s = spec.items[i];
        BItem &b = items[i];
        b.u = s.u;
        b.d = s.d;
        b.w = s.w;
        b.b = s.b;
        b.v_out = s.v_out;
        b.words = s.words;
        b.wstride = s.wstride;
        b.H = s.H;
        b.W = s.W;
        b.N = s.N;
        b.R = s.R;
        b.Z = s.N * s.R;
        const int T = spec.lam > 0.f ? spec.T : 0;
        b.TH = s.TH;
        b.RH = s.TH + 2 * T + 2;
        b.TW = 62 * kBC + 2 - 2 * T - 2;
        b.tiles_x = (s.W + b.TW - 1) / b.TW;
        b.tiles = b.tiles_x * ((s.H + b.TH - 1) / b.TH);
        b.units_x = (s.H * s.W + kBNT - 1) / kBNT;
        b.units_iter = b.units_x + (long long)b.tiles * b.Z;
        levels = std::max(levels, zs ? 1 + b.Z : 2);
        max_rh = std::max(max_rh, b.RH);
    }
    // level tables: per level p, the items having phase p and their unit counts
    std::vector<long long> level_cum(levels + 1, 0);
    std::vector<int> lvl_start(levels + 1, 0), ent_item;
    std::vector<long long> ent_cum;
    for (int p = 0; p < levels; ++p) {
        lvl_start[p] = (int)ent_item.size();
        long long acc = 0;
        for (int i = 0; i < n; ++i) {
            const BItem &b = items[i];
            long long c = 0;
            if (p == 0) c = b.units_x;
            else if (zs) c = (p - 1 < b.Z) ? b.tiles : 0;
            else c = (p == 1) ? (long long)b.tiles * b.Z : 0;
            if (c == 0) continue;
            ent_item.push_back(i);
            ent_cum.push_back(acc);
            acc += c;
        }
        level_cum[p + 1] = level_cum[p] + acc;
    }
    lvl_start[levels] = (int)ent_item.size();
    const long long units_iter = level_cum[levels];
    // one device allocation for descriptors, tables and counters
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t sz_items = al(sizeof(BItem) * n), sz_lc = al(sizeof(long long) * (levels + 1)),
                 sz_ls = al(sizeof(int) * (levels + 1)), sz_ei = al(sizeof(int) * ent_item.size()),
                 sz_ec = al(sizeof(long long) * ent_cum.size()), sz_cnt = al(8 * (n + 1)),
                 sz_err = 256, sz_desc = al(sizeof(BDesc));
    const size_t total = sz_items + sz_lc + sz_ls + sz_ei + sz_ec + sz_cnt + sz_err + sz_desc;
    char *base = nullptr;
    CSLSM_CUDA(cudaMalloc(&base, total));
    run.mem = base;
    char *q = base;
    BItem *d_items = (BItem *)q;
    q += sz_items;
    long long *d_lc = (long long *)q;
    q += sz_lc;
    int *d_ls = (int *)q;
    q += sz_ls;
    int *d_ei = (int *)q;
    q += sz_ei;
    long long *d_ec = (long long *)q;
    q += sz_ec;
    unsigned long long *d_cnt = (unsigned long long *)q;  // [0] ticket, [1..n] done
    q += sz_cnt;
    int *d_err = (int *)q;
    q += sz_err;
    BDesc *d_desc = (BDesc *)q;
    BDesc D{};
    D.items = d_items;
    D.n = n;
    D.iters = spec.iters;
    D.levels = levels;
    D.level_cum = d_lc;
    D.lvl_start = d_ls;
    D.ent_item = d_ei;
    D.ent_cum = d_ec;
    D.units_iter = units_iter;
    D.total = units_iter * spec.iters;
    D.ticket = d_cnt;
    D.done = d_cnt + 1;
    D.error = d_err;
    D.timeout_ns = (long long)(spec.wait_limit_s * 1e9);
    D.stall_test = spec.stall_test;
    D.rho = spec.rho;
    D.lam = spec.lam;
    D.gam = spec.gamma;
    D.tau = spec.tau;
    D.T = spec.T;
    CSLSM_CUDA(cudaMemcpy(d_items, items.data(), sizeof(BItem) * n, cudaMemcpyHostToDevice));
    CSLSM_CUDA(cudaMemcpy(d_lc, level_cum.data(), sizeof(long long) * (levels + 1),
                          cudaMemcpyHostToDevice));
    CSLSM_CUDA(cudaMemcpy(d_ls, lvl_start.data(), sizeof(int) * (levels + 1),
                          cudaMemcpyHostToDevice));
    CSLSM_CUDA(cudaMemcpy(d_ei, ent_item.data(), sizeof(int) * ent_item.size(),
                          cudaMemcpyHostToDevice));
    CSLSM_CUDA(cudaMemcpy(d_ec, ent_cum.data(), sizeof(long long) * ent_cum.size(),
                          cudaMemcpyHostToDevice));
    CSLSM_CUDA(cudaMemcpy(d_desc, &D, sizeof(BDesc), cudaMemcpyHostToDevice));
    run.desc = d_desc;
    run.counters = d_cnt;
    run.counters_bytes = 8 * (n + 1);
    run.error = d_err;
    run.smem = tv_smem_bytes(kBC, max_rh);
    if (run.smem > 227 * 1024) {
        set_error("batched TV tile needs %zu bytes of shared memory", run.smem);
        return CSLSM_ERR_UNSUPPORTED;
    }
    int per_sm = 0, dev = 0, sms = 0;
    cslsm_status e;
    if (spec.storage == CSLSM_STORE_BF16) e = occupancy<__nv_bfloat16>(run.smem, per_sm);
    else if (spec.storage == CSLSM_STORE_FP16) e = occupancy<__half>(run.smem, per_sm);
    else e = occupancy<float>(run.smem, per_sm);
    if (e) return e;
    CSLSM_CUDA(cudaGetDevice(&dev));
    CSLSM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (per_sm < 1) {
        set_error("persistent batch kernel does not fit on an SM");
        return CSLSM_ERR_UNSUPPORTED;
    }
    run.grid = per_sm * sms;
    run.storage = spec.storage;
    return CSLSM_OK;
}

cslsm_status batch_set_wait(const BatchRun &run, double limit_s, int stall_test)
{
    BDesc D{};
    CSLSM_CUDA(cudaMemcpy(&D, run.desc, sizeof(BDesc), cudaMemcpyDeviceToHost));
    D.timeout_ns = (long long)(limit_s * 1e9);
    D.stall_test = stall_test;
    CSLSM_CUDA(cudaMemcpy(run.desc, &D, sizeof(BDesc), cudaMemcpyHostToDevice));
    return CSLSM_OK;
}

cslsm_status batch_enqueue(const BatchRun &run, cudaStream_t s)
{
    CSLSM_CUDA(cudaMemsetAsync(run.counters, 0, run.counters_bytes, s));
    CSLSM_CUDA(cudaMemsetAsync(run.error, 0, sizeof(int), s));
    const BDesc *dp = (const BDesc *)run.desc;
    if (run.storage == CSLSM_STORE_BF16) return launch_persistent<__nv_bfloat16>(dp, run.grid, run.smem, s);
    if (run.storage == CSLSM_STORE_FP16) return launch_persistent<__half>(dp, run.grid, run.smem, s);
    return launch_persistent<float>(dp, run.grid, run.smem, s);
}

}  // namespace cslsm
