// Storage types of the ADMM state (u, d) and of the w = v + d workspace.
// All arithmetic is FP32; values are converted on load and rounded to nearest
// on store.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace cslsm {

template <typename S>
__device__ __forceinline__ float ld(const S *p);
template <>
__device__ __forceinline__ float ld<float>(const float *p)
{
    return *p;
}
template <>
__device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    return __bfloat162float(*p);
}
template <>
__device__ __forceinline__ float ld<__half>(const __half *p)
{
    return __half2float(*p);
}

// Loads that bypass L1 (cached in L2 only): safe for data another SM wrote
// earlier in the same kernel (the persistent batched solver).
template <typename S>
__device__ __forceinline__ float ld_l2(const S *p);
template <>
__device__ __forceinline__ float ld_l2<float>(const float *p)
{
    return __ldcg(p);
}
template <>
__device__ __forceinline__ float ld_l2<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    return __bfloat162float(__ldcg(p));
}
template <>
__device__ __forceinline__ float ld_l2<__half>(const __half *p)
{
    return __half2float(__ldcg(p));
}

template <typename S>
__device__ __forceinline__ void st(S *p, float v);
template <>
__device__ __forceinline__ void st<float>(float *p, float v)
{
    *p = v;
}
template <>
__device__ __forceinline__ void st<__nv_bfloat16>(__nv_bfloat16 *p, float v)
{
    *p = __float2bfloat16_rn(v);
}
template <>
__device__ __forceinline__ void st<__half>(__half *p, float v)
{
    *p = __float2half_rn(v);
}

// The value a store of v into S followed by a load gives back.
template <typename S>
__device__ __forceinline__ float rnd(float v)
{
    S t;
    st<S>(&t, v);
    return ld<S>(&t);
}

}  // namespace cslsm
