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

// Two consecutive elements, L2 only (8-byte aligned for float, 4-byte for
// 16-bit types).
template <typename S>
__device__ __forceinline__ float2 ld2_l2(const S *p);
template <>
__device__ __forceinline__ float2 ld2_l2<float>(const float *p)
{
    return __ldcg(reinterpret_cast<const float2 *>(p));
}
template <>
__device__ __forceinline__ float2 ld2_l2<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    const unsigned r = __ldcg(reinterpret_cast<const unsigned *>(p));
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&r));
}
template <>
__device__ __forceinline__ float2 ld2_l2<__half>(const __half *p)
{
    const unsigned r = __ldcg(reinterpret_cast<const unsigned *>(p));
    return __half22float2(*reinterpret_cast<const __half2 *>(&r));
}

// Four consecutive elements, L2 only (16-byte aligned for float, 8-byte for
// 16-bit types).
template <typename S>
__device__ __forceinline__ float4 ld4_l2(const S *p);
template <>
__device__ __forceinline__ float4 ld4_l2<float>(const float *p)
{
    return __ldcg(reinterpret_cast<const float4 *>(p));
}
template <>
__device__ __forceinline__ float4 ld4_l2<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    const uint2 r = __ldcg(reinterpret_cast<const uint2 *>(p));
    const float2 fa = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&r.x));
    const float2 fb = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&r.y));
    return make_float4(fa.x, fa.y, fb.x, fb.y);
}
template <>
__device__ __forceinline__ float4 ld4_l2<__half>(const __half *p)
{
    const uint2 r = __ldcg(reinterpret_cast<const uint2 *>(p));
    const float2 fa = __half22float2(*reinterpret_cast<const __half2 *>(&r.x));
    const float2 fb = __half22float2(*reinterpret_cast<const __half2 *>(&r.y));
    return make_float4(fa.x, fa.y, fb.x, fb.y);
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

// Two consecutive elements (8-byte aligned for float, 4-byte for 16-bit types).
template <typename S>
__device__ __forceinline__ float2 ld2(const S *p);
template <>
__device__ __forceinline__ float2 ld2<float>(const float *p)
{
    return *reinterpret_cast<const float2 *>(p);
}
template <>
__device__ __forceinline__ float2 ld2<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
}
template <>
__device__ __forceinline__ float2 ld2<__half>(const __half *p)
{
    return __half22float2(*reinterpret_cast<const __half2 *>(p));
}
template <typename S>
__device__ __forceinline__ void st2(S *p, float2 v);
template <>
__device__ __forceinline__ void st2<float>(float *p, float2 v)
{
    *reinterpret_cast<float2 *>(p) = v;
}
template <>
__device__ __forceinline__ void st2<__nv_bfloat16>(__nv_bfloat16 *p, float2 v)
{
    *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(v.x, v.y);
}
template <>
__device__ __forceinline__ void st2<__half>(__half *p, float2 v)
{
    *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(v.x, v.y);
}

// Four consecutive elements (16-byte aligned for float, 8-byte for 16-bit types).
template <typename S>
__device__ __forceinline__ float4 ld4(const S *p);
template <>
__device__ __forceinline__ float4 ld4<float>(const float *p)
{
    return *reinterpret_cast<const float4 *>(p);
}
template <>
__device__ __forceinline__ float4 ld4<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    const uint2 r = *reinterpret_cast<const uint2 *>(p);
    const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162 *>(&r.x);
    const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162 *>(&r.y);
    const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
}
template <>
__device__ __forceinline__ float4 ld4<__half>(const __half *p)
{
    const uint2 r = *reinterpret_cast<const uint2 *>(p);
    const __half2 a = *reinterpret_cast<const __half2 *>(&r.x);
    const __half2 b = *reinterpret_cast<const __half2 *>(&r.y);
    const float2 fa = __half22float2(a), fb = __half22float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
}

template <typename S>
__device__ __forceinline__ void st4(S *p, float4 v);
template <>
__device__ __forceinline__ void st4<float>(float *p, float4 v)
{
    *reinterpret_cast<float4 *>(p) = v;
}
template <>
__device__ __forceinline__ void st4<__nv_bfloat16>(__nv_bfloat16 *p, float4 v)
{
    const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
    uint2 r;
    r.x = *reinterpret_cast<const unsigned *>(&a);
    r.y = *reinterpret_cast<const unsigned *>(&b);
    *reinterpret_cast<uint2 *>(p) = r;
}
template <>
__device__ __forceinline__ void st4<__half>(__half *p, float4 v)
{
    const __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
    uint2 r;
    r.x = *reinterpret_cast<const unsigned *>(&a);
    r.y = *reinterpret_cast<const unsigned *>(&b);
    *reinterpret_cast<uint2 *>(p) = r;
}

// The value a store of v into S followed by a load gives back.
template <typename S>
__device__ __forceinline__ float rnd(float v)
{
    S t;
    st<S>(&t, v);
    return ld<S>(&t);
}

// The value a state store keeps.  FP32: v.  FP16: v rounded to nearest even.
// BF16: v rounded stochastically: the part of v below the BF16 ulp decides the
// direction with a threshold drawn from a hash of v's own bits, the voxel index
// and the field (u, d or w).  Round-to-nearest in BF16 loses the small late
// updates of a converging ADMM iteration (they fall below half an ulp and are
// rounded away, so the iterates stall early); stochastic rounding keeps them on
// average.  The threshold depends only on (value, index, field), so the same
// value at the same voxel is rounded the same way in every kernel and run.
constexpr unsigned kKeyU = 0x68e31da4u, kKeyD = 0xb5297a4du, kKeyW = 0x1b56c4e9u;

// 16-bit rounding threshold from (value bits, index, field): a multiply-add
// of the three and one multiply-xorshift round, the high bits taken.
__device__ __forceinline__ unsigned sr_threshold(unsigned b, size_t idx, unsigned field)
{
    unsigned h = (b ^ field) * 0x9e3779b1u + (unsigned)idx * 0x85ebca77u;
    h ^= h >> 15;
    h *= 0x2c1b3c6du;
    h ^= h >> 12;
    return h >> 16;
}

template <typename S>
__device__ __forceinline__ float keep(float v, size_t idx, unsigned field);
template <>
__device__ __forceinline__ float keep<float>(float v, size_t, unsigned)
{
    return v;
}
template <>
__device__ __forceinline__ float keep<__half>(float v, size_t, unsigned)
{
    return rnd<__half>(v);
}
template <>
__device__ __forceinline__ float keep<__nv_bfloat16>(float v, size_t idx, unsigned field)
{
    const unsigned b = __float_as_uint(v);
    if ((b & 0x7f800000u) == 0x7f800000u) return rnd<__nv_bfloat16>(v);  // inf, nan
    return __uint_as_float((b + sr_threshold(b, idx, field)) & 0xffff0000u);
}

}  // namespace cslsm
