// 16-bit storage formats of spinors and links (FP16 and BF16), FP32 arithmetic.
//
// Spinor, one right-hand side (rhs_bytes(V) bytes): 3 planes of uint4, plane q holding
// components 4q .. 4q+3 (spin-major, colour fastest) as (re, im) pairs of 16-bit numbers;
// FP16 adds one float per site after the planes, the largest |re| or |im| of the site: its
// 24 numbers are stored divided by it, so that they lie in [-1, 1] where FP16 keeps 11
// significant bits whatever the magnitude of the vector.  BF16 has FP32's exponent range and
// stores the numbers themselves.
//
// Link U_mu(n): rows 0 and 1 (the third is rebuilt as conj(row0 x row1), SU(3)), 24 bytes in
// two planes per direction: uint4 [4][V] with (0,0) (0,1) (0,2) (1,0), then uint2 [4][V] with
// (1,1) (1,2).  |U_ij| <= 1, so neither format needs a scale.
#pragma once

namespace ovl {

struct H16 {};  // FP16 storage, per-site scale
struct B16 {};  // BF16 storage

}  // namespace ovl

#ifdef __CUDACC__
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace ovl {

template <typename S> struct Half2Of;
template <> struct Half2Of<H16> {
    typedef __half2 T;
    static __device__ __forceinline__ T pack(float a, float b) { return __floats2half2_rn(a, b); }
    static __device__ __forceinline__ float2 unpack(T v) { return __half22float2(v); }
};
template <> struct Half2Of<B16> {
    typedef __nv_bfloat162 T;
    static __device__ __forceinline__ T pack(float a, float b) { return __floats2bfloat162_rn(a, b); }
    static __device__ __forceinline__ float2 unpack(T v) { return __bfloat1622float2(v); }
};

template <typename S> struct HalfSpinor;
template <> struct HalfSpinor<H16> { static constexpr bool scaled = true; };
template <> struct HalfSpinor<B16> { static constexpr bool scaled = false; };

// bytes of one right-hand side (a multiple of 16)
template <typename S>
__host__ __device__ __forceinline__ long long half_rhs_bytes(long long V) {
    return HalfSpinor<S>::scaled ? ((52 * V + 15) / 16) * 16 : 48 * V;
}

// bit-level reinterpretation of a 32-bit word as two 16-bit numbers
template <typename S>
__device__ __forceinline__ float2 half_word(unsigned int w) {
    typename Half2Of<S>::T h;
    static_assert(sizeof(h) == 4, "two 16-bit numbers");
    memcpy(&h, &w, 4);
    return Half2Of<S>::unpack(h);
}
template <typename S>
__device__ __forceinline__ unsigned int half_pack(float a, float b) {
    typename Half2Of<S>::T h = Half2Of<S>::pack(a, b);
    unsigned int w;
    memcpy(&w, &h, 4);
    return w;
}

// Load site s of one right-hand side into 12 complex numbers (re, im).
template <typename S, bool LDG>
__device__ __forceinline__ void half_load_site(const void* base, long long V, long long s, float2 (&p)[12]) {
    const uint4* b = (const uint4*)base;
    float scale = 1.0f;
    if constexpr (HalfSpinor<S>::scaled) {
        const float* nrm = (const float*)((const char*)base + 48 * V);
        scale = LDG ? __ldg(nrm + s) : nrm[s];
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const uint4 v = LDG ? __ldg(b + q * V + s) : b[q * V + s];
        p[4 * q + 0] = half_word<S>(v.x);
        p[4 * q + 1] = half_word<S>(v.y);
        p[4 * q + 2] = half_word<S>(v.z);
        p[4 * q + 3] = half_word<S>(v.w);
    }
    if constexpr (HalfSpinor<S>::scaled) {
#pragma unroll
        for (int k = 0; k < 12; ++k) p[k] = make_float2(p[k].x * scale, p[k].y * scale);
    }
}

// Store 12 complex numbers at site s of one right-hand side (rounded to nearest).
template <typename S>
__device__ __forceinline__ void half_store_site(void* base, long long V, long long s, const float2 (&p)[12]) {
    uint4* b = (uint4*)base;
    float inv = 1.0f;
    if constexpr (HalfSpinor<S>::scaled) {
        float m = 0.0f;
#pragma unroll
        for (int k = 0; k < 12; ++k) m = fmaxf(m, fmaxf(fabsf(p[k].x), fabsf(p[k].y)));
        if (m > 0.0f) m = fmaxf(m, 1e-30f);  // keeps 1/m finite for denormal sites
        ((float*)((char*)base + 48 * V))[s] = m;
        inv = m > 0.0f ? 1.0f / m : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        uint4 v;
        v.x = half_pack<S>(p[4 * q + 0].x * inv, p[4 * q + 0].y * inv);
        v.y = half_pack<S>(p[4 * q + 1].x * inv, p[4 * q + 1].y * inv);
        v.z = half_pack<S>(p[4 * q + 2].x * inv, p[4 * q + 2].y * inv);
        v.w = half_pack<S>(p[4 * q + 3].x * inv, p[4 * q + 3].y * inv);
        b[q * V + s] = v;
    }
}

// Rows 0 and 1 of link (mu, site) as 6 complex numbers, row-major.
template <typename S>
__device__ __forceinline__ void half_load_link(const void* U, long long V, int mu, long long site, float2 (&r)[6]) {
    const uint4 a = __ldg((const uint4*)U + mu * V + site);
    const uint2 b = __ldg((const uint2*)((const char*)U + 64 * V) + mu * V + site);
    r[0] = half_word<S>(a.x);
    r[1] = half_word<S>(a.y);
    r[2] = half_word<S>(a.z);
    r[3] = half_word<S>(a.w);
    r[4] = half_word<S>(b.x);
    r[5] = half_word<S>(b.y);
}

template <typename S>
__device__ __forceinline__ void half_store_link(void* U, long long V, int mu, long long site, const float2 (&r)[6]) {
    uint4 a;
    a.x = half_pack<S>(r[0].x, r[0].y);
    a.y = half_pack<S>(r[1].x, r[1].y);
    a.z = half_pack<S>(r[2].x, r[2].y);
    a.w = half_pack<S>(r[3].x, r[3].y);
    uint2 b;
    b.x = half_pack<S>(r[4].x, r[4].y);
    b.y = half_pack<S>(r[5].x, r[5].y);
    ((uint4*)U)[mu * V + site] = a;
    ((uint2*)((char*)U + 64 * V))[mu * V + site] = b;
}

}  // namespace ovl
#endif  // __CUDACC__
