// Device helpers of libmgfp: storage-type traits, 16-byte vector loads and
// stores with round-to-nearest-even conversion, and exact FP64 construction
// from FP16/FP32 values with integer and FP32 instructions only.
//
// On GB300 the FP64 pipe issues ~1.6 instructions per clock per SM (also for
// F2F/I2F conversions to and from FP64), against ~22 bytes per clock per SM
// of HBM bandwidth.  The mixed-precision kernels therefore keep FP64 as a
// storage format: they build FP64 bit patterns with integer instructions and
// spend FP64 instructions only on the fused multiply-adds of Alg. 2's solution and residual updates.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mg_internal.h"

namespace mgi {

constexpr unsigned kFull = 0xffffffffu;

template <class T> struct Tr;
template <> struct Tr<double> { static constexpr int V = 2; using C = double; };
template <> struct Tr<float> { static constexpr int V = 4; using C = float; };
template <> struct Tr<__half> { static constexpr int V = 8; using C = float; };
template <> struct Tr<__nv_bfloat16> { static constexpr int V = 8; using C = float; };

// Host-computed coefficient i of a SweepCoef in the arithmetic type C.
template <class C> __device__ __forceinline__ C coef(const SweepCoef& c, int i);
template <> __device__ __forceinline__ float coef<float>(const SweepCoef& c, int i) { return c.f[i]; }
template <> __device__ __forceinline__ double coef<double>(const SweepCoef& c, int i) { return c.d[i]; }

// ---------------------------------------------------------------- 16-byte vector loads (RO path)
__device__ __forceinline__ void ldv(const double* p, double (&v)[2]) {
    double2 t = __ldg(reinterpret_cast<const double2*>(p));
    v[0] = t.x; v[1] = t.y;
}
__device__ __forceinline__ void ldv(const float* p, float (&v)[4]) {
    float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ldv(const __half* p, float (&v)[8]) {
    uint4 t = __ldg(reinterpret_cast<const uint4*>(p));
    unsigned w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        __half2 h = *reinterpret_cast<__half2*>(&w[k]);
        float2 f = __half22float2(h);
        v[2 * k] = f.x; v[2 * k + 1] = f.y;
    }
}
__device__ __forceinline__ void ldv(const __nv_bfloat16* p, float (&v)[8]) {
    uint4 t = __ldg(reinterpret_cast<const uint4*>(p));
    unsigned w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&w[k]);
        float2 f = __bfloat1622float2(h);
        v[2 * k] = f.x; v[2 * k + 1] = f.y;
    }
}

// ---------------------------------------------------------------- 16-byte vector stores (RN rounding)
__device__ __forceinline__ void stv(double* p, const double (&v)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
}
__device__ __forceinline__ void stv(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void stv(__half* p, const float (&v)[8]) {
    unsigned w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        __half2 h = __floats2half2_rn(v[2 * k], v[2 * k + 1]);
        w[k] = *reinterpret_cast<unsigned*>(&h);
    }
    *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
}
__device__ __forceinline__ void stv(__nv_bfloat16* p, const float (&v)[8]) {
    unsigned w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
        w[k] = *reinterpret_cast<unsigned*>(&h);
    }
    *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
}

// ---------------------------------------------------------------- scalar loads / stores
__device__ __forceinline__ double ld1(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ld1(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ld1(const __half* p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ float ld1(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }

__device__ __forceinline__ void st1(double* p, double v) { *p = v; }
__device__ __forceinline__ void st1(float* p, double v) { *p = (float)v; }
__device__ __forceinline__ void st1(float* p, float v) { *p = v; }
__device__ __forceinline__ void st1(__half* p, float v) { *p = __float2half_rn(v); }
__device__ __forceinline__ void st1(__half* p, double v) { *p = __float2half_rn((float)v); }
__device__ __forceinline__ void st1(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void st1(__nv_bfloat16* p, double v) { *p = __float2bfloat16_rn((float)v); }

// Round a value of the arithmetic type to the storage type and back.
__device__ __forceinline__ double rnd(double v, const double*) { return v; }
__device__ __forceinline__ float rnd(float v, const float*) { return v; }
__device__ __forceinline__ float rnd(float v, const __half*) { return __half2float(__float2half_rn(v)); }
__device__ __forceinline__ float rnd(float v, const __nv_bfloat16*) {
    return __bfloat162float(__float2bfloat16_rn(v));
}

// ---------------------------------------------------------------- bit-level FP64 helpers
// FP64 -> FP32 by truncation of the significand (round toward zero), with
// integer instructions only.  Values below the FP32 normal range give 0,
// overflow gives inf, NaN stays NaN.
__device__ __forceinline__ float f64_to_f32_trunc(double d) {
    unsigned long long b = (unsigned long long)__double_as_longlong(d);
    unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    unsigned sign = hi & 0x80000000u;
    int ein = (int)((hi >> 20) & 0x7FF);
    unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    if (ein == 0x7FF)  // inf stays inf, NaN becomes a quiet NaN
        return __uint_as_float(sign | ((b & 0x000FFFFFFFFFFFFFull) ? 0x7FC00000u : 0x7F800000u));
    int e = ein - 1023 + 127;
    if (e <= 0) return __uint_as_float(sign);
    if (e >= 255) return __uint_as_float(sign | 0x7F800000u);
    return __uint_as_float(sign | ((unsigned)e << 23) | m);
}

// Bit pattern -> FP64 through an opaque move: the integer construction below
// stays integer work (the compiler does not turn it back into a conversion
// instruction, which would run on the FP64 pipe).
__device__ __forceinline__ double bits_to_f64(unsigned long long b) {
    double d;
    asm("mov.b64 %0, %1;" : "=d"(d) : "l"(b));
    return d;
}

// Exact FP32 -> FP64 with integer instructions only (no F2F on the FP64
// pipe): zero, normal, subnormal (renormalised), inf and NaN.
__device__ __forceinline__ double f32_to_f64(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
    unsigned e = (b >> 23) & 0xFFu;
    unsigned m = b & 0x7FFFFFu;
    unsigned long long e64;
    if (e == 0xFFu) {
        e64 = 0x7FFull;
    } else if (e != 0u) {
        e64 = e + 896u;
    } else if (m == 0u) {
        e64 = 0ull;
    } else {  // subnormal: shift the leading one into the implicit position
        const int sh = __clz((int)m) - 8;  // m < 2^23: leading zeros within the 23-bit field, + 1
        m = (m << sh) & 0x7FFFFFu;
        e64 = (unsigned long long)(897 - sh);
    }
    return bits_to_f64(sign | (e64 << 52) | ((unsigned long long)m << 29));
}

// Exact FP64 of a float holding an FP16 value (an FP32 normal, zero, inf or
// NaN: FP16 subnormals are FP32 normals), with integer instructions only.
__device__ __forceinline__ double half_to_f64(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xFFu;
    const unsigned long long e64 = e == 0xFFu ? 0x7FFull : (e ? e + 896ull : 0ull);
    return bits_to_f64(((unsigned long long)(b & 0x80000000u) << 32) | (e64 << 52) |
                       ((unsigned long long)(b & 0x7FFFFFu) << 29));
}

// Exact s * 2^eoff as FP64 for |s| < 2^53 (result in the normal range), with
// integer instructions only.
__device__ __forceinline__ double i64_to_f64(long long s, int eoff = 0) {
    if (s == 0) return 0.0;
    unsigned long long a = s < 0 ? (unsigned long long)(-s) : (unsigned long long)s;
    int lz = __clzll((long long)a);
    int e = 63 - lz + eoff;
    unsigned long long m = (a << (lz - 11)) & 0x000FFFFFFFFFFFFFull;
    unsigned long long bits = ((unsigned long long)(1023 + e) << 52) | m |
                              (s < 0 ? 0x8000000000000000ull : 0ull);
    return bits_to_f64(bits);
}

// An FP16 value (held exactly in a float) is a multiple of 2^-24 with
// |v| <= 65504 < 2^16, so v * 2^24 is an integer below 2^40.  Split it as
// hi * 2^18 + lo with hi = round(v * 2^6) (|hi| <= 2^22) and lo the exact
// remainder (|lo| <= 2^17), both obtained with the FP32 round-to-integer
// "magic number" 1.5 * 2^23.  Sums of a few such parts fit in int32 exactly.
struct HSplit { int hi; float lo; };  // lo in units of 2^-24, integer-valued float
__device__ __forceinline__ HSplit h_split(float v) {
    const float MAGIC = 12582912.0f;  // 1.5 * 2^23
    float t = __fmaf_rn(v, 64.0f, MAGIC);
    HSplit s;
    s.hi = __float_as_int(t) - __float_as_int(MAGIC);
    float hf = __fsub_rn(t, MAGIC);
    float r = __fmaf_rn(hf, -0.015625f, v);  // v - hi/64, exact
    s.lo = __fmul_rn(r, 16777216.0f);         // exact integer, |.| <= 2^17
    return s;
}

// Error-free transformations in FP32 (Knuth TwoSum, FMA-based TwoProd).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
// max of two keys as an explicit compare and select (an integer compare pair),
// not a 64-bit max instruction
__device__ __forceinline__ unsigned long long key_max(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("{\n .reg .pred p;\n setp.gt.u64 p, %1, %2;\n selp.b64 %0, %1, %2, p;\n}\n" : "=l"(r) : "l"(b), "l"(a));
    return r;
}
__device__ __forceinline__ unsigned long long warp_max(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long t = __shfl_xor_sync(kFull, v, o);
        v = key_max(v, t);
    }
    return v;
}
// |d| as an order-preserving unsigned key (NaN keys exceed +inf).  The sign
// is cleared on the high word taken apart by an opaque move, so the compiler
// does not turn the mask into an FP64 absolute value (an FP64-pipe add).
__device__ __forceinline__ unsigned long long abs_key(double d) {
    unsigned lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "d"(d));
    return ((unsigned long long)(hi & 0x7FFFFFFFu) << 32) | lo;
}

}  // namespace mgi
