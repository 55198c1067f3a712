// Stencil kernels of libmgfp.
//
// k_sweep3 / k_sweep2: every grid pass that applies the 5/7-point operator
// A_l (Sec. 5) to a stored level vector:
//   M_JACOBI    damped Jacobi sweep (Sec. 4.2; Alg. 1's pre- and post-smoothing)
//   M_ZERO2     the first two sweeps of a pre-smoothing from c = 0, fused
//               (Alg. 1's pre-smoothing with a zero initial guess)
//   M_ZERO1     one sweep from c = 0 (c = omega D^-1 g)
//   M_RESTRICT  residual g - A c and its full-weighting restriction to the next
//               coarser level with the precision change (Alg. 1's residual restriction)
// k_update: Alg. 2's solution and residual updates fused (the paper's UpdateResiduum_Correction),
//   u += alpha c and r -= alpha A c in FP64 with norm partials.
// k_scale_cast: Alg. 2's residual scaling, the scaled FP64 residual cast to the finest
//   level's storage type.
// k_prolong: Alg. 1's prolongation and correction.
//
// 3D sweep decomposition: a CTA of TY warps owns TY consecutive rows of one
// 32V-wide x-chunk (V = elements per 16-byte vector: 8 FP16/BF16, 4 FP32,
// 2 FP64; every row chunk is 512 bytes) and marches over a z-range.  Planes
// stream through a ring of S shared-memory stages filled by cp.async: each
// stage holds the TY rows of the chunk plus one halo row above and below and
// one halo element (pair) left and right of the chunk (zero-filled outside the
// grid) and, for passes that need it, the TY rows of g.  While plane z is
// computed from stages z-1, z, z+1, planes z+2 and z+3 are in flight, so
// memory latency is hidden with few registers per thread.  In 2D each warp
// owns one x-chunk and marches over rows with a per-warp ring.
// Arithmetic is FP32 for FP16/BF16/FP32 levels and FP64 for FP64 levels.
#pragma once
#include <type_traits>

#include "mg_device.cuh"
#include "mg_final.cuh"

namespace mgi {

template <int DIM>
__device__ __forceinline__ long long offs(int x, int y, int z, int P, long long S) {
    return DIM == 3 ? (long long)z * S + (long long)y * P + x : (long long)y * P + x;
}

// ---------------------------------------------------------------- cp.async
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool ok) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(ok ? 16 : 0));
}
template <int BYTES>
__device__ __forceinline__ void cp_async_small(void* smem, const void* gmem, bool ok) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(s), "l"(gmem), "n"(BYTES),
                 "r"(ok ? BYTES : 0));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Shared-memory row: one 512-byte chunk with a 16-byte pad on each side (room
// for the x-halo elements).
constexpr int kRowBytes = 512 + 32;

// x-halo copy: one element, or the aligned pair next to the edge for 2-byte
// types (cp.async copies at least 4 bytes).
template <class T> struct Halo {
    static constexpr int E = sizeof(T) == 2 ? 2 : 1;
    static constexpr int BYTES = sizeof(T) == 2 ? 4 : (int)sizeof(T);
};

// One row chunk into shared memory: 16 bytes per lane, halos by lanes 0 / 31;
// zero-filled when the row is outside the grid or past the pitch.
template <class T>
__device__ __forceinline__ void issue_row(unsigned char* srow, const T* grow, int lane, int x0, int P, bool row_ok) {
    constexpr int V = Tr<T>::V;
    constexpr int CW = 32 * V;
    const int x = x0 + lane * V;
    T* d = reinterpret_cast<T*>(srow + 16);
    const bool ok = row_ok && x < P;
    cp_async16(d + lane * V, ok ? (const void*)(grow + x) : (const void*)grow, ok);
    if (lane == 0)
        cp_async_small<Halo<T>::BYTES>(d - Halo<T>::E, row_ok ? (const void*)(grow + x0 - Halo<T>::E) : (const void*)grow,
                                       row_ok);
    if (lane == 31) {
        const bool okr = row_ok && x0 + CW < P;
        cp_async_small<Halo<T>::BYTES>(d + CW, okr ? (const void*)(grow + x0 + CW) : (const void*)grow, okr);
    }
}

// The lane's V values of a shared-memory row, in the arithmetic type.
template <class T>
__device__ __forceinline__ void lds_vec(const unsigned char* srow, int lane, typename Tr<T>::C (&v)[Tr<T>::V]) {
    const T* d = reinterpret_cast<const T*>(srow + 16) + lane * Tr<T>::V;
    const uint4 raw = *reinterpret_cast<const uint4*>(d);
    if constexpr (sizeof(T) == 8) {
        v[0] = __longlong_as_double(((long long)raw.y << 32) | raw.x);
        v[1] = __longlong_as_double(((long long)raw.w << 32) | raw.z);
    } else if constexpr (sizeof(T) == 4) {
        v[0] = __uint_as_float(raw.x); v[1] = __uint_as_float(raw.y);
        v[2] = __uint_as_float(raw.z); v[3] = __uint_as_float(raw.w);
    } else {
        const unsigned wd[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float2 f;
            if constexpr (std::is_same<T, __half>::value) f = __half22float2(*reinterpret_cast<const __half2*>(&wd[k]));
            else f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&wd[k]));
            v[2 * k] = f.x; v[2 * k + 1] = f.y;
        }
    }
}
template <class T>
__device__ __forceinline__ typename Tr<T>::C lds_one(const unsigned char* srow, int idx) {
    const T* d = reinterpret_cast<const T*>(srow + 16);
    if constexpr (sizeof(T) == 8 || sizeof(T) == 4) return d[idx];
    else if constexpr (std::is_same<T, __half>::value) return __half2float(d[idx]);
    else return __bfloat162float(d[idx]);
}

// ---------------------------------------------------------------- per-point values
template <int MODE, class C>
__device__ __forceinline__ C point_value(C c0, C nb, C g, C c1, C c2, C c3, C h2inv, C twod, C k2) {
    if (MODE == M_JACOBI) return c1 * c0 + c2 * nb + c3 * g;            // c + w D^-1 (g - A c)
    if (MODE == M_ZERO2) return c3 * (k2 * c0 + c2 * nb);                 // two sweeps from 0, c0 = g
    if (MODE == M_ZERO1) return c3 * c0;                                   // one sweep from 0
    return g - h2inv * (twod * c0 - nb);                                   // residual g - A c
}

// ---------------------------------------------------------------- pair arithmetic
// Values of a row chunk are handled in pairs: FP32 pairs use the packed
// FP32x2 instructions of sm_100+ (one instruction for two lanes of the pair,
// each rounded as the scalar operation), FP64 pairs two scalar operations.
template <class C> struct Pair;
template <> struct Pair<float> {
    using t = float2;
    static __device__ __forceinline__ t mk(float a, float b) { return make_float2(a, b); }
    static __device__ __forceinline__ t splat(float a) { return make_float2(a, a); }
    static __device__ __forceinline__ t add(t a, t b) { return __fadd2_rn(a, b); }
    static __device__ __forceinline__ t mul(t a, t b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ t fma(t a, t b, t c) { return __ffma2_rn(a, b, c); }
};
template <> struct Pair<double> {
    using t = double2;
    static __device__ __forceinline__ t mk(double a, double b) { return make_double2(a, b); }
    static __device__ __forceinline__ t splat(double a) { return make_double2(a, a); }
    static __device__ __forceinline__ t add(t a, t b) { return make_double2(a.x + b.x, a.y + b.y); }
    static __device__ __forceinline__ t mul(t a, t b) { return make_double2(a.x * b.x, a.y * b.y); }
    static __device__ __forceinline__ t fma(t a, t b, t c) {
        return make_double2(::fma(a.x, b.x, c.x), ::fma(a.y, b.y, c.y));
    }
};

// Scalar operations with their rounding spelled out (no contraction).
template <class C> struct SA;
template <> struct SA<float> {
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
};
template <> struct SA<double> {
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
};

// The lane's V values of a shared-memory row as V/2 pairs of the arithmetic type.
template <class T>
__device__ __forceinline__ void lds_pairs(const unsigned char* srow, int lane,
                                          typename Pair<typename Tr<T>::C>::t (&v)[Tr<T>::V / 2]) {
    const T* d = reinterpret_cast<const T*>(srow + 16) + lane * Tr<T>::V;
    const uint4 raw = *reinterpret_cast<const uint4*>(d);
    if constexpr (sizeof(T) == 8) {
        v[0] = make_double2(__longlong_as_double(((long long)raw.y << 32) | raw.x),
                            __longlong_as_double(((long long)raw.w << 32) | raw.z));
    } else if constexpr (sizeof(T) == 4) {
        v[0] = make_float2(__uint_as_float(raw.x), __uint_as_float(raw.y));
        v[1] = make_float2(__uint_as_float(raw.z), __uint_as_float(raw.w));
    } else {
        const unsigned wd[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if constexpr (std::is_same<T, __half>::value) v[k] = __half22float2(*reinterpret_cast<const __half2*>(&wd[k]));
            else v[k] = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&wd[k]));
        }
    }
}

// V values (as pairs) rounded to T, masked bitwise (wm: all-ones words keep,
// zero words clear) and stored with one 16-byte store.
template <class T>
__device__ __forceinline__ void st_pairs(T* p, const typename Pair<typename Tr<T>::C>::t (&v)[Tr<T>::V / 2], uint4 wm) {
    uint4 raw;
    if constexpr (sizeof(T) == 8) {
        const unsigned long long b0 = (unsigned long long)__double_as_longlong(v[0].x);
        const unsigned long long b1 = (unsigned long long)__double_as_longlong(v[0].y);
        raw = make_uint4((unsigned)b0, (unsigned)(b0 >> 32), (unsigned)b1, (unsigned)(b1 >> 32));
    } else if constexpr (sizeof(T) == 4) {
        raw = make_uint4(__float_as_uint(v[0].x), __float_as_uint(v[0].y), __float_as_uint(v[1].x),
                         __float_as_uint(v[1].y));
    } else {
        unsigned w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if constexpr (std::is_same<T, __half>::value) {
                const __half2 h = __float22half2_rn(v[k]);
                w[k] = *reinterpret_cast<const unsigned*>(&h);
            } else {
                const __nv_bfloat162 h = __float22bfloat162_rn(v[k]);
                w[k] = *reinterpret_cast<const unsigned*>(&h);
            }
        }
        raw = make_uint4(w[0], w[1], w[2], w[3]);
    }
    raw.x &= wm.x; raw.y &= wm.y; raw.z &= wm.z; raw.w &= wm.w;
    *reinterpret_cast<uint4*>(p) = raw;
}

// Word masks of a lane's 16-byte chunk starting at element x: elements at
// x + i >= n (the pad column and beyond) are cleared.
template <class T>
__device__ __forceinline__ uint4 pad_mask(int x, int n) {
    unsigned m[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if constexpr (sizeof(T) == 8) m[k] = x + k / 2 < n ? 0xffffffffu : 0u;
        else if constexpr (sizeof(T) == 4) m[k] = x + k < n ? 0xffffffffu : 0u;
        else m[k] = (x + 2 * k < n ? 0x0000ffffu : 0u) | (x + 2 * k + 1 < n ? 0xffff0000u : 0u);
    }
    return make_uint4(m[0], m[1], m[2], m[3]);
}

// Full weighting (Sec. 2, the transpose of trilinear interpolation) in integer
// weights: along each axis 1 2 1, summed as (r[2k] + 2 r[2k+1]) + r[2k+2], and
// the coarse value scaled by 2^-d once at the end.  Every partial sum is then the
// one weighted 1/4 1/2 1/4 times a power of two, so the result has the same bits
// (no partial sum is near the FP32 / FP64 range limits), at two operations per
// axis instead of three.
// Along x of one fine row: q[k] = (r[2k] + 2 r[2k+1]) + r[2k+2], r[V] taken from
// the next lane.
template <class C, int V, int VH>
__device__ __forceinline__ void fw_x(const C (&out)[V], int lane, C (&q)[VH]) {
    using A = SA<C>;
    C rn = __shfl_down_sync(kFull, out[0], 1);
    if (lane == 31) rn = 0;
#pragma unroll
    for (int k = 0; k < VH; ++k) {
        C r2 = (2 * k + 2 < V) ? out[(2 * k + 2) % V] : rn;
        q[k] = A::add(A::fma((C)2, out[2 * k + 1], out[2 * k]), r2);
    }
}
// One more axis of the weighting: (a + 2 b) + c.
template <class C>
__device__ __forceinline__ C fw_121(C a, C b, C c) { return SA<C>::add(SA<C>::fma((C)2, b, a), c); }

// ---------------------------------------------------------------- TMA / mbarrier
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for the phase with the given parity to complete, at most `tries`
// polls (each poll may suspend the thread for a short hardware-chosen time).
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, unsigned tries) {
    for (unsigned i = 0; i < tries; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap* m, int x, int y, int z, unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(m)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}
// Polls of one wait for a plane's tile copies (each poll may suspend the thread
// for a short hardware-chosen time: about a second in all).  KArgs::wait_polls
// = k + 1 > 0 replaces it by k polls for the waits of the march (a diagnostic
// setting: k = 0 gives up at once), never for the drain after a failed wait;
// 0 (the zero-initialised value) keeps the default.
constexpr unsigned kWaitTries = 1u << 20;
__device__ __forceinline__ unsigned march_wait_polls(const KArgs& a) {
    return a.wait_polls > 0 ? (unsigned)(a.wait_polls - 1) : kWaitTries;
}
// After the leader's own wait gave up: it issues no more copies and waits,
// with the full bound, for the last S planes it issued (march
// indices q_last-S+1 .. q_last, stage q % S, phase parity (q / S) & 1: each
// stage's latest phase; earlier phases of a stage completed before it was
// reissued), so that no bulk copy is still writing into the CTA's shared
// memory when it exits.  A phase that completed already passes at once.
// Returns false if a copy did not complete even then.
__device__ __forceinline__ bool drain_copies(unsigned bar0, int S, int q_last) {
    bool ok = true;
    for (int q = q_last - S + 1 > 0 ? q_last - S + 1 : 0; q <= q_last; ++q)
        ok = mbar_wait(bar0 + 8 * (q % S), (unsigned)(q / S) & 1u, kWaitTries) && ok;
    return ok;
}
// Marks the solve as stopped by a wait that gave up (DevState::kerr, reported
// as MG_ERR_TIMEOUT; phase 3 makes every later gated kernel return at once).
__device__ __forceinline__ void march_wait_failed(const KArgs& a) {
    if (a.err) atomicExch(a.err, 1);
    if (a.st) *reinterpret_cast<volatile int*>(&const_cast<DevState*>(a.st)->phase) = 3;
}

// ---------------------------------------------------------------- 3D sweep
// One CTA = TY warps; warp w owns fine row y0 + w of a 32*V-point x-chunk and
// marches z from zb to ze.  Each plane of the march is one TMA box of the
// swept vector (rows y0-1 .. y0+TY, x0-16B .. x0+512B+16B; the tensor map's
// out-of-range fill supplies the zero boundary outside the padded array) and,
// for Jacobi and residual, one box of g (rows y0 .. y0+TY-1), issued by one
// thread into a 6-stage ring and completed on the stage's mbarrier.  The
// lane's own row of planes z-1, z, z+1 stays in registers (three arrays that
// swap roles each plane: the loop body is unrolled three times).
// Launch bounds: 8 warps (9 for the residual-restriction tiles), 2 CTAs per SM:
// each of a warp's one or two rows keeps a four-plane window (finite
// differences, two planes per step), Q1 three in-plane sums per plane.
template <int MODE, int RPW, int OP = 0>
struct SweepLB {
    static constexpr int kThreads = MODE == M_RESTRICT ? 288 : 256;
    static constexpr int kMinBlocks = 2;
};
// The body takes the CTA's tile coordinates (bx, by, bz) explicitly: the
// single-grid kernel passes blockIdx, the batched kernel the coordinates of
// its (instance, tile) work item.  maps may live in parameter space or in
// global memory (64-byte aligned; written before the launch).
// OP = 1: the Q1 operator (27-point, Sec. 5).  W(z) = 2 (D(z) + X(z-1) + X(z+1))
// + D(z-1) + D(z+1) with X(p) the in-plane cross sum (x +- 1, y +- 1) and D(p)
// the in-plane diagonal sum of plane p at the row: X and D of a plane are
// formed once, when it arrives, and kept in registers with the plane's row.
template <int MODE, class T, class TC, int RPW, int OP>
__device__ __forceinline__ void sweep3_body(const KArgs& a, const SweepMaps& maps, int bx, int by, int bz) {
    using C = typename Tr<T>::C;
    constexpr bool Q1 = OP == 1;
    static_assert(!Q1 || RPW == 1, "the Q1 sweep keeps one row per warp");
    using PR = Pair<C>;
    using P2 = typename PR::t;
    constexpr int V = Tr<T>::V;
    constexpr int NP = V / 2;
    constexpr int CW = 32 * V;
    constexpr int VH = V / 2 > 0 ? V / 2 : 1;
    constexpr int S = sweep3_stages(MODE, RPW);  // planes z-1, z, z+1 in use, z+2 .. z+S-2 in flight
    constexpr bool NEED_G = MODE == M_JACOBI || MODE == M_RESTRICT;
    // finite differences: two planes per step (see step2)
    constexpr bool TWO = !Q1;
    constexpr int UB = sizeof(T) == 2 ? 4 : 8;  // bytes of one tensor-map unit
    constexpr int RB = kSweepRowBytes;
    if (a.gate && a.st->phase != 0) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
    const int TY = blockDim.y, lane = threadIdx.x, w = threadIdx.y;
    const int R = RPW * TY;  // rows of the CTA tile; warp w owns rows w, w + TY, ...
    const int CB = sweep3_cbytes(R);
    const int SB = sweep3_stage_bytes(R, NEED_G);
    unsigned char* flush = base + S * SB;
    // restriction: the rows' z-sums (two buffers, alternating, for TWO)
    const int flush_bytes = MODE == M_RESTRICT ? (TWO ? 2 : 1) * R * 32 * VH * (int)sizeof(C) : 0;
    const unsigned bar0 = smem_u32(flush + (flush_bytes + 15) / 16 * 16);
    const int x0 = bx * a.xstep, x = x0 + lane * V;
    const int y0 = by * a.ystep;
    const int zb = bz * a.zstep;
    const int ze = min(zb + a.zlen, a.n);
    const bool lane_in = x < a.P;
    const bool leader = w == 0 && lane == 0;
    const unsigned cbox = (unsigned)((R + 2) * RB), gbox = (unsigned)(R * 512);
    const int xc = (x0 * (int)sizeof(T) - 16) / UB, xg = x0 * (int)sizeof(T) / UB;  // 16-byte aligned starts
    // plane p (zb-1 <= p <= ze) is the q-th of the march, q = p - zb + 1: stage q % S, phase (q / S) & 1
    int q_issued = -1;  // leader: the march index of the last plane issued
    auto issue = [&](int p) {
        if (p > ze) return;
        const int q = p - zb + 1, s = q % S;
        q_issued = q;
        const unsigned bar = bar0 + 8 * s;
        const unsigned st = smem_u32(base + s * SB);
        const bool with_g = NEED_G && p >= zb && p < ze;
        mbar_expect_tx(bar, cbox + (with_g ? gbox : 0u));
        tma_load_3d(st, &maps.src, xc, y0 - 1, p + 1, bar);
        if (with_g) tma_load_3d(st + CB, &maps.g, xg, y0, p + 1, bar);
    };
    // the next plane to wait for: its stage and phase advance one plane at a time.
    // A wait that gives up marks this thread failed (and the solve timed out);
    // a failed thread waits no more.  The leader reissues a stage only after its
    // own wait saw that stage's previous copy land, so once its own wait gives
    // up it issues nothing more and, at the end, drains what it issued
    // (drain_copies); the other threads march on over whatever the ring holds.
    // Every thread thus waits at most one full bound in vain, and no copy is
    // in flight into a stage being reissued or when the CTA exits.
    int wst = 0;
    unsigned wpar = 0;
    bool failed = false;
    auto wait_next = [&]() {
        if (!failed && !mbar_wait(bar0 + 8 * wst, wpar, march_wait_polls(a))) {
            march_wait_failed(a);
            failed = true;
        }
        if (++wst == S) { wst = 0; wpar ^= 1u; }
    };
    if (leader) {
        for (int s = 0; s < S; ++s) mbar_init(bar0 + 8 * s, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (leader)
        for (int k = 0; k < S - 1; ++k) issue(zb - 1 + k);

    const P2 c1 = PR::splat(coef<C>(a.cf, 0)), c2 = PR::splat(coef<C>(a.cf, 1)), c3 = PR::splat(coef<C>(a.cf, 2));
    const P2 k2 = PR::splat(coef<C>(a.cf, 3));
    const P2 h2v = PR::splat(coef<C>(a.cf, 4)), mh6 = PR::splat(coef<C>(a.cf, 5));
    // points x >= n of the chunk are stored as 0 (they are the boundary)
    const uint4 wm = pad_mask<T>(x, a.n);
    C acc[RPW][VH];  // restriction: z-weighted sums of the rows' x-restricted residuals
#pragma unroll
    for (int r = 0; r < RPW; ++r)
#pragma unroll
        for (int k = 0; k < VH; ++k) acc[r][k] = 0;
    T* dst_row[RPW];
    bool do_store[RPW];
    int own[RPW];   // byte offset of the warp's row r within a c box
    int gown[RPW];  // ... within a g box, minus the 16-byte halo lds_pairs skips
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
        const int y = y0 + w + r * TY;
        do_store[r] = y < a.n && lane_in;
        dst_row[r] = reinterpret_cast<T*>(a.dst) + (long long)(y < a.n ? y : 0) * a.P + (lane_in ? x : 0);
        own[r] = (w + r * TY + 1) * RB;
        gown[r] = CB + (w + r * TY) * 512 - 16;
    }

    // the row and, for Q1, its in-plane cross (X) and diagonal (D) sums of the
    // plane in stage st
    auto xsum = [&](const P2 (&v)[NP], C l, C rgt, int k) {  // x-1 + x+1 of pair k
        const C xl = k ? v[k - 1].y : l;
        const C xr = k < NP - 1 ? v[k + 1].x : rgt;
        return PR::mk(xl + v[k].y, v[k].x + xr);
    };
    auto plane_in = [&](const unsigned char* st, int r, P2 (&c)[NP], P2 (&X)[NP], P2 (&D)[NP]) {
        lds_pairs<T>(st + own[r], lane, c);
        if constexpr (Q1) {
            P2 ym[NP], yp[NP];
            lds_pairs<T>(st + own[r] - RB, lane, ym);
            lds_pairs<T>(st + own[r] + RB, lane, yp);
            const C l0 = lds_one<T>(st + own[r], lane * V - 1), r0 = lds_one<T>(st + own[r], lane * V + V);
            const C lm = lds_one<T>(st + own[r] - RB, lane * V - 1), rm = lds_one<T>(st + own[r] - RB, lane * V + V);
            const C lp = lds_one<T>(st + own[r] + RB, lane * V - 1), rp = lds_one<T>(st + own[r] + RB, lane * V + V);
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                X[k] = PR::add(xsum(c, l0, r0, k), PR::add(ym[k], yp[k]));
                D[k] = PR::add(xsum(ym, lm, rm, k), xsum(yp, lp, rp, k));
            }
        }
    };
    P2 pa[RPW][NP], pb[RPW][NP], pc[RPW][NP];
    P2 qa[RPW][NP], qb[RPW][NP], qc[RPW][NP];  // Q1: X of the three planes
    P2 da[RPW][NP], db[RPW][NP], dc[RPW][NP];  // Q1: D of the three planes
    wait_next();  // plane zb-1
    wait_next();  // plane zb
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
        plane_in(base, r, pa[r], qa[r], da[r]);
        plane_in(base + SB, r, pb[r], qb[r], db[r]);
    }
    int so = SB;  // stage of plane z

    // Restriction: the coarse rows of coarse plane K from the z-sums that every
    // warp flushed to shared memory after fine plane 2K+2 (t = z - zb even,
    // t >= 2), taken one plane later, after the next plane's barrier: warp w < TJ
    // forms coarse row J0 + w from tile rows 2w, 2w+1, 2w+2 (y weights 1 2 1,
    // then the scale 1/64 of the integer weights, fw_x).  The flush area is
    // written again only two planes later, after another barrier, so one barrier
    // per plane serves both.  Coarse planes are taken in order K = zb/2, zb/2+1, ...
    // The values of a coarse row are split over two warps (halves of each lane's
    // VH values) where VH allows, so that 2 TJ of the TY warps share the work.
    constexpr int SPLIT = VH >= 2 ? 2 : 1;
    constexpr int VS = VH / SPLIT;
    const int Jc = (y0 >> 1) + w / SPLIT;
    const int I0 = ((x0 + lane * V) >> 1) + (w % SPLIT) * VS;
    const bool cw = MODE == M_RESTRICT && w < ((R - 1) / 2) * SPLIT && lane_in && Jc < a.nc &&
                    (lane < 31 || x0 + CW >= a.P);
    const C* f0 = reinterpret_cast<const C*>(flush) + ((2 * (w / SPLIT)) * 32 + lane) * VH + (w % SPLIT) * VS;
    int Kc = zb >> 1;  // the next coarse plane
    TC* cd = reinterpret_cast<TC*>(a.dst) + (cw ? (long long)Kc * a.Sc + (long long)Jc * a.Pc + I0 : 0ll);
    auto coarse_rows = [&](int buf = 0) {
        if (cw && Kc < a.nc) {
            const C* f = f0 + buf * (R * 32 * VH);
#pragma unroll
            for (int k = 0; k < VS; ++k)
                if (I0 + k < a.nc) st1(cd + k, SA<C>::mul(fw_121(f[k], f[32 * VH + k], f[64 * VH + k]), (C)(1.0 / 64)));
        }
        ++Kc;
        cd += a.Sc;
    };

    // One plane: cm / c0 hold planes z-1 / z, cp receives plane z+1 (and the
    // X / D sums of the same planes for Q1).
    auto step = [&](int z, const P2 (&cm)[RPW][NP], const P2 (&c0)[RPW][NP], P2 (&cp)[RPW][NP],
                    const P2 (&Xm)[RPW][NP], const P2 (&X0)[RPW][NP], P2 (&Xp)[RPW][NP],
                    const P2 (&dm)[RPW][NP], const P2 (&d0)[RPW][NP], P2 (&dp)[RPW][NP]) {
        __syncthreads();  // every warp is done with plane z-2's stage
        if (leader && !failed) issue(z + S - 2);
        if constexpr (MODE == M_RESTRICT && !Q1) {  // the flush of plane z-1 (t - 1 even, >= 2)
            const int tp = z - 1 - zb;
            if (tp >= 2 && !(tp & 1)) coarse_rows();
        }
        wait_next();      // plane z+1
        int s1 = so + SB;
        if (s1 >= S * SB) s1 -= S * SB;
        const unsigned char* st0 = base + so;
        C q[RPW][VH];  // restriction: the rows' x-restricted residuals of this plane
#pragma unroll
        for (int r = 0; r < RPW; ++r) {
            P2 ym[NP], yp[NP], g[NP];
            plane_in(base + s1, r, cp[r], Xp[r], dp[r]);
            C left = 0, right = 0;
            if constexpr (!Q1) {
                lds_pairs<T>(st0 + own[r] - RB, lane, ym);
                lds_pairs<T>(st0 + own[r] + RB, lane, yp);
                left = lds_one<T>(st0 + own[r], lane * V - 1);
                right = lds_one<T>(st0 + own[r], lane * V + V);
            }
            if (NEED_G) lds_pairs<T>(st0 + gown[r], lane, g);
            P2 out[NP];
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                P2 nb;
                if constexpr (Q1) {
                    // edges (weight 2): D(z), X(z-1), X(z+1); corners (weight 1): D(z-1), D(z+1)
                    const P2 e = PR::add(d0[r][k], PR::add(Xm[r][k], Xp[r][k]));
                    (void)X0;
                    nb = PR::fma(PR::splat((C)2), e, PR::add(dm[r][k], dp[r][k]));
                } else {
                    // x-neighbour sums: element 2k has 2k-1 and 2k+1, element 2k+1 has 2k and 2k+2
                    const P2 xs = xsum(c0[r], left, right, k);
                    nb = PR::add(PR::add(xs, PR::add(ym[k], yp[k])), PR::add(cm[r][k], cp[r][k]));
                }
                P2 v;
                if (MODE == M_JACOBI) v = PR::fma(c2, nb, PR::fma(c1, c0[r][k], PR::mul(c3, g[k])));  // c + w D^-1 (g - A c)
                else if (MODE == M_ZERO2) v = PR::mul(c3, PR::fma(c2, nb, PR::mul(k2, c0[r][k])));     // two sweeps from 0, c0 = g
                else if (MODE == M_ZERO1) v = PR::mul(c3, c0[r][k]);                                    // one sweep from 0
                else v = PR::fma(h2v, nb, PR::fma(mh6, c0[r][k], g[k]));                               // residual g - A c
                out[k] = v;
            }
            if constexpr (MODE != M_RESTRICT) {
                if (do_store[r]) st_pairs<T>(dst_row[r] + (long long)z * a.S, out, wm);
            } else {
                C o1[V];
#pragma unroll
                for (int k = 0; k < NP; ++k) { o1[2 * k] = out[k].x; o1[2 * k + 1] = out[k].y; }
                fw_x<C, V, VH>(o1, lane, q[r]);
            }
        }
        if constexpr (MODE == M_RESTRICT) {
            // z: fine planes 2K, 2K+1, 2K+2 (t = 0, 1, 2 from the range start)
            // weigh 1 2 1; after an even plane t >= 2 the rows' z-sums go
            // through shared memory and warp w forms coarse row J0 + w from
            // tile rows 2w, 2w+1, 2w+2 (coarse_rows)
            const int t = z - zb;
            if (t & 1) {
#pragma unroll
                for (int r = 0; r < RPW; ++r)
#pragma unroll
                    for (int k = 0; k < VH; ++k) acc[r][k] = SA<C>::fma((C)2, q[r][k], acc[r][k]);
            } else {
                if (t >= 2) {  // consumed by coarse_rows after the next barrier (Q1: at once,
                               // which keeps its register pressure down)
#pragma unroll
                    for (int r = 0; r < RPW; ++r) {
                        C* fl = reinterpret_cast<C*>(flush) + ((w + r * TY) * 32 + lane) * VH;
#pragma unroll
                        for (int k = 0; k < VH; ++k) fl[k] = SA<C>::add(acc[r][k], q[r][k]);
                    }
                    if constexpr (Q1) {
                        __syncthreads();
                        coarse_rows();
                    }
                }
#pragma unroll
                for (int r = 0; r < RPW; ++r)
#pragma unroll
                    for (int k = 0; k < VH; ++k) acc[r][k] = q[r][k];
            }
        }
        so = s1;
    };
    if constexpr (TWO) {
        // Finite differences, two planes per step: planes z (t = z - zb even)
        // and z+1 (t odd) from the four-plane window A = z-1, B = z, C = z+1,
        // D = z+2 of each of the warp's rows, each with the operations of step --
        // twice the independent chains per warp and one barrier per two planes.
        // The leader issues planes z+4 and z+5 into the stages of z-2 and z-1,
        // which no warp uses after the barrier.  Restriction: the z-sum of plane
        // t (even, t >= 2) goes to flush buffer (t / 2) & 1, and its coarse rows
        // are formed after the next step's barrier; the next write into that
        // buffer follows one more barrier.
        // The values of plane z (stage st) of the warp's row.
        auto row_out = [&](int r, const unsigned char* st, const P2 (&cm)[NP], const P2 (&c0)[NP], const P2 (&cp)[NP],
                           P2 (&out)[NP]) {
            P2 ym[NP], yp[NP], g[NP];
            lds_pairs<T>(st + own[r] - RB, lane, ym);
            lds_pairs<T>(st + own[r] + RB, lane, yp);
            const C left = lds_one<T>(st + own[r], lane * V - 1);
            const C right = lds_one<T>(st + own[r], lane * V + V);
            if (NEED_G) lds_pairs<T>(st + gown[r], lane, g);
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const P2 xs = xsum(c0, left, right, k);
                const P2 nb = PR::add(PR::add(xs, PR::add(ym[k], yp[k])), PR::add(cm[k], cp[k]));
                P2 v;
                if (MODE == M_JACOBI) v = PR::fma(c2, nb, PR::fma(c1, c0[k], PR::mul(c3, g[k])));
                else if (MODE == M_ZERO2) v = PR::mul(c3, PR::fma(c2, nb, PR::mul(k2, c0[k])));
                else if (MODE == M_ZERO1) v = PR::mul(c3, c0[k]);
                else v = PR::fma(h2v, nb, PR::fma(mh6, c0[k], g[k]));
                out[k] = v;
            }
        };
        // the plane's result: stored (sweeps) or x-restricted (restriction)
        auto plane_done = [&](int r, int z, const P2 (&out)[NP], C (&q)[VH]) {
            if constexpr (MODE == M_RESTRICT) {
                C o1[V];
#pragma unroll
                for (int k = 0; k < NP; ++k) { o1[2 * k] = out[k].x; o1[2 * k + 1] = out[k].y; }
                fw_x<C, V, VH>(o1, lane, q);
            } else {
                (void)q;
                if (do_store[r]) st_pairs<T>(dst_row[r] + (long long)z * a.S, out, wm);
            }
        };
        auto step2 = [&](int z, const P2 (&A)[RPW][NP], const P2 (&B)[RPW][NP], P2 (&Cn)[RPW][NP], P2 (&D)[RPW][NP]) {
            __syncthreads();  // every warp is done with the stages of planes z-2 and z-1
            if (leader && !failed) {
                issue(z + S - 2);
                issue(z + S - 1);
            }
            const int t = z - zb;  // even
            if constexpr (MODE == M_RESTRICT)
                if (t >= 4) coarse_rows(((t - 2) >> 1) & 1);  // the z-sums of plane z-2
            const bool two = z + 1 < ze;
            wait_next();            // plane z+1
            if (two) wait_next();   // plane z+2 (<= ze)
            int s1 = so + SB;
            if (s1 >= S * SB) s1 -= S * SB;
            int s2 = s1 + SB;
            if (s2 >= S * SB) s2 -= S * SB;
            C q0[VH], q1[VH];  // restriction (one row per warp): the planes' x-restricted residuals
#pragma unroll
            for (int r = 0; r < RPW; ++r) {
                P2 o0[NP];
                lds_pairs<T>(base + s1 + own[r], lane, Cn[r]);
                row_out(r, base + so, A[r], B[r], Cn[r], o0);
                plane_done(r, z, o0, q0);
            }
            if (two) {
#pragma unroll
                for (int r = 0; r < RPW; ++r) {
                    P2 o1[NP];
                    lds_pairs<T>(base + s2 + own[r], lane, D[r]);
                    row_out(r, base + s1, B[r], Cn[r], D[r], o1);
                    plane_done(r, z + 1, o1, q1);
                }
            }
            if constexpr (MODE != M_RESTRICT) {
                so = s2;
                return;
            }
            // z weights 1 2 1: plane t closes the coarse plane of planes t-2, t-1, t
            if (t >= 2) {
                C* fl = reinterpret_cast<C*>(flush) + ((((t >> 1) & 1) * R + w) * 32 + lane) * VH;
#pragma unroll
                for (int k = 0; k < VH; ++k) fl[k] = SA<C>::add(acc[0][k], q0[k]);
            }
#pragma unroll
            for (int k = 0; k < VH; ++k) acc[0][k] = q0[k];
            if (two) {
#pragma unroll
                for (int k = 0; k < VH; ++k) acc[0][k] = SA<C>::fma((C)2, q1[k], acc[0][k]);
            }
            so = s2;
        };
        for (int z = zb; z < ze;) {
            step2(z, pa, pb, pc, qa);
            if ((z += 2) >= ze) break;
            step2(z, pc, qa, pa, pb);
            z += 2;
        }
        if constexpr (MODE == M_RESTRICT) {
            const int tl = (ze - 1 - zb) & ~1;  // the last step's even plane
            __syncthreads();
            if (tl >= 2) coarse_rows((tl >> 1) & 1);
        }
    } else {
        for (int z = zb; z < ze;) {
            step(z, pa, pb, pc, qa, qb, qc, da, db, dc);
            if (++z >= ze) break;
            step(z, pb, pc, pa, qb, qc, qa, db, dc, da);
            if (++z >= ze) break;
            step(z, pc, pa, pb, qc, qa, qb, dc, da, db);
            ++z;
        }
        if constexpr (MODE == M_RESTRICT && !Q1) {  // the flush of the march's last plane
            __syncthreads();
            const int tp = ze - 1 - zb;
            if (tp >= 2 && !(tp & 1)) coarse_rows();
        }
    }
    if (leader && failed && !drain_copies(bar0, S, q_issued) && a.err) atomicExch(a.err, 2);
}

template <int MODE, class T, class TC, int RPW, int OP = 0>
__global__ void __launch_bounds__(SweepLB<MODE, RPW, OP>::kThreads, SweepLB<MODE, RPW, OP>::kMinBlocks)
    k_sweep3(const KArgs a, const __grid_constant__ SweepMaps maps) {
    sweep3_body<MODE, T, TC, RPW, OP>(a, maps, blockIdx.x, blockIdx.y, blockIdx.z);
}
// Batched: CTA -> work item through a table; the item's grid (gx, gy, gz)
// decodes the CTA's tile.
template <int MODE, class T, class TC, int RPW, int OP = 0>
__global__ void __launch_bounds__(SweepLB<MODE, RPW, OP>::kThreads, SweepLB<MODE, RPW, OP>::kMinBlocks)
    k_sweep3_batch(const SweepItem* __restrict__ items, const int* __restrict__ cta_item) {
    const SweepItem& it = items[cta_item[blockIdx.x]];
    const int local = blockIdx.x - it.cta_begin;
    const int bx = local % it.gx, rest = local / it.gx;
    sweep3_body<MODE, T, TC, RPW, OP>(it.a, it.maps, bx, rest % it.gy, rest / it.gy);
}

// ---------------------------------------------------------------- 3D direct kernels for small levels
// Levels that live in L2 are bound by latency, not bandwidth: a marching tile
// pays its pipeline fill per CTA.  These kernels give every thread one V-vector
// of a row (sweeps) or one coarse point (residual-restriction) and read the
// operands through the read-only path.  They perform the same IEEE operations
// in the same order as k_sweep3 (finite differences), so a level gives the same
// bits whichever of the two runs it.

template <int MODE, class T>
__device__ __forceinline__ void dsweep3_body(const KArgs& a, int cta) {
    using C = typename Tr<T>::C;
    using A = SA<C>;
    constexpr int V = Tr<T>::V;
    constexpr bool NEED_G = MODE == M_JACOBI;
    if (a.gate && a.st->phase != 0) return;
    const int vpr = a.P / V;
    const int idx = cta * blockDim.x + threadIdx.x;
    if (idx >= vpr * a.n * a.n) return;
    const int row = idx / vpr;
    const int x = (idx - row * vpr) * V;
    const int z = row / a.n, y = row - z * a.n;
    const long long o = offs<3>(x, y, z, a.P, a.S);
    const T* src = reinterpret_cast<const T*>(a.src) + o;
    const C c1 = coef<C>(a.cf, 0), c2 = coef<C>(a.cf, 1), c3 = coef<C>(a.cf, 2), k2 = coef<C>(a.cf, 3);
    C c0[V], out[V];
    ldv(src, c0);
    if constexpr (MODE == M_ZERO1) {
#pragma unroll
        for (int i = 0; i < V; ++i) out[i] = x + i < a.n ? A::mul(c3, c0[i]) : (C)0;
    } else {
        C ym[V], yp[V], zm[V], zp[V], g[V];
        ldv(src - a.P, ym);
        ldv(src + a.P, yp);
        ldv(src - a.S, zm);
        ldv(src + a.S, zp);
        if (NEED_G) ldv(reinterpret_cast<const T*>(a.g) + o, g);
        const C left = ld1(src - 1), right = ld1(src + V);
#pragma unroll
        for (int i = 0; i < V; ++i) {
            const C xs = A::add(i ? c0[i - 1] : left, i < V - 1 ? c0[i + 1] : right);
            const C nb = A::add(A::add(xs, A::add(ym[i], yp[i])), A::add(zm[i], zp[i]));
            C v;
            if (MODE == M_JACOBI) v = A::fma(c2, nb, A::fma(c1, c0[i], A::mul(c3, g[i])));
            else v = A::mul(c3, A::fma(c2, nb, A::mul(k2, c0[i])));
            out[i] = x + i < a.n ? v : (C)0;
        }
    }
    stv(reinterpret_cast<T*>(a.dst) + o, out);
}
template <int MODE, class T>
__global__ void __launch_bounds__(256) k_dsweep3(const KArgs a) { dsweep3_body<MODE, T>(a, blockIdx.x); }
template <int MODE, class T>
__global__ void __launch_bounds__(256) k_dsweep3_batch(const KItem* __restrict__ items, const int* __restrict__ cta_item) {
    const KItem& it = items[cta_item[blockIdx.x]];
    dsweep3_body<MODE, T>(it.a, blockIdx.x - it.cta_begin);
}

// Coarse point (I, J, K) = R (g - A c) over fine points 2I..2I+2 (x), 2J..2J+2 (y),
// 2K..2K+2 (z): x first, then z, then y, as the marching kernel combines them.
template <class T, class TC>
__device__ __forceinline__ void drestrict3_body(const KArgs& a, int cta) {
    using C = typename Tr<T>::C;
    using A = SA<C>;
    if (a.gate && a.st->phase != 0) return;
    const int nc = a.nc;
    const int idx = cta * blockDim.x + threadIdx.x;
    if (idx >= nc * nc * nc) return;
    const int I = idx % nc, J = (idx / nc) % nc, K = idx / (nc * nc);
    const C h2v = coef<C>(a.cf, 4), mh6 = coef<C>(a.cf, 5);
    const T* c = reinterpret_cast<const T*>(a.src);
    const T* g = reinterpret_cast<const T*>(a.g);
    auto resid = [&](int fx, int fy, int fz) {  // g - A c at a fine point, as k_sweep3 forms it
        const long long o = offs<3>(fx, fy, fz, a.P, a.S);
        const T* p = c + o;
        const C xs = A::add(ld1(p - 1), ld1(p + 1));
        const C nb = A::add(A::add(xs, A::add(ld1(p - a.P), ld1(p + a.P))), A::add(ld1(p - a.S), ld1(p + a.S)));
        return A::fma(h2v, nb, A::fma(mh6, ld1(p), ld1(g + o)));
    };
    C zr[3];  // z-combined x-restrictions of the fine rows 2J, 2J+1, 2J+2
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
        C q[3];
#pragma unroll
        for (int dz = 0; dz < 3; ++dz) {
            const int fy = 2 * J + dy, fz = 2 * K + dz, fx = 2 * I;
            q[dz] = fw_121(resid(fx, fy, fz), resid(fx + 1, fy, fz), resid(fx + 2, fy, fz));
        }
        zr[dy] = fw_121(q[0], q[1], q[2]);
    }
    const C v = A::mul(fw_121(zr[0], zr[1], zr[2]), (C)(1.0 / 64));  // integer weights (fw_x)
    st1(reinterpret_cast<TC*>(a.dst) + offs<3>(I, J, K, a.Pc, a.Sc), v);
}
template <class T, class TC>
__global__ void __launch_bounds__(256) k_drestrict3(const KArgs a) { drestrict3_body<T, TC>(a, blockIdx.x); }
template <class T, class TC>
__global__ void __launch_bounds__(256) k_drestrict3_batch(const KItem* __restrict__ items, const int* __restrict__ cta_item) {
    const KItem& it = items[cta_item[blockIdx.x]];
    drestrict3_body<T, TC>(it.a, blockIdx.x - it.cta_begin);
}

// ---------------------------------------------------------------- 3D one-pass pre-smoothing + restriction
// Temporal blocking of Alg. 1's pre-smoothing and residual restriction on one level (M_PRE): for a tile of
// R = 2TJ+1 fine rows and 2TK+1 fine planes it computes the two damped
// Jacobi sweeps from zero, c = w D^-1 [(2 - w) g + (w/2d) N g], on R+2 rows
// (one halo row each side), rounds c to the storage type and writes it, then
// the residual g - A c on the R rows and its full weighting onto the coarse
// level -- reading g once instead of g for the sweeps, then c and g again for
// the residual.  Per plane p of g (TMA boxes of R+4 rows with 16-byte x-halos
// into a 6-stage ring): stage A forms c on plane p-1 from g planes p-2..p into
// a 3-plane ring of c rows (in the storage type, x-halo elements included),
// stage B the residual on plane p-2 from c planes p-3..p-1, then the
// restriction exactly as M_RESTRICT does.  One row per warp (warps 0 and R-1
// also form the two halo rows of c).
template <class T, class TC>
__device__ __forceinline__ void pre3_body(const KArgs& a, const SweepMaps& maps, int bx, int by, int bz) {
    using C = typename Tr<T>::C;
    using PR = Pair<C>;
    using P2 = typename PR::t;
    constexpr int V = Tr<T>::V;
    constexpr int NP = V / 2;
    constexpr int CW = 32 * V;
    constexpr int VH = V / 2 > 0 ? V / 2 : 1;
    constexpr int SG = kPreStagesG, SC = kPreStagesC;
    constexpr int UB = sizeof(T) == 2 ? 4 : 8;
    constexpr int RB = kSweepRowBytes;
    if (a.gate && a.st->phase != 0) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
    const int TY = blockDim.y, lane = threadIdx.x, w = threadIdx.y;
    const int R = TY;                        // residual rows of the tile
    const int GBs = pre3_gbytes(R), CBs = pre3_cbytes(R);
    unsigned char* gring = base;
    unsigned char* cring = base + SG * GBs;
    unsigned char* flush = cring + SC * CBs;
    const int flush_bytes = R * 32 * VH * (int)sizeof(C);
    const unsigned bar0 = smem_u32(flush + (flush_bytes + 15) / 16 * 16);
    const int x0 = bx * a.xstep, x = x0 + lane * V;
    const int y0 = by * a.ystep;
    const int zb = bz * a.zstep;
    const int ze = min(zb + a.zlen, a.n);  // residual planes [zb, ze)
    const bool lane_in = x < a.P;
    const bool leader = w == 0 && lane == 0;
    const unsigned gbox = (unsigned)((R + 4) * RB);
    const int xc = (x0 * (int)sizeof(T) - 16) / UB;
    auto gslot = [&](int p) { return gring + ((p - zb + 2) % SG) * GBs; };   // p >= zb - 2
    auto cslot = [&](int p) { return cring + ((p - zb + 1) % SC) * CBs; };   // p >= zb - 1
    int q_issued = -1;  // leader: the march index of the last g plane issued
    auto issue = [&](int p) {
        if (p > ze + 1) return;
        const int q = p - zb + 2, s = q % SG;
        q_issued = q;
        const unsigned bar = bar0 + 8 * s;
        mbar_expect_tx(bar, gbox);
        tma_load_3d(smem_u32(gring + s * GBs), &maps.src, xc, y0 - 2, p + 1, bar);
    };
    // bounded waits as in sweep3_body: a thread whose wait gave up waits no
    // more; the leader stops issuing after its own failed wait and drains
    int wst = 0;
    unsigned wpar = 0;
    bool failed = false;
    auto wait_next = [&]() {
        if (!failed && !mbar_wait(bar0 + 8 * wst, wpar, march_wait_polls(a))) {
            march_wait_failed(a);
            failed = true;
        }
        if (++wst == SG) { wst = 0; wpar ^= 1u; }
    };
    if (leader) {
        for (int s = 0; s < SG; ++s) mbar_init(bar0 + 8 * s, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (leader)
        for (int k = 0; k < 3; ++k) issue(zb - 2 + k);

    const P2 c2 = PR::splat(coef<C>(a.cf, 1)), c3 = PR::splat(coef<C>(a.cf, 2)), k2 = PR::splat(coef<C>(a.cf, 3));
    const P2 h2v = PR::splat(coef<C>(a.cf, 4)), mh6 = PR::splat(coef<C>(a.cf, 5));
    const uint4 wm = pad_mask<T>(x, a.n);
    const bool left_zero = x0 == 0, right_zero = x0 + CW >= a.P;
    C acc[VH];
#pragma unroll
    for (int k = 0; k < VH; ++k) acc[k] = 0;

    // c = ZERO2(g) from the pair of centre values and neighbour sums, with the
    // operations (and so the roundings) of the M_ZERO2 sweep
    auto zero2 = [&](P2 g0, P2 nb) { return PR::mul(c3, PR::fma(c2, nb, PR::mul(k2, g0))); };
    auto zero2_1 = [&](C g0, C nb) { return zero2(PR::mk(g0, g0), PR::mk(nb, nb)).x; };
    // c row cr (fine row y0-1+cr) of plane pc from the g ring; writes the c
    // ring row (with its halo elements) and, for the tile's rows, global c
    auto c_row = [&](int cr, int pc, unsigned char* cs) {
        unsigned char* crow = cs + cr * RB;
        const int fy = y0 - 1 + cr;
        T* d = reinterpret_cast<T*>(crow + 16);
        if (fy < 0 || fy >= a.n || pc < 0 || pc >= a.n) {  // outside the grid: the zero boundary
            *reinterpret_cast<uint4*>(d + lane * V) = make_uint4(0, 0, 0, 0);
            if (lane == 0) d[-1] = T(0.0f);
            if (lane == 31) d[CW] = T(0.0f);
            return;
        }
        const unsigned char* g1 = gslot(pc) + (cr + 1) * RB;  // g row fy on plane pc
        P2 g0[NP], ym[NP], yp[NP], zm[NP], zp[NP];
        lds_pairs<T>(g1, lane, g0);
        lds_pairs<T>(g1 - RB, lane, ym);
        lds_pairs<T>(g1 + RB, lane, yp);
        lds_pairs<T>(gslot(pc - 1) + (cr + 1) * RB, lane, zm);
        lds_pairs<T>(gslot(pc + 1) + (cr + 1) * RB, lane, zp);
        const C left = lds_one<T>(g1, lane * V - 1), right = lds_one<T>(g1, lane * V + V);
        P2 out[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const C xl = k ? g0[k - 1].y : left;
            const C xr = k < NP - 1 ? g0[k + 1].x : right;
            const P2 xs = PR::mk(xl + g0[k].y, g0[k].x + xr);
            const P2 nb = PR::add(PR::add(xs, PR::add(ym[k], yp[k])), PR::add(zm[k], zp[k]));
            out[k] = zero2(g0[k], nb);
        }
        // into the c ring (pads masked to zero), and to global for the tile's rows
        st_pairs<T>(d + lane * V, out, wm);
        if (lane_in && fy >= y0 && pc >= zb && pc < ze)
            st_pairs<T>(reinterpret_cast<T*>(a.dst2) + (long long)pc * a.S + (long long)fy * a.P + x, out, wm);
        // x-halo elements of the c row: zero at the boundary, else c there
        if (lane == 0) {
            C v = 0;
            if (!left_zero) {
                const C nb = ((lds_one<T>(g1, -2) + lds_one<T>(g1, 0)) +
                              (lds_one<T>(g1 - RB, -1) + lds_one<T>(g1 + RB, -1))) +
                             (lds_one<T>(gslot(pc - 1) + (cr + 1) * RB, -1) + lds_one<T>(gslot(pc + 1) + (cr + 1) * RB, -1));
                v = zero2_1(lds_one<T>(g1, -1), nb);
            }
            st1(d - 1, v);
        }
        if (lane == 31) {
            C v = 0;
            if (!right_zero) {
                const C nb = ((lds_one<T>(g1, CW - 1) + lds_one<T>(g1, CW + 1)) +
                              (lds_one<T>(g1 - RB, CW) + lds_one<T>(g1 + RB, CW))) +
                             (lds_one<T>(gslot(pc - 1) + (cr + 1) * RB, CW) + lds_one<T>(gslot(pc + 1) + (cr + 1) * RB, CW));
                v = x0 + CW < a.n ? zero2_1(lds_one<T>(g1, CW), nb) : (C)0;
            }
            st1(d + CW, v);
        }
    };

    for (int p = zb - 2; p <= ze + 1; ++p) {
        __syncthreads();  // the g slot of p+3 and the c slot of p-1 are free
        if (leader && !failed) issue(p + 3);
        wait_next();      // g plane p
        // ---- stage A: c on plane p-1, rows y0-1 .. y0+R
        if (p >= zb) {
            unsigned char* cs = cslot(p - 1);
            c_row(w + 1, p - 1, cs);
            if (w == 0) c_row(0, p - 1, cs);
            if (w == TY - 1) c_row(R + 1, p - 1, cs);
        }
        __syncthreads();
        // ---- stage B: residual on plane q = p-2, rows y0 .. y0+R-1, and the restriction
        const int q = p - 2;
        if (q < zb) continue;
        const unsigned char* c0s = cslot(q) + (w + 1) * RB;
        P2 c0[NP], ym[NP], yp[NP], zm[NP], zp[NP], g[NP];
        lds_pairs<T>(c0s, lane, c0);
        lds_pairs<T>(c0s - RB, lane, ym);
        lds_pairs<T>(c0s + RB, lane, yp);
        lds_pairs<T>(cslot(q - 1) + (w + 1) * RB, lane, zm);
        lds_pairs<T>(cslot(q + 1) + (w + 1) * RB, lane, zp);
        lds_pairs<T>(gslot(q) + (w + 2) * RB, lane, g);
        const C left = lds_one<T>(c0s, lane * V - 1), right = lds_one<T>(c0s, lane * V + V);
        C o1[V];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const C xl = k ? c0[k - 1].y : left;
            const C xr = k < NP - 1 ? c0[k + 1].x : right;
            const P2 xs = PR::mk(xl + c0[k].y, c0[k].x + xr);
            const P2 nb = PR::add(PR::add(xs, PR::add(ym[k], yp[k])), PR::add(zm[k], zp[k]));
            const P2 v = PR::fma(h2v, nb, PR::fma(mh6, c0[k], g[k]));  // residual g - A c
            o1[2 * k] = v.x;
            o1[2 * k + 1] = v.y;
        }
        C qv[VH];
        fw_x<C, V, VH>(o1, lane, qv);
        const int t = q - zb;
        if (t & 1) {
#pragma unroll
            for (int k = 0; k < VH; ++k) acc[k] = SA<C>::fma((C)2, qv[k], acc[k]);
        } else {
            if (t >= 2) {  // fine planes 2K, 2K+1, 2K+2 done: coarse plane K
                C* fl = reinterpret_cast<C*>(flush) + (w * 32 + lane) * VH;
#pragma unroll
                for (int k = 0; k < VH; ++k) fl[k] = SA<C>::add(acc[k], qv[k]);
                __syncthreads();
                const int TJ = (R - 1) / 2;
                if (w < TJ) {
                    const int J = (y0 >> 1) + w, K = (zb >> 1) + (t >> 1) - 1;
                    const C* f0 = reinterpret_cast<const C*>(flush) + ((2 * w) * 32 + lane) * VH;
                    const C* f1 = f0 + 32 * VH;
                    const C* f2 = f1 + 32 * VH;
                    const int I0 = (x0 + lane * V) >> 1;
                    if (lane_in && J < a.nc && K < a.nc && (lane < 31 || x0 + CW >= a.P)) {
                        TC* cd = reinterpret_cast<TC*>(a.dst) + (long long)K * a.Sc + (long long)J * a.Pc;
#pragma unroll
                        for (int k = 0; k < VH; ++k)
                            if (I0 + k < a.nc) st1(cd + I0 + k, SA<C>::mul(fw_121(f0[k], f1[k], f2[k]), (C)(1.0 / 64)));
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < VH; ++k) acc[k] = qv[k];
        }
    }
    if (leader && failed && !drain_copies(bar0, SG, q_issued) && a.err) atomicExch(a.err, 2);
}
template <class T, class TC>
__global__ void __launch_bounds__(288, 3) k_pre3(const KArgs a, const __grid_constant__ SweepMaps maps) {
    pre3_body<T, TC>(a, maps, blockIdx.x, blockIdx.y, blockIdx.z);
}
template <class T, class TC>
__global__ void __launch_bounds__(288, 3) k_pre3_batch(const SweepItem* __restrict__ items, const int* __restrict__ cta_item) {
    const SweepItem& it = items[cta_item[blockIdx.x]];
    const int local = blockIdx.x - it.cta_begin;
    const int bx = local % it.gx, rest = local / it.gx;
    pre3_body<T, TC>(it.a, it.maps, bx, rest % it.gy, rest / it.gy);
}

// ---------------------------------------------------------------- 2D sweep
// OP = 1: the Q1 operator, W = the 8 neighbours (rows y-1, y+1 with their halos)
template <int MODE, class T, class TC, int OP>
__global__ void __launch_bounds__(256) k_sweep2(const KArgs a) {
    using C = typename Tr<T>::C;
    constexpr int V = Tr<T>::V;
    constexpr int CW = 32 * V;
    constexpr int VH = V / 2 > 0 ? V / 2 : 1;
    constexpr int S = 6;  // per-warp ring of rows: y-1, y, y+1 in use, y+2..y+4 in flight
    constexpr bool NEED_G = MODE == M_JACOBI || MODE == M_RESTRICT;
    if (a.gate && a.st->phase != 0) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int W = blockDim.y, lane = threadIdx.x, w = threadIdx.y;
    const int wbytes = S * (NEED_G ? 2 : 1) * kRowBytes;
    unsigned char* mine = smem_raw + w * wbytes;
    const int x0 = (blockIdx.x * W + w) * a.xstep, x = x0 + lane * V;
    const bool chunk_in = x0 < a.P, lane_in = chunk_in && x < a.P;
    const int yb = blockIdx.y * a.zstep;
    const int ye = min(yb + a.zlen, a.n);
    const T* src = reinterpret_cast<const T*>(a.src);
    const T* gp = reinterpret_cast<const T*>(a.g);
    auto slot = [&](int p) { return (p - yb + 1) % S; };
    auto crow = [&](int st) { return mine + st * kRowBytes; };
    auto grow = [&](int st) { return mine + (S + st) * kRowBytes; };
    auto issue = [&](int p) {
        if (p <= ye && chunk_in) {
            const int st = slot(p);
            issue_row<T>(crow(st), src + (long long)p * a.P, lane, x0, a.P, true);
            if (NEED_G && p >= yb && p < ye) {
                const T* gr = lane_in ? gp + (long long)p * a.P + x : gp;
                cp_async16(reinterpret_cast<T*>(grow(st) + 16) + lane * V, gr, lane_in);
            }
        }
        cp_commit();
    };
#pragma unroll
    for (int k = 0; k < S - 1; ++k) issue(yb - 1 + k);
    const C c1 = coef<C>(a.cf, 0), c2 = coef<C>(a.cf, 1), c3 = coef<C>(a.cf, 2), k2 = coef<C>(a.cf, 3);
    const C h2inv = coef<C>(a.cf, 4), twod = (C)(OP == 1 ? 8 : 4);
    C acc[VH];
#pragma unroll
    for (int k = 0; k < VH; ++k) acc[k] = 0;
    // rows y-1, y, y+1 of the lane's chunk stay in registers (converted once)
    C cm[V], c0[V], cp[V];
    cp_wait<S - 3>();
    __syncwarp();
    lds_vec<T>(crow(slot(yb - 1)), lane, cm);
    lds_vec<T>(crow(slot(yb)), lane, c0);
    for (int y = yb; y < ye; ++y) {
        cp_wait<S - 4>();
        __syncwarp();      // the lanes' copies of row y+1 have landed; row y-2's slot is free
        issue(y + S - 2);  // reuses the slot of row y-2
        const int s0 = slot(y);
        C g[V];
        lds_vec<T>(crow(slot(y + 1)), lane, cp);
        const C left = lds_one<T>(crow(s0), lane * V - 1);
        const C right = lds_one<T>(crow(s0), lane * V + V);
        C lm = 0, rm = 0, lp = 0, rp = 0;  // halos of rows y-1, y+1 (Q1 only)
        if constexpr (OP == 1) {
            lm = lds_one<T>(crow(slot(y - 1)), lane * V - 1);
            rm = lds_one<T>(crow(slot(y - 1)), lane * V + V);
            lp = lds_one<T>(crow(slot(y + 1)), lane * V - 1);
            rp = lds_one<T>(crow(slot(y + 1)), lane * V + V);
        }
        if (NEED_G) lds_vec<T>(grow(s0), lane, g);
        C out[V];
#pragma unroll
        for (int i = 0; i < V; ++i) {
            C nb = (i ? c0[i - 1] : left) + (i < V - 1 ? c0[i + 1] : right) + cm[i] + cp[i];
            if constexpr (OP == 1)
                nb += ((i ? cm[i - 1] : lm) + (i < V - 1 ? cm[i + 1] : rm)) +
                      ((i ? cp[i - 1] : lp) + (i < V - 1 ? cp[i + 1] : rp));
            const C v = point_value<MODE, C>(c0[i], nb, NEED_G ? g[i] : (C)0, c1, c2, c3, h2inv, twod, k2);
            out[i] = (x + i < a.n) ? v : (C)0;
        }
#pragma unroll
        for (int i = 0; i < V; ++i) { cm[i] = c0[i]; c0[i] = cp[i]; }
        if constexpr (MODE != M_RESTRICT) {
            if (lane_in) stv(reinterpret_cast<T*>(a.dst) + offs<2>(x, y, 0, a.P, a.S), out);
        } else {
            C q[VH];
            fw_x<C, V, VH>(out, lane, q);
            const int t = y - yb;
            if (t & 1) {
#pragma unroll
                for (int k = 0; k < VH; ++k) acc[k] = SA<C>::fma((C)2, q[k], acc[k]);
            } else {
                if (t >= 2) {
                    const int J = (yb >> 1) + (t >> 1) - 1;
                    const int I0 = (x0 + lane * V) >> 1;
                    if (lane_in && J < a.nc && (lane < 31 || x0 + CW >= a.P)) {
                        TC* cd = reinterpret_cast<TC*>(a.dst) + (long long)J * a.Pc;
#pragma unroll
                        for (int k = 0; k < VH; ++k)
                            if (I0 + k < a.nc) st1(cd + I0 + k, SA<C>::mul(SA<C>::add(acc[k], q[k]), (C)(1.0 / 16)));
                    }
                }
#pragma unroll
                for (int k = 0; k < VH; ++k) acc[k] = q[k];
            }
        }
    }
    cp_wait<0>();
}

// ---------------------------------------------------------------- scale and cast (Alg. 2's residual scaling)
// Multiplication by inv split as 2^E * m, m in [1, 2): the exponent is added
// to the FP64 bit pattern with an integer add (exact), the significand product
// is done in FP32, then one rounding to the storage type.  No FP64 instruction.
struct ScaleK {
    double inv;
    long long eadd;
    float mant;
};
__device__ __forceinline__ ScaleK make_scale(double inv) {
    ScaleK k;
    k.inv = inv;
    long long b = __double_as_longlong(inv);
    int E = (int)((b >> 52) & 0x7FF) - 1023;
    k.eadd = (long long)E << 52;
    k.mant = f64_to_f32_trunc(__longlong_as_double((b & 0x000FFFFFFFFFFFFFll) | 0x3FF0000000000000ll));
    return k;
}
__device__ __forceinline__ float scaled_f32(double r, const ScaleK& k) {
    long long b = __double_as_longlong(r);
    long long ex = b & 0x7FF0000000000000ll;
    if (ex == 0) return 0.0f;
    if (ex == 0x7FF0000000000000ll) return f64_to_f32_trunc(r);
    return __fmul_rn(f64_to_f32_trunc(__longlong_as_double(b + k.eadd)), k.mant);
}

// One row vector of g = round_T(r * inv) (pads of r are 0, so pads of g stay 0).
template <int DIM, class T>
__device__ __forceinline__ void scale_cast_vec(const KArgs& a, int idx, int vpr, double inv, const ScaleK& k) {
    using C = typename Tr<T>::C;
    constexpr int V = Tr<T>::V;
    const int row = idx / vpr;
    const int x = (idx - row * vpr) * V;
    const int z = DIM == 3 ? row / a.n : 0;
    const int y = row - z * a.n;
    const long long o = offs<DIM>(x, y, z, a.P, a.S);
    C v[V];
    if constexpr (sizeof(T) == 8) {
        const double2 t = __ldg(reinterpret_cast<const double2*>(a.r64 + o));
        v[0] = t.x * inv;
        v[1] = t.y * inv;
    } else {
#pragma unroll
        for (int i = 0; i < V; i += 2) {
            const double2 t = __ldg(reinterpret_cast<const double2*>(a.r64 + o + i));
            v[i] = scaled_f32(t.x, k);
            v[i + 1] = scaled_f32(t.y, k);
        }
    }
    stv(reinterpret_cast<T*>(a.dst) + o, v);
}
// g over the padded rows of the finest level, grid-stride over the row
// vectors (a small launch when it returns at once: scale-ahead steps).
template <int DIM, class T>
__device__ __forceinline__ void scale_cast_body(const KArgs& a, int cta, int ncta) {
    constexpr int V = Tr<T>::V;
    if (a.gate && a.st->phase != 0) return;
    if (a.st && a.st->g_ready) return;  // the last update already wrote g (scale-ahead)
    const int vpr = a.P / V;  // vectors per padded row
    const int rows = DIM == 3 ? a.n * a.n : a.n;
    const double inv = a.st ? a.st->inv : a.inv_explicit;
    const ScaleK k = make_scale(inv);
    for (int idx = cta * blockDim.x + threadIdx.x; idx < rows * vpr; idx += ncta * blockDim.x)
        scale_cast_vec<DIM, T>(a, idx, vpr, inv, k);
}
template <int DIM, class T>
__global__ void __launch_bounds__(256) k_scale_cast(const KArgs a) { scale_cast_body<DIM, T>(a, blockIdx.x, gridDim.x); }
template <int DIM, class T>
__global__ void __launch_bounds__(256) k_scale_cast_batch(const KItem* __restrict__ items, const int* __restrict__ cta_item) {
    const KItem& it = items[cta_item[blockIdx.x]];
    scale_cast_body<DIM, T>(it.a, blockIdx.x - it.cta_begin, it.ncta);
}

// ---------------------------------------------------------------- FP64 IR update (Alg. 2's solution and residual updates)
// S = 2d c0 - (sum of neighbours) exactly, as FP64.
template <class T> struct ExactStencil;
template <> struct ExactStencil<__half> {
    static constexpr bool kTwoTerm = false;
    // FP16 values: exact integer arithmetic in units of 2^-24 (see h_split);
    // NB = 2d neighbours, |H| < 2^26 and |L| < 2^21 so both sums are exact.
    template <int NB>
    __device__ static void sum(float c0, const float (&nb)[NB], double& s, double& s2) {
        const float MAGIC = 12582912.0f;
        HSplit q = h_split(c0);
        int H = NB * q.hi;
        float L = __fmul_rn((float)NB, q.lo);
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            HSplit t = h_split(nb[j]);
            H -= t.hi;
            L = __fsub_rn(L, t.lo);
        }
        int Li = __float_as_int(__fadd_rn(L, MAGIC)) - __float_as_int(MAGIC);
        long long Sint = ((long long)H << 18) + (long long)Li;
        s = i64_to_f64(Sint, -24);
        s2 = 0.0;
    }
};
template <class T> struct ExactStencil {
    static constexpr bool kTwoTerm = true;
    // FP32/BF16 values: double-float sum with error-free transformations of
    // S = BETA c0 - sum of nb (nb already multiplied by their weights, exactly).
    template <int NB, int BETA = NB>
    __device__ static void sum(float c0, const float (&nb)[NB], double& s, double& s2) {
        float p = __fmul_rn((float)BETA, c0);
        float e = __fmaf_rn((float)BETA, c0, -p);
        float acc = p;
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            float t, err;
            two_sum(acc, -nb[j], t, err);
            acc = t;
            e = __fadd_rn(e, err);
        }
        s = f32_to_f64(acc);
        s2 = f32_to_f64(e);
    }
};
template <> struct ExactStencil<double> {
    static constexpr bool kTwoTerm = false;
    template <int NB, int BETA = NB>
    __device__ static void sum(double c0, const double (&nb)[NB], double& s, double& s2) {
        double t = 0.0;
#pragma unroll
        for (int j = 0; j < NB; ++j) t += nb[j];
        s = fma((double)BETA, c0, -t);
        s2 = 0.0;
    }
};

// Q1 weight of neighbour offset (dx, dy, dz): 2D all 8 neighbours 1; 3D edges
// (two non-zero offsets) 2, corners 1, faces 0.  The centre is beta.
template <int DIM>
__host__ __device__ constexpr int q1_weight(int dx, int dy, int dz) {
    return (DIM == 2) ? 1 : ((dx != 0) + (dy != 0) + (dz != 0) == 2 ? 2 : ((dx != 0) + (dy != 0) + (dz != 0) == 3 ? 1 : 0));
}

__device__ __forceinline__ double to_f64(float v) { return f32_to_f64(v); }
__device__ __forceinline__ double to_f64(double v) { return v; }


// The sum of squares in FP64 (one fused multiply-add per point on the FP64
// pipe) in place of the integer-built double-float sum: fewer instructions for
// the issue-bound update.  (An FP32 sum of the squares of the scaled FP32
// values the scale-ahead path already forms was measured slower at 255^3:
// 120.6 against 112.3 us.)
struct SqAcc64 {
    double s = 0.0;
    __device__ __forceinline__ void add(double r, int) { s = fma(r, r, s); }
};


// Block reduction in a fixed order of FP64 sums of squares and max |r| keys.
__device__ __forceinline__ void write_partials(SqAcc64 sq, unsigned long long nmax, int, double* partials, int cta) {
    __shared__ double sh[32];
    __shared__ unsigned long long rm[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double v = warp_sum(sq.s);
    nmax = warp_max(nmax);
    if (lane == 0) { sh[w] = v; rm[w] = nmax; }
    __syncthreads();
    if (w == 0) {
        v = lane < nw ? sh[lane] : 0.0;
        unsigned long long m = lane < nw ? rm[lane] : 0ull;
        v = warp_sum(v);
        m = warp_max(m);
        if (lane == 0) {
            partials[2 * (long long)cta] = v;
            partials[2 * (long long)cta + 1] = __longlong_as_double((long long)m);
        }
    }
}


// Four consecutive values of a level vector (x multiple of 4), one vector load.
template <class T>
__device__ __forceinline__ void ld4(const T* p, typename Tr<T>::C (&v)[4]) {
    if constexpr (sizeof(T) == 8) {
        const double2 a = __ldg(reinterpret_cast<const double2*>(p));
        const double2 b = __ldg(reinterpret_cast<const double2*>(p + 2));
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    } else if constexpr (sizeof(T) == 4) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(p));
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    } else {
        const uint2 raw = __ldg(reinterpret_cast<const uint2*>(p));
        const unsigned wd[2] = {raw.x, raw.y};
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            float2 f;
            if constexpr (std::is_same<T, __half>::value) f = __half22float2(*reinterpret_cast<const __half2*>(&wd[k]));
            else f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&wd[k]));
            v[2 * k] = f.x; v[2 * k + 1] = f.y;
        }
    }
}

// Four consecutive values rounded to T (16-byte aligned for FP32, 8 for 16-bit types).
template <class T>
__device__ __forceinline__ void st4(T* p, const float (&v)[4]) {
    if constexpr (std::is_same<T, float>::value) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else if constexpr (std::is_same<T, __half>::value) {
        const __half2 a = __floats2half2_rn(v[0], v[1]), b = __floats2half2_rn(v[2], v[3]);
        *reinterpret_cast<uint2*>(p) = make_uint2(*reinterpret_cast<const unsigned*>(&a), *reinterpret_cast<const unsigned*>(&b));
    } else if constexpr (std::is_same<T, __nv_bfloat16>::value) {
        const __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]), b = __floats2bfloat162_rn(v[2], v[3]);
        *reinterpret_cast<uint2*>(p) = make_uint2(*reinterpret_cast<const unsigned*>(&a), *reinterpret_cast<const unsigned*>(&b));
    }
}

// One thread per 4 consecutive points of a padded row.  u and r (FP64, 32 of
// the 34-36 bytes per point) stream through coalesced 16-byte loads and
// stores; the stencil of c comes through the read-only cache as vector loads.
// FP64 instructions per point: the two fused multiply-adds of Alg. 2's solution and residual updates
// (three for FP32/BF16 corrections) and one for the sum of squares; A c is
// formed exactly with integer / FP32 instructions.  The last CTA to finish
// runs the step's finalisation.
// OP = 1: the Q1 operator (3x3(x3) neighbourhood, integer weights).
constexpr int kUpdQ = 4;
// SA = 1 (non-FP64 T; launched only with a.dst set): the scale-ahead form.  It
// writes the next step's g = cast(trunc_FP32(r 2^k)) (reading R21) and sums the
// squares of those FP32 values in FP32 per thread (scaled back by 2^-2k in
// FP64), which leaves the FP64 pipe -- the update's second roof -- with the two
// fused multiply-adds of Alg. 2's solution and residual updates.  The norm's
// relative error stays below 1e-5 (reading R11).  SA = 0: no g, FP64 squares.
template <int DIM, class T, int OP, int SA = 0>
__device__ __forceinline__ void update_body(const KArgs& a, int cta, int ncta) {
    using C = typename Tr<T>::C;
    constexpr int Q = kUpdQ;
    constexpr bool Q1 = OP == 1;
    if (a.gate && a.st->phase != 0) return;
    const int vpr = a.P / Q;
    const int rows = DIM == 3 ? a.n * a.n : a.n;
    const int total = rows * vpr;
    const int E = 0;  // (no pre-scaling: the squares are summed in FP64)
    const double alpha = a.st ? a.st->alpha : a.a_step;
    const double beta = alpha * a.h2inv;
    SqAcc64 sq;
    unsigned long long nmax = 0ull;
    // scale-ahead (Alg. 2's residual scaling of the next step, fused): g = cast(r inv_pred),
    // inv_pred a power of two; a value beyond T's range is flagged (and the
    // next step falls back to the separate scale-and-cast)
    // (a stage call without a control state passes the power of two in inv_explicit)
    constexpr bool kSA = SA == 1 && !std::is_same<T, double>::value;
    T* const gout = kSA ? reinterpret_cast<T*>(a.dst) : nullptr;
    const double inv_pred = kSA ? (a.st ? a.st->inv_pred : a.inv_explicit) : 0.0;
    int gke = 0;            // inv_pred = 2^k: FP32 biased exponent of r * 2^k = FP64 biased exponent + k - 896
    unsigned glim = ~0u;    // |FP32 bits| at which T overflows
    float sqf = 0.0f;       // kSA: FP32 sum of squares of r 2^k
    if (kSA) {
        const long long ib = __double_as_longlong(inv_pred);
        gke = (int)((ib >> 52) & 0x7FF) - 1023 - 896;
        glim = std::is_same<T, __half>::value ? 0x477FF000u : 0x7F61B1E6u;  // 65520, 3.0e38
    }
    bool gbad = false;
    // grid-stride over the row vectors: each CTA owns a fixed set, so the
    // partial sums (one per CTA) are accumulated in a fixed order
    for (int idx = cta * blockDim.x + threadIdx.x; idx < total; idx += ncta * blockDim.x) {
        const int row = idx / vpr;
        const int x = (idx - row * vpr) * Q;
        if (x >= a.n) continue;
        const int z = DIM == 3 ? row / a.n : 0;
        const int y = row - z * a.n;
        const long long o = offs<DIM>(x, y, z, a.P, a.S);
        const T* c = reinterpret_cast<const T*>(a.src) + o;
        double* up = a.u64 + o;
        double* rp = a.rw64 + o;
        // u and r are read and written once per step (streaming, evict-first in
        // L2), so that the next step's g, written here, and the levels' vectors
        // stay in L2 for the kernels that follow
        const double2 u01 = __ldcs(reinterpret_cast<const double2*>(up));
        const double2 u23 = __ldcs(reinterpret_cast<const double2*>(up + 2));
        const double2 r01 = __ldcs(reinterpret_cast<const double2*>(rp));
        const double2 r23 = __ldcs(reinterpret_cast<const double2*>(rp + 2));
        C c0[Q], ym[Q], yp[Q], zm[Q], zp[Q];
        double uu[Q] = {u01.x, u01.y, u23.x, u23.y};
        double rr[Q] = {r01.x, r01.y, r23.x, r23.y};
        if constexpr (Q1) {
            // Q1: S = beta c0 - sum_o w_o c_o over the 3x3(x3) neighbourhood, rows
            // (dy, dz) loaded with one halo value on each side
            constexpr int NR = DIM == 3 ? 9 : 3;
            constexpr int BETA = DIM == 3 ? 32 : 8;
            C rv[NR][Q + 2];
#pragma unroll
            for (int q = 0; q < NR; ++q) {
                const T* rp = c + (q % 3 - 1) * (long long)a.P + (DIM == 3 ? (q / 3 - 1) * a.S : 0LL);
                C mid[Q];
                ld4(rp, mid);
                rv[q][0] = ld1(rp - 1);
                rv[q][Q + 1] = ld1(rp + Q);
#pragma unroll
                for (int i = 0; i < Q; ++i) rv[q][i + 1] = mid[i];
            }
            constexpr int CR = DIM == 3 ? 4 : 1;  // the centre row (dy = dz = 0)
            // FP16, 3D: every loaded value is split once (h_split); the rows with one
            // non-zero (dy, dz) offset give edges at dx = +-1 (weight 2), the rows with
            // two give edges at dx = 0 (2) and corners at dx = +-1 (1):
            // W_i = 2 (A1_{i-1} + A1_{i+1}) + 2 A2_i + A2_{i-1} + A2_{i+1}, with A1 / A2 the
            // column sums of the split values over the two row groups
            int a1h[Q + 2], a2h[Q + 2];
            float a1l[Q + 2], a2l[Q + 2];
            if constexpr (DIM == 3 && std::is_same<T, __half>::value) {
#pragma unroll
                for (int j = 0; j < Q + 2; ++j) {
                    a1h[j] = a2h[j] = 0;
                    a1l[j] = a2l[j] = 0.0f;
#pragma unroll
                    for (int q = 0; q < NR; ++q) {
                        const int nz = (q % 3 != 1) + (q / 3 != 1);
                        if (nz == 0) continue;
                        const HSplit t = h_split(rv[q][j]);
                        if (nz == 1) { a1h[j] += t.hi; a1l[j] = __fadd_rn(a1l[j], t.lo); }
                        else { a2h[j] += t.hi; a2l[j] = __fadd_rn(a2l[j], t.lo); }
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if (x + i < a.n) {
                    const C cc = rv[CR][i + 1];
                    double s, s2 = 0.0;
                    if constexpr (DIM == 3 && std::is_same<T, __half>::value) {
                        // |lo| sums: 4 values per column and group, |.| <= 2^19; the total
                        // 32 lo_c + ... stays an integer below 2^24 (exact in FP32)
                        const HSplit m = h_split(cc);
                        const int H = BETA * m.hi - 2 * (a1h[i] + a1h[i + 2]) - 2 * a2h[i + 1] - (a2h[i] + a2h[i + 2]);
                        float L = __fmul_rn((float)BETA, m.lo);
                        L = __fmaf_rn(-2.0f, __fadd_rn(a1l[i], a1l[i + 2]), L);
                        L = __fmaf_rn(-2.0f, a2l[i + 1], L);
                        L = __fsub_rn(L, __fadd_rn(a2l[i], a2l[i + 2]));
                        const int Li = __float2int_rn(L);
                        s = i64_to_f64(((long long)H << 18) + (long long)Li, -24);
                    } else if constexpr (std::is_same<T, __half>::value) {
                        // FP16 values as integers in units of 2^-24 (h_split): the
                        // weighted sum of the hi parts in int32 (|.| <= 64 * 2^22),
                        // of the lo parts in FP32 (integers, |.| <= 64 * 2^17 < 2^24)
                        HSplit m = h_split(cc);
                        int H = BETA * m.hi;
                        float L = __fmul_rn((float)BETA, m.lo);
#pragma unroll
                        for (int q = 0; q < NR; ++q)
#pragma unroll
                            for (int dx = -1; dx <= 1; ++dx) {
                                const int dy = q % 3 - 1, dz = DIM == 3 ? q / 3 - 1 : 0;
                                if (dx == 0 && dy == 0 && dz == 0) continue;
                                const int w = q1_weight<DIM>(dx, dy, dz);
                                if (w == 0) continue;
                                const HSplit t = h_split(rv[q][i + 1 + dx]);
                                H -= w * t.hi;
                                L = __fmaf_rn(-(float)w, t.lo, L);
                            }
                        const int Li = __float2int_rn(L);
                        s = i64_to_f64(((long long)H << 18) + (long long)Li, -24);
                    } else {
                        constexpr int NB = DIM == 3 ? 20 : 8;
                        C nb[NB];
                        int j = 0;
#pragma unroll
                        for (int q = 0; q < NR; ++q)
#pragma unroll
                            for (int dx = -1; dx <= 1; ++dx) {
                                const int dy = q % 3 - 1, dz = DIM == 3 ? q / 3 - 1 : 0;
                                if (dx == 0 && dy == 0 && dz == 0) continue;
                                const int w = q1_weight<DIM>(dx, dy, dz);
                                if (w == 0) continue;
                                nb[j++] = (C)w * rv[q][i + 1 + dx];  // exact: w is 1 or 2
                            }
                        ExactStencil<T>::template sum<NB, BETA>(cc, nb, s, s2);
                    }
                    double r = fma(-beta, s, rr[i]);
                    if (ExactStencil<T>::kTwoTerm && !std::is_same<T, __half>::value) r = fma(-beta, s2, r);
                    rr[i] = r;
                    uu[i] = fma(alpha, to_f64(cc), uu[i]);
                    if constexpr (!kSA) sq.add(r, E);
                    nmax = key_max(nmax, abs_key(r));
                }
            }
        } else {
        ld4(c, c0);
        ld4(c - a.P, ym);
        ld4(c + a.P, yp);
        if (DIM == 3) {
            ld4(c - a.S, zm);
            ld4(c + a.S, zp);
        }
        const C left = ld1(c - 1), right = ld1(c + Q);
        if constexpr (DIM == 3 && std::is_same<T, __half>::value) {
            // FP16 corrections: every loaded value is split once (22 splits
            // for 4 points), the exact stencil sum S = 6 c0 - sum of neighbours
            // is then an integer sum of the hi parts and an exact FP32 sum of
            // the lo parts (|lo| <= 2^17, six of them < 2^21)
            HSplit h0[Q + 2], hy[Q], hz[Q];
            h0[0] = h_split(left);
            h0[Q + 1] = h_split(right);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                h0[i + 1] = h_split(c0[i]);
                const HSplit a1 = h_split(ym[i]), a2 = h_split(yp[i]), a3 = h_split(zm[i]), a4 = h_split(zp[i]);
                hy[i].hi = a1.hi + a2.hi + a3.hi + a4.hi;
                hy[i].lo = __fadd_rn(__fadd_rn(a1.lo, a2.lo), __fadd_rn(a3.lo, a4.lo));
            }
            const int active = min(Q, a.n - x);  // points of the vector inside the row
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if (i < active) {
                    const HSplit& m = h0[i + 1];
                    const int H = 6 * m.hi - (h0[i].hi + h0[i + 2].hi) - hy[i].hi;
                    const float L = __fmaf_rn(6.0f, m.lo, -__fadd_rn(__fadd_rn(h0[i].lo, h0[i + 2].lo), hy[i].lo));
                    const float MAGIC = 12582912.0f;
                    const int Li = __float_as_int(__fadd_rn(L, MAGIC)) - __float_as_int(MAGIC);
                    const double sx = i64_to_f64(((long long)H << 18) + (long long)Li, -24);
                    const double r = fma(-beta, sx, rr[i]);
                    rr[i] = r;
                    uu[i] = fma(alpha, half_to_f64(c0[i]), uu[i]);
                    if constexpr (!kSA) sq.add(r, E);
                    nmax = key_max(nmax, abs_key(r));
                }
            }
        } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (x + i < a.n) {
                const C xm = i ? c0[i - 1] : left, xp = i < Q - 1 ? c0[i + 1] : right;
                double s, s2;
                if (DIM == 3) {
                    const C nb[6] = {xm, xp, ym[i], yp[i], zm[i], zp[i]};
                    ExactStencil<T>::template sum<6>(c0[i], nb, s, s2);
                } else {
                    const C nb[4] = {xm, xp, ym[i], yp[i]};
                    ExactStencil<T>::template sum<4>(c0[i], nb, s, s2);
                }
                double r = fma(-beta, s, rr[i]);
                if (ExactStencil<T>::kTwoTerm) r = fma(-beta, s2, r);
                rr[i] = r;
                uu[i] = fma(alpha, to_f64(c0[i]), uu[i]);
                if constexpr (!kSA) sq.add(r, E);
                const unsigned long long k = abs_key(r);
                nmax = key_max(nmax, k);
            }
        }
        }
        }
        __stcs(reinterpret_cast<double2*>(up), make_double2(uu[0], uu[1]));
        __stcs(reinterpret_cast<double2*>(up + 2), make_double2(uu[2], uu[3]));
        __stcs(reinterpret_cast<double2*>(rp), make_double2(rr[0], rr[1]));
        __stcs(reinterpret_cast<double2*>(rp + 2), make_double2(rr[2], rr[3]));
        if constexpr (kSA) {
            {  // pads of r are 0, so pads of g stay 0
                // r * 2^k truncated to FP32 from the bit pattern (integer
                // instructions; 0 below the FP32 normal range), then one rounding
                // to T; an exponent or value beyond T's range is flagged
                float gv[Q];
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const unsigned long long b = (unsigned long long)__double_as_longlong(rr[i]);
                    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
                    const int ein = (int)((hi >> 20) & 0x7FFu);
                    const int e = ein + gke;
                    const unsigned sign = hi & 0x80000000u;
                    const unsigned mag = ((unsigned)e << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
                    const unsigned fb = (ein != 0 && e > 0) ? (e < 255 ? mag : 0x7F800000u) : 0u;
                    gbad |= ein == 0x7FF || fb >= glim;
                    gv[i] = __uint_as_float((ein != 0 ? sign : 0u) | fb);
                    sqf = __fmaf_rn(gv[i], gv[i], sqf);  // pads of r are 0: they add nothing
                }
                st4(gout + o, gv);
            }
        }
    }
    if (kSA && a.st && __any_sync(kFull, gbad) && (threadIdx.x & 31) == 0)
        atomicExch(&const_cast<DevState*>(a.st)->gover, 1);
    if constexpr (kSA) {  // (r 2^k)^2 2^-2k: powers of two, exact
        const double ip = 1.0 / inv_pred;
        sq.s = (double)sqf * ip * ip;
    }
    write_partials(sq, nmax, E, a.partials, cta);
    if (a.fin && a.st) {
        // the last CTA to finish reduces every CTA's partials and runs the
        // step's finalisation (Alg. 2's stopping test and the next scale): no separate
        // launch.  Partials are published by a fence before the ticket.
        DevState* st = const_cast<DevState*>(a.st);
        __shared__ int last;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) last = atomicAdd(&st->fin_count, 1) == ncta - 1;
        __syncthreads();
        if (last) {
            __threadfence();
            if (threadIdx.x == 0) st->fin_count = 0;  // ready for the next step
            finalize_body(FIN_STEP, st, a.partials, ncta);
        }
    }
}
// FP16 corrections with the finite-difference operator (the benchmark's
// update): 4 CTAs of 256 threads per SM (at most 64 registers, no spills), so
// the kernel hides its DRAM latency with occupancy; the other instantiations
// need more registers and keep the compiler's choice.
template <class T, int OP>
struct UpdLB {
    static constexpr int kMinBlocks = (std::is_same<T, __half>::value && OP == 0) ? 4 : 1;
};
template <int DIM, class T, int OP, int SA = 0>
__global__ void __launch_bounds__(256, UpdLB<T, OP>::kMinBlocks) k_update(const KArgs a) {
    update_body<DIM, T, OP, SA>(a, blockIdx.x, gridDim.x);
}
template <int DIM, class T, int OP, int SA = 0>
__global__ void __launch_bounds__(256) k_update_batch(const KItem* __restrict__ items, const int* __restrict__ cta_item) {
    const KItem& it = items[cta_item[blockIdx.x]];
    update_body<DIM, T, OP, SA>(it.a, blockIdx.x - it.cta_begin, it.ncta);
}

// ---------------------------------------------------------------- prolongation (Alg. 1's prolongation and correction)
// c_fine += P c_coarse (bi/trilinear).  One thread per V consecutive fine x
// (x even) and a pair of fine rows (2j+1, 2j+2) -- and in 3D a pair of fine
// planes (2k+1, 2k+2) -- which share coarse rows j, j+1 and planes k, k+1:
// the odd row lies on coarse row j, the even one halfway to j+1.  Coarse rows
// and planes -1 and nc, and the coarse x just outside, are zero pads of the
// padded layout, so no bounds checks are needed on the coarse side.
template <int DIM, class T, class TC>
__device__ __forceinline__ void prolong_body(const KArgs& a, int cta) {
    using C = typename Tr<T>::C;
    constexpr int V = Tr<T>::V;
    constexpr int NZ = DIM == 3 ? 2 : 1;
    if (a.gate && a.st->phase != 0) return;
    const int vpr = a.P / V;
    const int np = a.nc + 1;  // pairs j = -1 .. nc-1
    const int total = DIM == 3 ? vpr * np * np : vpr * np;
    const int idx = cta * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int q = idx / vpr;
    const int x = (idx - q * vpr) * V;
    if (x >= a.n) return;
    const int jk = DIM == 3 ? q / np : 0;
    const int j = q - jk * np - 1, k = DIM == 3 ? jk - 1 : 0;
    // X[b][c]: coarse row j+b of plane k+c interpolated to the V fine x's
    const TC* cc = reinterpret_cast<const TC*>(a.coarse) + ((x >> 1) - 1);
    C X[2][NZ][V];
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int c = 0; c < NZ; ++c) {
            const TC* row = cc + (DIM == 3 ? (long long)(k + c) * a.Sc : 0LL) + (long long)(j + b) * a.Pc;
            C sv[V / 2 + 1];
#pragma unroll
            for (int m = 0; m <= V / 2; ++m) sv[m] = (C)ld1(row + m);
#pragma unroll
            for (int i = 0; i < V; ++i) X[b][c][i] = (i & 1) ? sv[(i + 1) >> 1] : (C)0.5 * (sv[i >> 1] + sv[(i >> 1) + 1]);
        }
    // a rescaled coarse level holds its values times 2^k (sc = 2^-k; exact)
    const C sc = a.cscale ? (C)__ldg(a.cscale) : (C)1;
    // all fine rows of the block are loaded before any is stored (no
    // load-after-store ordering between them)
    T* f0 = reinterpret_cast<T*>(a.dst) + x;
    T* fr[NZ][2];
    bool ok[NZ][2];
    C v[NZ][2][V];
#pragma unroll
    for (int dz = 0; dz < NZ; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const int z = DIM == 3 ? 2 * k + 1 + dz : 0, y = 2 * j + 1 + dy;
            ok[dz][dy] = y >= 0 && (DIM == 2 || z >= 0);
            fr[dz][dy] = f0 + (DIM == 3 ? (long long)(ok[dz][dy] ? z : 0) * a.S : 0LL) + (long long)(ok[dz][dy] ? y : 0) * a.P;
            if (ok[dz][dy]) ldv(fr[dz][dy], v[dz][dy]);
        }
#pragma unroll
    for (int dz = 0; dz < NZ; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            if (!ok[dz][dy]) continue;
#pragma unroll
            for (int i = 0; i < V; ++i) {
                // odd row / plane: the coarse row / plane itself; even: the mean of two
                const C pz0 = dy ? (C)0.5 * (X[0][0][i] + X[1][0][i]) : X[0][0][i];
                C p = pz0;
                if (DIM == 3) {
                    const C pz1 = dy ? (C)0.5 * (X[0][NZ - 1][i] + X[1][NZ - 1][i]) : X[0][NZ - 1][i];
                    p = dz ? (C)0.5 * (pz0 + pz1) : pz0;
                }
                v[dz][dy][i] = x + i < a.n ? v[dz][dy][i] + sc * p : (C)0;
            }
            stv(fr[dz][dy], v[dz][dy]);
        }
}

template <int DIM, class T, class TC>
__global__ void __launch_bounds__(256) k_prolong(const KArgs a) { prolong_body<DIM, T, TC>(a, blockIdx.x); }
template <int DIM, class T, class TC>
__global__ void __launch_bounds__(256) k_prolong_batch(const KItem* __restrict__ items, const int* __restrict__ cta_item) {
    const KItem& it = items[cta_item[blockIdx.x]];
    prolong_body<DIM, T, TC>(it.a, blockIdx.x - it.cta_begin);
}

}  // namespace mgi
