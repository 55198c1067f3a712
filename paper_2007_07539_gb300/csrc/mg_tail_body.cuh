// Coarse-tail kernel of libmgfp: the whole multigrid cycle on the coarsest
// levels (the Alg. 1 recursion below a size threshold) in one launch, with
// every tail level held in shared memory -- of one CTA, or distributed over
// the CTAs of one thread-block cluster (up to 16 SMs' shared memory).
//
// On small grids each stage of the cycle touches a few kilobytes to a few
// hundred kilobytes, so a kernel per stage costs its launch latency and
// ramp-up, and a kernel that works through global memory costs an L2 round
// trip and a grid-wide barrier per stage.  Here the levels 0..T live in compact
// shared-memory arrays (c, t, g per level, n^d values each; the zero boundary
// is a bounds check) plus one residual scratch in the arithmetic type, and the
// CTA (cluster) runs a program of stages -- damped Jacobi sweeps, residual,
// full-weighting restriction with the precision change, base solve,
// prolongation and correction -- built by the same schedule code as the big
// levels, separated by a CTA (cluster) barrier.  The program starts by loading
// g (and, on later W-cycle visits, c) of level T from its padded global array
// and ends by storing c back there.
//
// Distribution over a cluster: a level of N points is cut into chunks of
// 2^sh consecutive compact points; point p lives in CTA p >> sh at local
// index p & (2^sh - 1), every array at the same byte offset in every CTA.
// A CTA computes the points it owns (stores are local) and reads neighbours
// and coarse / fine values of other CTAs through distributed shared memory.
// Each point's value is the same expression as in the single-CTA tail (sh =
// 30: one chunk), so both give the same bits.
// Arithmetic per level: FP32 for FP16/BF16/FP32 storage, FP64 for FP64.
//
// This header holds the kernel templates; each (dimension, one CTA / cluster)
// combination is instantiated in a translation unit of its own
// (mg_tail_d{2,3}_{cta,cl}.cu, compiled in parallel), and mg_tail.cu launches
// them.
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "mg_compact.cuh"
#include "mg_march.cuh"
#include "mg_tail.h"

namespace cgrp = cooperative_groups;

namespace mgi {

// This CTA's dynamic shared memory (the level arrays), addressed as shared
// memory so that local accesses are plain shared loads and stores.
extern __shared__ __align__(16) unsigned char tail_dsm[];

// The tail's view of its (distributed) shared memory.
struct TailSm {
    unsigned char* sm;            // this CTA's dynamic shared memory
    unsigned char* const* rb;     // dynamic shared memory of every CTA of the cluster (generic pointers)
    int rank;                     // this CTA's rank in the cluster (0 for a single CTA)
    int cs;                       // CTAs of the cluster (1: a single CTA, plain shared-memory accesses)
};

// value of point p of the array at byte offset off of a level with chunk shift sh
template <class T, bool CL>
__device__ __forceinline__ typename Tr<T>::C dget(const TailSm& x, int off, int sh, int p) {
    if constexpr (!CL) {
        return cget(reinterpret_cast<const T*>(tail_dsm + off), p);
    } else {
        const int r = p >> sh;
        const int q = p & ((1 << sh) - 1);
        if (r == x.rank) return cget(reinterpret_cast<const T*>(tail_dsm + off), q);
        return cget(reinterpret_cast<const T*>(x.rb[r] + off), q);
    }
}
// this CTA's element q (local index) of the array at byte offset off
template <class T>
__device__ __forceinline__ typename Tr<T>::C lget(const TailSm&, int off, int q) {
    return cget(reinterpret_cast<const T*>(tail_dsm + off), q);
}
template <class T, class V>
__device__ __forceinline__ void lput(const TailSm&, int off, int q, V v) {
    st1(reinterpret_cast<T*>(tail_dsm + off) + q, v);
}
// the points [lo, hi) of an N-point level (chunk shift sh) owned by this CTA
template <bool CL>
__device__ __forceinline__ void owned(const TailSm& x, int N, int sh, int& lo, int& hi) {
    if constexpr (!CL) {
        lo = 0;
        hi = N;
        return;
    }
    lo = min(N, x.rank << sh);
    hi = min(N, (x.rank + 1) << sh);
}
template <int DIM>
__device__ __forceinline__ int npoints(int n) { return DIM == 3 ? n * n * n : n * n; }

// ---- Jacobi family (Alg. 1 smoother; M_ZERO2 / M_ZERO1 start from c = 0)
template <int DIM, class T, bool CL>
__device__ void t_sweep(const TailOp& op, const TailSm& x) {
    using C = typename Tr<T>::C;
    const int n = op.n;
    const C c1 = coef<C>(op.cf, 0), c2 = coef<C>(op.cf, 1), c3 = coef<C>(op.cf, 2), k2 = coef<C>(op.cf, 3);
    // the stage's fields in registers: the stores below go to shared memory,
    // where the staged stage record lives too
    const int src = op.src, g = op.g, dst = op.dst, sh = op.sh, mode = op.mode, opk = op.op;
    const unsigned long long mn = op.mn;
    int lo, hi;
    owned<CL>(x, npoints<DIM>(n), sh, lo, hi);
    auto get = [&](int t) { return dget<T, CL>(x, src, sh, t); };
    for (int p = lo + threadIdx.x; p < hi; p += blockDim.x) {
        int i, j, k;
        decode<DIM>(p, n, mn, i, j, k);
        const int q = p - lo;
        const C c0 = lget<T>(x, src, q);
        const C nb = cwsum_f<DIM, C>(opk, get, p, n, i, j, k);
        C v;
        if (mode == M_JACOBI) v = c1 * c0 + c2 * nb + c3 * lget<T>(x, g, q);
        else if (mode == M_ZERO2) v = c3 * (k2 * c0 + c2 * nb);
        else v = c3 * c0;
        lput<T>(x, dst, q, v);
    }
}

// ---- r = g - A c into the scratch (arithmetic type, no rounding to storage)
template <int DIM, class T, bool CL>
__device__ void t_resid(const TailOp& op, const TailSm& x) {
    using C = typename Tr<T>::C;
    const int n = op.n;
    const C alpha = coef<C>(op.cf, 4), beta = (C)op_beta_d<DIM>(op.op);
    const int src = op.src, g = op.g, sh = op.sh, opk = op.op;
    const unsigned long long mn = op.mn;
    int lo, hi;
    owned<CL>(x, npoints<DIM>(n), sh, lo, hi);
    auto get = [&](int t) { return dget<T, CL>(x, src, sh, t); };
    C* r = reinterpret_cast<C*>(tail_dsm + op.dst);
    for (int p = lo + threadIdx.x; p < hi; p += blockDim.x) {
        int i, j, k;
        decode<DIM>(p, n, mn, i, j, k);
        const int q = p - lo;
        const C nb = cwsum_f<DIM, C>(opk, get, p, n, i, j, k);
        r[q] = lget<T>(x, g, q) - alpha * (beta * lget<T>(x, src, q) - nb);  // g - alpha (beta c - W)
    }
}

// ---- full weighting of the scratch residual onto the coarser level (cast to TC)
template <int DIM, class T, class TC, bool CL>
__device__ void t_restrict(const TailOp& op, const TailSm& x) {
    using C = typename Tr<T>::C;
    const int nf = op.n, nc = op.nc;
    const int Nc = npoints<DIM>(nc);
    const int src = op.src, sh = op.sh, dst = op.dst, sslot = op.sslot;
    const unsigned long long mnc = op.mnc;
    int lo, hi;
    owned<CL>(x, Nc, op.shc, lo, hi);
    for (int p = lo + threadIdx.x; p < hi; p += blockDim.x) {
        int I, J, K;
        decode<DIM>(p, nc, mnc, I, J, K);
        const int f0 = DIM == 3 ? ((2 * K) * nf + 2 * J) * nf + 2 * I : (2 * J) * nf + 2 * I;
        C s = 0;
#pragma unroll
        for (int dk = 0; dk < (DIM == 3 ? 3 : 1); ++dk) {
            C sj = 0;
#pragma unroll
            for (int dj = 0; dj < 3; ++dj) {
                const int f = f0 + (DIM == 3 ? dk * nf * nf : 0) + dj * nf;
                const C si = (C)0.25 * dget<C, CL>(x, src, sh, f) + (C)0.5 * dget<C, CL>(x, src, sh, f + 1) +
                             (C)0.25 * dget<C, CL>(x, src, sh, f + 2);
                sj += (dj == 1 ? (C)0.5 : (C)0.25) * si;
            }
            s += (DIM == 3 ? (dk == 1 ? (C)0.5 : (C)0.25) : (C)1) * sj;
        }
        if (sslot >= 0) reinterpret_cast<C*>(tail_dsm + op.scr2)[p] = s;  // single CTA only
        else lput<TC>(x, dst, p - lo, s);
    }
    if (op.sslot >= 0) {
        // restriction into a rescaled FP16 level (DSH_MG, Sec. 6; single-CTA
        // tails only): the coarse residual times 2^k, max-norm in
        // [2^(rsig-1), 2^rsig), then the cast; the matching prolongation
        // multiplies by the stored 2^-k
        const C* v = reinterpret_cast<const C*>(tail_dsm + op.scr2);
        C m = 0;
        for (int p = threadIdx.x; p < Nc; p += blockDim.x) m = max(m, fabs(v[p]));
        const int k = rescale_shift<C>(block_max<C>(m), op.rsig);
        if (threadIdx.x == 0) *reinterpret_cast<double*>(tail_dsm + op.sslot) = pow2d(-k);
        const C f = std::is_same<C, double>::value ? (C)pow2d(k) : (C)pow2f(k);
        for (int p = threadIdx.x; p < Nc; p += blockDim.x) lput<TC>(x, op.dst, p, v[p] * f);
    }
}

// ---- prolongation and correction c += P c_coarse (coarse values outside the grid are zero)
template <int DIM, class T, class TC, bool CL>
__device__ void t_prolong(const TailOp& op, const TailSm& x) {
    using C = typename Tr<T>::C;
    const int n = op.n, nc = op.nc;
    // a rescaled coarse level holds its values times 2^k: the weights carry 2^-k
    const C sc = op.sslot >= 0 ? (C)*reinterpret_cast<const double*>(tail_dsm + op.sslot) : (C)1;
    const int coarse = op.coarse, shc = op.shc, dst = op.dst;
    const unsigned long long mn = op.mn;
    int lo, hi;
    owned<CL>(x, npoints<DIM>(n), op.sh, lo, hi);
    for (int p = lo + threadIdx.x; p < hi; p += blockDim.x) {
        int i, j, k;
        decode<DIM>(p, n, mn, i, j, k);
        // fine i = 2I + 1 sits on coarse I; even i lies between coarse i/2 - 1 and i/2
        const int il = (i - 1) >> 1, ih = i >> 1;  // equal for odd i
        const int jl = (j - 1) >> 1, jh = j >> 1;
        const int kl = DIM == 3 ? (k - 1) >> 1 : 0, kh = DIM == 3 ? k >> 1 : 0;
        C w = sc;
        if (!(i & 1)) w *= (C)0.5;
        if (!(j & 1)) w *= (C)0.5;
        if (DIM == 3 && !(k & 1)) w *= (C)0.5;
        C s = 0;
#pragma unroll
        for (int a = 0; a < (DIM == 3 ? 2 : 1); ++a) {
            const int K = a ? kh : kl;
            if (DIM == 3 && (K < 0 || K >= nc || (a && kh == kl))) continue;
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int J = b ? jh : jl;
                if (J < 0 || J >= nc || (b && jh == jl)) continue;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int I = c ? ih : il;
                    if (I < 0 || I >= nc || (c && ih == il)) continue;
                    s += (C)dget<TC, CL>(x, coarse, shc, DIM == 3 ? (K * nc + J) * nc + I : J * nc + I);
                }
            }
        }
        const int q = p - lo;
        lput<T>(x, dst, q, lget<T>(x, dst, q) + w * s);
    }
}

// ---- exact base solve c = A0^-1 g with the dense FP64 inverse (m = n^d)
// One warp per row: lane l sums the products of columns l, l+32, ... in order,
// then lane 0 takes the lanes' sums by a fixed shuffle tree (deterministic) --
// the row's loads are in flight together and the FP64 chain is short, where a
// thread per row waited on a chain of m/2 dependent FMAs.
template <int DIM, class T, bool CL>
__device__ void t_coarse(const TailOp& op, const TailSm& x, const double* minv, int m) {
    int lo, hi;
    owned<CL>(x, m, op.sh, lo, hi);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int p = lo + wid; p < hi; p += nw) {
        const double* row = minv + (long long)p * m;
        double s = 0.0;
        for (int q = lane; q < m; q += 32) s = fma(__ldg(row + q), (double)dget<T, CL>(x, op.g, op.sh, q), s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(kFull, s, o);
        if (lane == 0) lput<T>(x, op.dst, p - lo, s);
    }
}

// ---- base solve by conjugate gradients in the level's type (op.mode == 1;
// single-CTA tails only); scratch at op.src: r and p (T), then A p
// (arithmetic type), 16-byte aligned slots of n^d * 8 bytes each
template <int DIM, class T, bool CL>
__device__ void t_cg(const TailOp& op, const TailSm& x) {
    using C = typename Tr<T>::C;
    const int N = npoints<DIM>(op.n);
    const int slot = ((N * 8 + 15) / 16) * 16;
    unsigned char* sm = tail_dsm;
    T* r = reinterpret_cast<T*>(sm + op.src);
    T* p = reinterpret_cast<T*>(sm + op.src + slot);
    C* q = reinterpret_cast<C*>(sm + op.src + 2 * slot);
    cg_base<DIM, T>(op.n, op.mn, op.op, coef<C>(op.cf, 4), (C)op_beta_d<DIM>(op.op),
                    reinterpret_cast<const T*>(sm + op.g), reinterpret_cast<T*>(sm + op.dst), r, p, q, op.cgtol,
                    op.cgmax);
}

template <int DIM, class T, bool CL>
__device__ void t_zero(const TailOp& op, const TailSm& x) {
    int lo, hi;
    owned<CL>(x, npoints<DIM>(op.n), op.sh, lo, hi);
    T* d = reinterpret_cast<T*>(tail_dsm + op.dst);
    for (int p = lo + threadIdx.x; p < hi; p += blockDim.x) d[p - lo] = T(0.0f);
}

// ---- padded global array <-> compact shared array (storage bits copied as is)
template <int DIM, class T, bool CL>
__device__ void t_copy(const TailOp& op, const TailSm& x, bool load) {
    const int n = op.n;
    int lo, hi;
    owned<CL>(x, npoints<DIM>(n), op.sh, lo, hi);
    T* s = reinterpret_cast<T*>(tail_dsm + (load ? op.dst : op.src));
    T* g = reinterpret_cast<T*>(op.gptr);
#pragma unroll 4
    for (int p = lo + threadIdx.x; p < hi; p += blockDim.x) {
        int i, j, k;
        decode<DIM>(p, n, op.mn, i, j, k);
        const int o = DIM == 3 ? k * op.S + j * op.P + i : j * op.P + i;
        if (load) s[p - lo] = g[o];
        else g[o] = s[p - lo];
    }
}

// TU = void: any storage type per stage (mixed-precision tails); otherwise
// every stage of the program has prec == prec_c == the type TU.
template <int DIM, class T, class TU, bool CL>
__device__ void run_tail_op_t(const TailOp& op, const TailSm& sm, const double* minv, int m0) {
    switch (op.kind) {
        case TK_SWEEP: t_sweep<DIM, T, CL>(op, sm); return;
        case TK_RESID: t_resid<DIM, T, CL>(op, sm); return;
        case TK_COARSE:
            if (op.mode == 1) t_cg<DIM, T, CL>(op, sm);
            else t_coarse<DIM, T, CL>(op, sm, minv, m0);
            return;
        case TK_ZERO: t_zero<DIM, T, CL>(op, sm); return;
        case TK_LOAD: t_copy<DIM, T, CL>(op, sm, true); return;
        case TK_STORE: t_copy<DIM, T, CL>(op, sm, false); return;
        default: break;
    }
    if constexpr (!std::is_void<TU>::value) {
        if (op.kind == TK_RESTRICT) t_restrict<DIM, T, T, CL>(op, sm);
        else t_prolong<DIM, T, T, CL>(op, sm);
    } else {
        switch (op.prec_c) {  // transfers between this level (T) and the coarser one
            case MG_FP64:
                if (op.kind == TK_RESTRICT) t_restrict<DIM, T, double, CL>(op, sm);
                else t_prolong<DIM, T, double, CL>(op, sm);
                return;
            case MG_FP32:
                if (op.kind == TK_RESTRICT) t_restrict<DIM, T, float, CL>(op, sm);
                else t_prolong<DIM, T, float, CL>(op, sm);
                return;
            case MG_FP16:
                if (op.kind == TK_RESTRICT) t_restrict<DIM, T, __half, CL>(op, sm);
                else t_prolong<DIM, T, __half, CL>(op, sm);
                return;
            default:
                if (op.kind == TK_RESTRICT) t_restrict<DIM, T, __nv_bfloat16, CL>(op, sm);
                else t_prolong<DIM, T, __nv_bfloat16, CL>(op, sm);
                return;
        }
    }
}

template <int DIM, class TU, bool CL>
__device__ __forceinline__ void tail_body(const TailOp* __restrict__ prog, int nops, const double* __restrict__ minv,
                                          int m0, const DevState* st, int gate, int cs, const TailOp* first) {
    // gate: every CTA of the cluster reads the same state (written before the
    // launch), so all of them return here or none
    if (gate && st->phase != 0) return;
    // the base solve's dense inverse, read row by row by a few threads late in
    // the program: fetched into this SM's L1 now, while the first stages run
    // (at most 512 KB; only the matrix's own lines)
    if (minv && m0 > 0) {
        const long long lines = ((long long)m0 * m0 * 8 + 127) / 128;
        for (long long l = threadIdx.x; l < lines && l < 4096; l += blockDim.x)
            asm volatile("prefetch.global.L1 [%0];" ::"l"(reinterpret_cast<const char*>(minv) + l * 128));
    }
    unsigned char* sm = tail_dsm;
    __shared__ TailOp chunk[kTailChunk];             // the next stages, staged once per chunk
    __shared__ unsigned char* rbase[kTailMaxCluster];  // every CTA's dynamic shared memory
    TailSm x;
    x.sm = sm;
    x.rb = rbase;
    x.rank = 0;
    x.cs = cs;
    if constexpr (CL) {
        cgrp::cluster_group cl = cgrp::this_cluster();
        x.rank = (int)cl.block_rank();
        if ((int)threadIdx.x < cs) rbase[threadIdx.x] = static_cast<unsigned char*>(cl.map_shared_rank((void*)sm, threadIdx.x));
        cl.sync();  // every CTA of the cluster is running (its shared memory exists) before remote reads
    } else {
        rbase[0] = sm;
        __syncthreads();
    }
    auto run = [&](const TailOp& op) {
        if constexpr (!std::is_void<TU>::value) {
            run_tail_op_t<DIM, TU, TU, CL>(op, x, minv, m0);
        } else {
            switch (op.prec) {
                case MG_FP64: run_tail_op_t<DIM, double, void, CL>(op, x, minv, m0); break;
                case MG_FP32: run_tail_op_t<DIM, float, void, CL>(op, x, minv, m0); break;
                case MG_FP16: run_tail_op_t<DIM, __half, void, CL>(op, x, minv, m0); break;
                default: run_tail_op_t<DIM, __nv_bfloat16, void, CL>(op, x, minv, m0); break;
            }
        }
    };
    // A one-CTA tail runs its first stage (the load of its top level's g) from
    // the copy passed as a kernel parameter, with the program's staging: both
    // sets of global loads are in flight together, and one barrier ends both.
    const bool pre = !CL && first && first->kind == TK_LOAD && nops > 0;
    for (int s0 = 0; s0 < nops; s0 += kTailChunk) {
        const int cnt = min(kTailChunk, nops - s0);
        const unsigned long long* src = reinterpret_cast<const unsigned long long*>(prog + s0);
        unsigned long long* dst = reinterpret_cast<unsigned long long*>(chunk);
        for (int w = threadIdx.x; w < cnt * kTailOpWords; w += blockDim.x) dst[w] = __ldg(src + w);
        if (s0 == 0 && pre) run(*first);
        __syncthreads();
        for (int s = (s0 == 0 && pre) ? 1 : 0; s < cnt; ++s) {
            run(chunk[s]);
            // the stage's stores are visible to every CTA before the next stage;
            // after the last stage no CTA leaves while another may read its memory
            if constexpr (CL) cgrp::this_cluster().sync();
            else __syncthreads();
        }
    }
}

template <int DIM, class TU, bool CL>
__global__ void __launch_bounds__(kTailThreads) k_tail(const TailOp* __restrict__ prog, int nops,
                                                        const double* __restrict__ minv, int m0,
                                                        const DevState* st, int gate, int cs,
                                                        const __grid_constant__ TailOp first) {
    tail_body<DIM, TU, CL>(prog, nops, minv, m0, st, gate, cs, &first);
}
// Batched: one CTA (cluster of cs CTAs) per instance, each with its own
// program, base inverse and state.
template <int DIM, class TU, bool CL>
__global__ void __launch_bounds__(kTailThreads) k_tail_batch(const TailItem* __restrict__ items, int cs) {
    const TailItem& it = items[blockIdx.x / cs];
    tail_body<DIM, TU, CL>(it.prog, it.nops, it.minv, it.m0, it.st, 1, cs, nullptr);
}

// The kernel of one uniform tail storage type (-1: mixed precisions).
template <int DIM, bool CL>
TailFn tail_kernel(int uniform_prec) {
    switch (uniform_prec) {
        case MG_FP64: return &k_tail<DIM, double, CL>;
        case MG_FP32: return &k_tail<DIM, float, CL>;
        case MG_FP16: return &k_tail<DIM, __half, CL>;
        case MG_BF16: return &k_tail<DIM, __nv_bfloat16, CL>;
        default: return &k_tail<DIM, void, CL>;
    }
}
template <int DIM, bool CL>
TailBatchFn tail_batch_kernel(int uniform_prec) {
    switch (uniform_prec) {
        case MG_FP64: return &k_tail_batch<DIM, double, CL>;
        case MG_FP32: return &k_tail_batch<DIM, float, CL>;
        case MG_FP16: return &k_tail_batch<DIM, __half, CL>;
        case MG_BF16: return &k_tail_batch<DIM, __nv_bfloat16, CL>;
        default: return &k_tail_batch<DIM, void, CL>;
    }
}

}  // namespace mgi
