// Coarse-tail kernel of libmgfp: the whole multigrid cycle on the coarsest
// levels (the Alg. 1 recursion below a size threshold) in one launch of one
// CTA, with every tail level held in shared memory.
//
// On small grids each stage of the cycle touches a few kilobytes, so a kernel
// per stage costs its launch latency and ramp-up, and a kernel that works
// through global memory costs an L2 round trip and a grid-wide barrier per
// stage.  Here the levels 0..T live in compact shared-memory arrays (c, t, g
// per level, n^d values each; the zero boundary is a bounds check) plus one
// residual scratch in the arithmetic type, and one CTA runs a program of
// stages -- damped Jacobi sweeps, residual, full-weighting restriction with
// the precision change, base solve, prolongation and correction -- built by
// the same schedule code as the big levels, separated by __syncthreads.  The
// program starts by loading g (and, on later W-cycle visits, c) of level T
// from its padded global array and ends by storing c back there.
// Arithmetic per level: FP32 for FP16/BF16/FP32 storage, FP64 for FP64.
#include <cuda_runtime.h>

#include "mg_compact.cuh"
#include "mg_march.cuh"
#include "mg_tail.h"

namespace mgi {

template <class T>
__device__ __forceinline__ typename Tr<T>::C sget(const unsigned char* sm, int off, int p) {
    return cget(reinterpret_cast<const T*>(sm + off), p);
}
template <class T, class V>
__device__ __forceinline__ void sput(unsigned char* sm, int off, int p, V v) {
    st1(reinterpret_cast<T*>(sm + off) + p, v);
}
// W of the operator (op 0: the 2d axis neighbours; 1: Q1) at point p of the
// array at byte offset off
template <int DIM, class T>
__device__ __forceinline__ typename Tr<T>::C nbsum(int op, const unsigned char* sm, int off, int p, int n, int i,
                                                   int j, int k) {
    return cwsum<DIM, T>(op, reinterpret_cast<const T*>(sm + off), p, n, i, j, k);
}

// ---- Jacobi family (Alg. 1 smoother; M_ZERO2 / M_ZERO1 start from c = 0)
template <int DIM, class T>
__device__ void t_sweep(const TailOp& op, unsigned char* sm) {
    using C = typename Tr<T>::C;
    const int n = op.n;
    const int N = DIM == 3 ? n * n * n : n * n;
    const C c1 = coef<C>(op.cf, 0), c2 = coef<C>(op.cf, 1), c3 = coef<C>(op.cf, 2), k2 = coef<C>(op.cf, 3);
    for (int p = threadIdx.x; p < N; p += blockDim.x) {
        int i, j, k;
        decode<DIM>(p, n, op.mn, i, j, k);
        const C c0 = sget<T>(sm, op.src, p);
        const C nb = nbsum<DIM, T>(op.op, sm, op.src, p, n, i, j, k);
        C v;
        if (op.mode == M_JACOBI) v = c1 * c0 + c2 * nb + c3 * sget<T>(sm, op.g, p);
        else if (op.mode == M_ZERO2) v = c3 * (k2 * c0 + c2 * nb);
        else v = c3 * c0;
        sput<T>(sm, op.dst, p, v);
    }
}

// ---- r = g - A c into the scratch (arithmetic type, no rounding to storage)
template <int DIM, class T>
__device__ void t_resid(const TailOp& op, unsigned char* sm) {
    using C = typename Tr<T>::C;
    const int n = op.n;
    const int N = DIM == 3 ? n * n * n : n * n;
    const C alpha = coef<C>(op.cf, 4), beta = (C)op_beta_d<DIM>(op.op);
    C* r = reinterpret_cast<C*>(sm + op.dst);
    for (int p = threadIdx.x; p < N; p += blockDim.x) {
        int i, j, k;
        decode<DIM>(p, n, op.mn, i, j, k);
        const C nb = nbsum<DIM, T>(op.op, sm, op.src, p, n, i, j, k);
        r[p] = sget<T>(sm, op.g, p) - alpha * (beta * sget<T>(sm, op.src, p) - nb);  // g - alpha (beta c - W)
    }
}

// ---- full weighting of the scratch residual onto the coarser level (cast to TC)
template <int DIM, class T, class TC>
__device__ void t_restrict(const TailOp& op, unsigned char* sm) {
    using C = typename Tr<T>::C;
    const C* r = reinterpret_cast<const C*>(sm + op.src);
    const int nf = op.n, nc = op.nc;
    const int Nc = DIM == 3 ? nc * nc * nc : nc * nc;
    for (int p = threadIdx.x; p < Nc; p += blockDim.x) {
        int I, J, K;
        decode<DIM>(p, nc, op.mnc, I, J, K);
        const int f0 = DIM == 3 ? ((2 * K) * nf + 2 * J) * nf + 2 * I : (2 * J) * nf + 2 * I;
        C s = 0;
#pragma unroll
        for (int dk = 0; dk < (DIM == 3 ? 3 : 1); ++dk) {
            C sj = 0;
#pragma unroll
            for (int dj = 0; dj < 3; ++dj) {
                const C* q = r + f0 + (DIM == 3 ? dk * nf * nf : 0) + dj * nf;
                const C si = (C)0.25 * q[0] + (C)0.5 * q[1] + (C)0.25 * q[2];
                sj += (dj == 1 ? (C)0.5 : (C)0.25) * si;
            }
            s += (DIM == 3 ? (dk == 1 ? (C)0.5 : (C)0.25) : (C)1) * sj;
        }
        if (op.sslot >= 0) reinterpret_cast<C*>(sm + op.scr2)[p] = s;
        else sput<TC>(sm, op.dst, p, s);
    }
    if (op.sslot >= 0) {
        // restriction into a rescaled FP16 level (DSH_MG, Sec. 6): the coarse
        // residual times 2^k, max-norm in [2^(rsig-1), 2^rsig), then the cast;
        // the matching prolongation multiplies by the stored 2^-k
        const C* v = reinterpret_cast<const C*>(sm + op.scr2);
        C m = 0;
        for (int p = threadIdx.x; p < Nc; p += blockDim.x) m = max(m, fabs(v[p]));
        const int k = rescale_shift<C>(block_max<C>(m), op.rsig);
        if (threadIdx.x == 0) *reinterpret_cast<double*>(sm + op.sslot) = pow2d(-k);
        const C f = std::is_same<C, double>::value ? (C)pow2d(k) : (C)pow2f(k);
        for (int p = threadIdx.x; p < Nc; p += blockDim.x) sput<TC>(sm, op.dst, p, v[p] * f);
    }
}

// ---- prolongation and correction c += P c_coarse (coarse values outside the grid are zero)
template <int DIM, class T, class TC>
__device__ void t_prolong(const TailOp& op, unsigned char* sm) {
    using C = typename Tr<T>::C;
    const int n = op.n, nc = op.nc;
    const int N = DIM == 3 ? n * n * n : n * n;
    // a rescaled coarse level holds its values times 2^k: the weights carry 2^-k
    const C sc = op.sslot >= 0 ? (C)*reinterpret_cast<const double*>(sm + op.sslot) : (C)1;
    for (int p = threadIdx.x; p < N; p += blockDim.x) {
        int i, j, k;
        decode<DIM>(p, n, op.mn, i, j, k);
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
                    s += (C)sget<TC>(sm, op.coarse, DIM == 3 ? (K * nc + J) * nc + I : J * nc + I);
                }
            }
        }
        sput<T>(sm, op.dst, p, sget<T>(sm, op.dst, p) + w * s);
    }
}

// ---- exact base solve c = A0^-1 g with the dense FP64 inverse (m = n^d)
template <int DIM, class T>
__device__ void t_coarse(const TailOp& op, unsigned char* sm, const double* minv, int m) {
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
        const double* row = minv + (long long)p * m;
        double s0 = 0.0, s1 = 0.0;
        int q = 0;
        for (; q + 2 <= m; q += 2) {
            s0 = fma(__ldg(row + q), (double)sget<T>(sm, op.g, q), s0);
            s1 = fma(__ldg(row + q + 1), (double)sget<T>(sm, op.g, q + 1), s1);
        }
        for (; q < m; ++q) s0 = fma(__ldg(row + q), (double)sget<T>(sm, op.g, q), s0);
        sput<T>(sm, op.dst, p, s0 + s1);
    }
}

// ---- base solve by conjugate gradients in the level's type (op.mode == 1);
// scratch at op.src: r and p (T), then A p (arithmetic type), 16-byte aligned
// slots of n^d * 8 bytes each
template <int DIM, class T>
__device__ void t_cg(const TailOp& op, unsigned char* sm) {
    using C = typename Tr<T>::C;
    const int N = DIM == 3 ? op.n * op.n * op.n : op.n * op.n;
    const int slot = ((N * 8 + 15) / 16) * 16;
    T* r = reinterpret_cast<T*>(sm + op.src);
    T* p = reinterpret_cast<T*>(sm + op.src + slot);
    C* q = reinterpret_cast<C*>(sm + op.src + 2 * slot);
    cg_base<DIM, T>(op.n, op.mn, op.op, coef<C>(op.cf, 4), (C)op_beta_d<DIM>(op.op),
                    reinterpret_cast<const T*>(sm + op.g), reinterpret_cast<T*>(sm + op.dst), r, p, q, op.cgtol,
                    op.cgmax);
}

template <int DIM, class T>
__device__ void t_zero(const TailOp& op, unsigned char* sm) {
    const int N = DIM == 3 ? op.n * op.n * op.n : op.n * op.n;
    T* d = reinterpret_cast<T*>(sm + op.dst);
    for (int p = threadIdx.x; p < N; p += blockDim.x) d[p] = T(0.0f);
}

// ---- padded global array <-> compact shared array (storage bits copied as is)
template <int DIM, class T>
__device__ void t_copy(const TailOp& op, unsigned char* sm, bool load) {
    const int n = op.n;
    const int N = DIM == 3 ? n * n * n : n * n;
    T* s = reinterpret_cast<T*>(sm + (load ? op.dst : op.src));
    T* g = reinterpret_cast<T*>(op.gptr);
    for (int p = threadIdx.x; p < N; p += blockDim.x) {
        int i, j, k;
        decode<DIM>(p, n, op.mn, i, j, k);
        const int o = DIM == 3 ? k * op.S + j * op.P + i : j * op.P + i;
        if (load) s[p] = g[o];
        else g[o] = s[p];
    }
}

// TU = void: any storage type per stage (mixed-precision tails); otherwise
// every stage of the program has prec == prec_c == the type TU.
template <int DIM, class T, class TU>
__device__ void run_tail_op_t(const TailOp& op, unsigned char* sm, const double* minv, int m0) {
    switch (op.kind) {
        case TK_SWEEP: t_sweep<DIM, T>(op, sm); return;
        case TK_RESID: t_resid<DIM, T>(op, sm); return;
        case TK_COARSE:
            if (op.mode == 1) t_cg<DIM, T>(op, sm);
            else t_coarse<DIM, T>(op, sm, minv, m0);
            return;
        case TK_ZERO: t_zero<DIM, T>(op, sm); return;
        case TK_LOAD: t_copy<DIM, T>(op, sm, true); return;
        case TK_STORE: t_copy<DIM, T>(op, sm, false); return;
        default: break;
    }
    if constexpr (!std::is_void<TU>::value) {
        if (op.kind == TK_RESTRICT) t_restrict<DIM, T, T>(op, sm);
        else t_prolong<DIM, T, T>(op, sm);
    } else {
        switch (op.prec_c) {  // transfers between this level (T) and the coarser one
            case MG_FP64:
                if (op.kind == TK_RESTRICT) t_restrict<DIM, T, double>(op, sm);
                else t_prolong<DIM, T, double>(op, sm);
                return;
            case MG_FP32:
                if (op.kind == TK_RESTRICT) t_restrict<DIM, T, float>(op, sm);
                else t_prolong<DIM, T, float>(op, sm);
                return;
            case MG_FP16:
                if (op.kind == TK_RESTRICT) t_restrict<DIM, T, __half>(op, sm);
                else t_prolong<DIM, T, __half>(op, sm);
                return;
            default:
                if (op.kind == TK_RESTRICT) t_restrict<DIM, T, __nv_bfloat16>(op, sm);
                else t_prolong<DIM, T, __nv_bfloat16>(op, sm);
                return;
        }
    }
}

template <int DIM, class TU>
__device__ __forceinline__ void tail_body(const TailOp* __restrict__ prog, int nops, const double* __restrict__ minv,
                                          int m0, const DevState* st, int gate) {
    if (gate && st->phase != 0) return;  // one CTA: the branch is uniform
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ TailOp chunk[kTailChunk];  // the next stages, staged once per chunk
    for (int s0 = 0; s0 < nops; s0 += kTailChunk) {
        const int cnt = min(kTailChunk, nops - s0);
        const unsigned long long* src = reinterpret_cast<const unsigned long long*>(prog + s0);
        unsigned long long* dst = reinterpret_cast<unsigned long long*>(chunk);
        for (int w = threadIdx.x; w < cnt * kTailOpWords; w += blockDim.x) dst[w] = __ldg(src + w);
        __syncthreads();
        for (int s = 0; s < cnt; ++s) {
            const TailOp& op = chunk[s];
            if constexpr (!std::is_void<TU>::value) {
                run_tail_op_t<DIM, TU, TU>(op, sm, minv, m0);
            } else {
                switch (op.prec) {
                    case MG_FP64: run_tail_op_t<DIM, double, void>(op, sm, minv, m0); break;
                    case MG_FP32: run_tail_op_t<DIM, float, void>(op, sm, minv, m0); break;
                    case MG_FP16: run_tail_op_t<DIM, __half, void>(op, sm, minv, m0); break;
                    default: run_tail_op_t<DIM, __nv_bfloat16, void>(op, sm, minv, m0); break;
                }
            }
            __syncthreads();
        }
    }
}

template <int DIM, class TU>
__global__ void __launch_bounds__(kTailThreads) k_tail(const TailOp* __restrict__ prog, int nops,
                                                        const double* __restrict__ minv, int m0,
                                                        const DevState* st, int gate) {
    tail_body<DIM, TU>(prog, nops, minv, m0, st, gate);
}
// Batched: one CTA per instance, each with its own program, base inverse and state.
template <int DIM, class TU>
__global__ void __launch_bounds__(kTailThreads) k_tail_batch(const TailItem* __restrict__ items) {
    const TailItem& it = items[blockIdx.x];
    tail_body<DIM, TU>(it.prog, it.nops, it.minv, it.m0, it.st, 1);
}

using TailFn = void (*)(const TailOp*, int, const double*, int, const DevState*, int);
using TailBatchFn = void (*)(const TailItem*);

template <int DIM>
static TailBatchFn pick_tail_batch(int uniform_prec) {
    switch (uniform_prec) {
        case MG_FP64: return &k_tail_batch<DIM, double>;
        case MG_FP32: return &k_tail_batch<DIM, float>;
        case MG_FP16: return &k_tail_batch<DIM, __half>;
        case MG_BF16: return &k_tail_batch<DIM, __nv_bfloat16>;
        default: return &k_tail_batch<DIM, void>;
    }
}

int launch_tail_batch(int dim, int uniform_prec, const TailItem* items, int nitems, size_t smem, void* stream) {
    const TailBatchFn f = dim == 3 ? pick_tail_batch<3>(uniform_prec) : pick_tail_batch<2>(uniform_prec);
    if (smem > 32 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
    }
    f<<<nitems, kTailThreads, smem, (cudaStream_t)stream>>>(items);
    return (int)cudaGetLastError();
}

template <int DIM>
static TailFn pick_tail(int uniform_prec) {
    switch (uniform_prec) {
        case MG_FP64: return &k_tail<DIM, double>;
        case MG_FP32: return &k_tail<DIM, float>;
        case MG_FP16: return &k_tail<DIM, __half>;
        case MG_BF16: return &k_tail<DIM, __nv_bfloat16>;
        default: return &k_tail<DIM, void>;
    }
}

int launch_tail(int dim, int uniform_prec, const TailOp* prog, int nops, const double* minv, int m0,
                const DevState* st, int gate, size_t smem, void* stream) {
    const TailFn f = dim == 3 ? pick_tail<3>(uniform_prec) : pick_tail<2>(uniform_prec);
    if (smem > 32 * 1024) {  // 48 KB default minus the static stage chunk
        const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
    }
    f<<<1, kTailThreads, smem, (cudaStream_t)stream>>>(prog, nops, minv, m0, st, gate);
    return (int)cudaGetLastError();
}

}  // namespace mgi
