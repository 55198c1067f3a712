// Coarse-tail kernel of libmgfp: the whole multigrid cycle on the coarsest
// levels (Alg. 1 recursion below a size threshold) in one launch.
//
// On small grids each stage of the cycle moves a few kilobytes, so separate
// kernels cost their launch latency and ramp-up, not bandwidth.  Here one
// thread-block cluster (16 CTAs, or 8) runs a program of stages -- damped
// Jacobi sweeps, residual, full-weighting restriction with the precision
// change, base solve, prolongation and correction -- that the host builds
// with the same schedule code as the big levels.  Stages are separated by
// the cluster's hardware barrier (barrier.cluster arrive.release /
// wait.acquire, which order the stage's global writes before the next
// stage's reads at cluster scope); data written by other CTAs is read at L2
// level (ld.cg), so no CTA sees a stale L1 line.  Arithmetic per level: FP32 for FP16/BF16/FP32
// storage, FP64 for FP64 storage; the residual is kept in that type in a
// scratch array between the residual and restriction stages.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "mg_march.cuh"
#include "mg_tail.h"

namespace cg = cooperative_groups;

namespace mgi {

__device__ __forceinline__ double ldcg_any(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ldcg_any(const float* p) { return __ldcg(p); }
__device__ __forceinline__ float ldcg_any(const __half* p) {
    unsigned short v = __ldcg(reinterpret_cast<const unsigned short*>(p));
    return __half2float(__ushort_as_half(v));
}
__device__ __forceinline__ float ldcg_any(const __nv_bfloat16* p) {
    unsigned short v = __ldcg(reinterpret_cast<const unsigned short*>(p));
    return __bfloat162float(__ushort_as_bfloat16(v));
}

// (i, j, k) of interior point p (x fastest); 32-bit arithmetic (tail levels
// have at most kTailMaxPoints points)
template <int DIM>
__device__ __forceinline__ void decode(int p, int n, int& i, int& j, int& k) {
    const int q = p / n;
    i = p - q * n;
    if (DIM == 3) {
        k = q / n;
        j = q - k * n;
    } else {
        j = q;
        k = 0;
    }
}

// ---- Jacobi family on one level (padded layout, pads are the zero boundary)
template <int DIM, class T>
__device__ void t_sweep(const TailOp& op, int tid, int nthr) {
    using C = typename Tr<T>::C;
    const T* c = reinterpret_cast<const T*>(op.src);
    const T* g = reinterpret_cast<const T*>(op.g);
    T* out = reinterpret_cast<T*>(op.dst);
    const C h2inv = (C)op.h2inv, om = (C)op.omega, twod = (C)(2 * DIM);
    const C c1 = (C)1 - om, c2 = om / twod, c3 = om / (twod * h2inv);
    const int N = DIM == 3 ? op.n * op.n * op.n : op.n * op.n;
#pragma unroll 4
    for (int p = tid; p < N; p += nthr) {
        int i, j, k;
        decode<DIM>(p, op.n, i, j, k);
        const long long o = offs<DIM>(i, j, k, op.P, op.S);
        const T* q = c + o;
        const C c0 = ldcg_any(q);
        C nb = ldcg_any(q - 1) + ldcg_any(q + 1) + ldcg_any(q - op.P) + ldcg_any(q + op.P);
        if (DIM == 3) nb += ldcg_any(q - op.S) + ldcg_any(q + op.S);
        C v;
        if (op.mode == M_JACOBI) v = c1 * c0 + c2 * nb + c3 * ldcg_any(g + o);
        else if (op.mode == M_ZERO2) v = c3 * (((C)2 - om) * c0 + c2 * nb);
        else v = c3 * c0;
        st1(out + o, v);
    }
}

// ---- residual r = g - A c into the contiguous scratch (arithmetic type)
template <int DIM, class T>
__device__ void t_resid(const TailOp& op, int tid, int nthr) {
    using C = typename Tr<T>::C;
    const T* c = reinterpret_cast<const T*>(op.src);
    const T* g = reinterpret_cast<const T*>(op.g);
    C* r = reinterpret_cast<C*>(op.scratch);
    const C h2inv = (C)op.h2inv, twod = (C)(2 * DIM);
    const int N = DIM == 3 ? op.n * op.n * op.n : op.n * op.n;
#pragma unroll 4
    for (int p = tid; p < N; p += nthr) {
        int i, j, k;
        decode<DIM>(p, op.n, i, j, k);
        const long long o = offs<DIM>(i, j, k, op.P, op.S);
        const T* q = c + o;
        C nb = ldcg_any(q - 1) + ldcg_any(q + 1) + ldcg_any(q - op.P) + ldcg_any(q + op.P);
        if (DIM == 3) nb += ldcg_any(q - op.S) + ldcg_any(q + op.S);
        r[p] = ldcg_any(g + o) - h2inv * (twod * ldcg_any(q) - nb);
    }
}

// ---- full weighting of the scratch residual onto the coarser level (cast to TC)
template <int DIM, class T, class TC>
__device__ void t_restrict(const TailOp& op, int tid, int nthr) {
    using C = typename Tr<T>::C;
    const C* r = reinterpret_cast<const C*>(op.scratch);
    TC* gc = reinterpret_cast<TC*>(op.dst);
    const int nf = op.n, nc = op.nc;
    const int Nc = DIM == 3 ? nc * nc * nc : nc * nc;
    const C w1[3] = {(C)0.25, (C)0.5, (C)0.25};
#pragma unroll 2
    for (int p = tid; p < Nc; p += nthr) {
        int I, J, K;
        decode<DIM>(p, nc, I, J, K);
        C s = 0;
        for (int dk = 0; dk < (DIM == 3 ? 3 : 1); ++dk)
            for (int dj = 0; dj < 3; ++dj)
                for (int di = 0; di < 3; ++di) {
                    const int fi = 2 * I + di, fj = 2 * J + dj, fk = DIM == 3 ? 2 * K + dk : 0;
                    const int f = DIM == 3 ? (fk * nf + fj) * nf + fi : fj * nf + fi;
                    s += w1[di] * w1[dj] * (DIM == 3 ? w1[dk] : (C)1) * __ldcg(r + f);
                }
        st1(gc + offs<DIM>(I, J, K, op.Pc, op.Sc), s);
    }
}

// ---- prolongation and correction c_f += P c_c
template <int DIM, class T, class TC>
__device__ void t_prolong(const TailOp& op, int tid, int nthr) {
    using C = typename Tr<T>::C;
    T* cf = reinterpret_cast<T*>(op.dst);
    const TC* cc = reinterpret_cast<const TC*>(op.coarse);
    const int N = DIM == 3 ? op.n * op.n * op.n : op.n * op.n;
#pragma unroll 4
    for (int p = tid; p < N; p += nthr) {
        int i, j, k;
        decode<DIM>(p, op.n, i, j, k);
        int Il, Ih, Jl, Jh, Kl = 0, Kh = 0;
        C w = 1;
        if (i & 1) { Il = Ih = (i - 1) >> 1; } else { Il = (i >> 1) - 1; Ih = i >> 1; w *= (C)0.5; }
        if (j & 1) { Jl = Jh = (j - 1) >> 1; } else { Jl = (j >> 1) - 1; Jh = j >> 1; w *= (C)0.5; }
        if (DIM == 3) {
            if (k & 1) { Kl = Kh = (k - 1) >> 1; } else { Kl = (k >> 1) - 1; Kh = k >> 1; w *= (C)0.5; }
        }
        C s = 0;
        for (int K = Kl; K <= Kh; ++K)
            for (int J = Jl; J <= Jh; ++J)
                for (int I = Il; I <= Ih; ++I) s += (C)ldcg_any(cc + offs<DIM>(I, J, K, op.Pc, op.Sc));
        const long long o = offs<DIM>(i, j, k, op.P, op.S);
        st1(cf + o, (C)ldcg_any(cf + o) + w * s);
    }
}

// ---- exact base solve c = A0^-1 g (dense FP64 inverse), by the cluster's
// first CTA with g staged in shared memory (m <= 4096 doubles)
template <int DIM, class T>
__device__ void t_coarse(const TailOp& op, const double* minv, int m, int rank) {
    extern __shared__ double gs[];
    if (rank != 0) return;
    const T* g = reinterpret_cast<const T*>(op.g);
    T* c = reinterpret_cast<T*>(op.dst);
    for (int q = threadIdx.x; q < m; q += blockDim.x) {
        int i, j, k;
        decode<DIM>(q, op.n, i, j, k);
        gs[q] = (double)ldcg_any(g + offs<DIM>(i, j, k, op.P, op.S));
    }
    __syncthreads();
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
        const double* row = minv + (long long)p * m;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int q = 0;
        for (; q + 4 <= m; q += 4) {
            s0 = fma(__ldg(row + q), gs[q], s0);
            s1 = fma(__ldg(row + q + 1), gs[q + 1], s1);
            s2 = fma(__ldg(row + q + 2), gs[q + 2], s2);
            s3 = fma(__ldg(row + q + 3), gs[q + 3], s3);
        }
        for (; q < m; ++q) s0 = fma(__ldg(row + q), gs[q], s0);
        int i, j, k;
        decode<DIM>(p, op.n, i, j, k);
        st1(c + offs<DIM>(i, j, k, op.P, op.S), (s0 + s1) + (s2 + s3));
    }
}

template <int DIM, class T>
__device__ void t_zero(const TailOp& op, int tid, int nthr) {
    T* c = reinterpret_cast<T*>(op.dst);
    const int N = DIM == 3 ? op.n * op.n * op.n : op.n * op.n;
#pragma unroll 4
    for (int p = tid; p < N; p += nthr) {
        int i, j, k;
        decode<DIM>(p, op.n, i, j, k);
        st1(c + offs<DIM>(i, j, k, op.P, op.S), (typename Tr<T>::C)0);
    }
}

template <int DIM, class T>
__device__ void run_tail_op_t(const TailOp& op, const double* minv, int m0, int tid, int nthr, int rank) {
    switch (op.kind) {
        case TK_SWEEP: t_sweep<DIM, T>(op, tid, nthr); return;
        case TK_RESID: t_resid<DIM, T>(op, tid, nthr); return;
        case TK_COARSE: t_coarse<DIM, T>(op, minv, m0, rank); return;
        case TK_ZERO: t_zero<DIM, T>(op, tid, nthr); return;
        default: break;
    }
    switch (op.prec_c) {  // transfers between this level (T) and the coarser one
        case MG_FP64:
            if (op.kind == TK_RESTRICT) t_restrict<DIM, T, double>(op, tid, nthr);
            else t_prolong<DIM, T, double>(op, tid, nthr);
            return;
        case MG_FP32:
            if (op.kind == TK_RESTRICT) t_restrict<DIM, T, float>(op, tid, nthr);
            else t_prolong<DIM, T, float>(op, tid, nthr);
            return;
        case MG_FP16:
            if (op.kind == TK_RESTRICT) t_restrict<DIM, T, __half>(op, tid, nthr);
            else t_prolong<DIM, T, __half>(op, tid, nthr);
            return;
        default:
            if (op.kind == TK_RESTRICT) t_restrict<DIM, T, __nv_bfloat16>(op, tid, nthr);
            else t_prolong<DIM, T, __nv_bfloat16>(op, tid, nthr);
            return;
    }
}

template <int DIM>
__global__ void __launch_bounds__(kTailThreads) k_tail(const TailOp* __restrict__ prog, int nops,
                                                        const double* __restrict__ minv, int m0,
                                                        const DevState* st, int gate) {
    // every CTA reads the same state word before any barrier, so all of them
    // take the same branch
    if (gate && st->phase != 0) return;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int tid = rank * blockDim.x + threadIdx.x;
    const int nthr = (int)cl.num_blocks() * blockDim.x;
    for (int s = 0; s < nops; ++s) {
        const TailOp op = prog[s];
        switch (op.prec) {
            case MG_FP64: run_tail_op_t<DIM, double>(op, minv, m0, tid, nthr, rank); break;
            case MG_FP32: run_tail_op_t<DIM, float>(op, minv, m0, tid, nthr, rank); break;
            case MG_FP16: run_tail_op_t<DIM, __half>(op, minv, m0, tid, nthr, rank); break;
            default: run_tail_op_t<DIM, __nv_bfloat16>(op, minv, m0, tid, nthr, rank); break;
        }
        cl.sync();  // arrive.release / wait.acquire at cluster scope
    }
}

int tail_cluster_size(int dim) {
    static int cached[4] = {0, 0, 0, 0};
    if (cached[dim]) return cached[dim];
    void (*f)(const TailOp*, int, const double*, int, const DevState*, int) = dim == 3 ? &k_tail<3> : &k_tail<2>;
    int best = 8;
    if (cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 16;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(16);
        cfg.blockDim = dim3(kTailThreads);
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, f, &cfg) == cudaSuccess && nclusters > 0) best = 16;
    }
    cudaGetLastError();
    cached[dim] = best;
    return best;
}

int launch_tail(int dim, const TailOp* prog, int nops, const double* minv, int m0, const DevState* st, int gate,
                void* stream) {
    void (*f)(const TailOp*, int, const double*, int, const DevState*, int) = dim == 3 ? &k_tail<3> : &k_tail<2>;
    const int cs = tail_cluster_size(dim);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(kTailThreads);
    cfg.dynamicSmemBytes = (size_t)m0 * sizeof(double);
    cfg.stream = (cudaStream_t)stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return (int)cudaLaunchKernelEx(&cfg, f, prog, nops, minv, m0, st, gate);
}

}  // namespace mgi
