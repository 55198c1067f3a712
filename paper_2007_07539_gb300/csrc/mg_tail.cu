// Launches of the coarse-tail kernel (mg_tail_body.cuh): one CTA, or a
// thread-block cluster of cs CTAs started with cudaLaunchKernelEx and a
// cluster-dimension attribute.
#include <cuda_runtime.h>

#include "mg_tail.h"

namespace mgi {

// The one-CTA kernels use plain shared-memory accesses; the cluster kernels
// address the distributed shared memory.
static TailFn pick_tail(int dim, int uniform_prec, int cs) {
    if (dim == 3) return cs > 1 ? tail_kernel<3, true>(uniform_prec) : tail_kernel<3, false>(uniform_prec);
    return cs > 1 ? tail_kernel<2, true>(uniform_prec) : tail_kernel<2, false>(uniform_prec);
}
static TailBatchFn pick_tail_batch(int dim, int uniform_prec, int cs) {
    if (dim == 3)
        return cs > 1 ? tail_batch_kernel<3, true>(uniform_prec) : tail_batch_kernel<3, false>(uniform_prec);
    return cs > 1 ? tail_batch_kernel<2, true>(uniform_prec) : tail_batch_kernel<2, false>(uniform_prec);
}

// Launch attributes of a tail kernel: dynamic shared memory, and for clusters
// of more than 8 CTAs the non-portable cluster size.
template <class F>
static cudaError_t tail_attrs(F f, size_t smem, int cs) {
    if (smem > 32 * 1024) {  // 48 KB default minus the static stage chunk
        const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (cs > 8) return cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return cudaSuccess;
}

template <class F, class... Args>
static int launch_clustered(F f, int nclusters, int cs, size_t smem, cudaStream_t s, Args... args) {
    cudaError_t e = tail_attrs(f, smem, cs);
    if (e != cudaSuccess) return (int)e;
    if (cs <= 1) {
        f<<<nclusters, kTailThreads, smem, s>>>(args...);
        return (int)cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nclusters * cs));
    cfg.blockDim = dim3(kTailThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, f, args...);
    return (int)e;
}

int launch_tail_batch(int dim, int uniform_prec, const TailItem* items, int nitems, size_t smem, int cs, void* stream) {
    return launch_clustered(pick_tail_batch(dim, uniform_prec, cs), nitems, cs, smem, (cudaStream_t)stream, items, cs);
}

int launch_tail(int dim, int uniform_prec, const TailOp* prog, int nops, const double* minv, int m0,
                const DevState* st, int gate, size_t smem, int cs, void* stream, const TailOp* first) {
    TailOp f0{};
    if (first) f0 = *first;
    else f0.kind = -1;  // none: the kernel runs every stage from the staged program
    return launch_clustered(pick_tail(dim, uniform_prec, cs), 1, cs, smem, (cudaStream_t)stream, prog, nops, minv,
                            m0, st, gate, cs, f0);
}

// Whether a cluster of cs CTAs of the tail kernel with smem bytes of dynamic
// shared memory can be resident on this device (0 without a device).
int tail_cluster_ok(int dim, int uniform_prec, int cs, size_t smem) {
    const TailFn f = pick_tail(dim, uniform_prec, cs);
    if (tail_attrs(f, smem, cs) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cs);
    cfg.blockDim = dim3(kTailThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, f, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nc;
}

}  // namespace mgi
