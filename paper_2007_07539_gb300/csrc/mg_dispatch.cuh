// Kernel selection for one fine storage type T.  Each mg_k_<type>.cu includes
// this file once and defines launch_kernel_<type>.
#pragma once
#include "mg_march.cuh"

namespace mgi {

using KFn = void (*)(KArgs);

template <int DIM, class T, class TC>
KFn pick_tc(int kind, int mode) {
    if (kind == K_SWEEP && mode == M_RESTRICT) return DIM == 3 ? &k_sweep3<M_RESTRICT, T, TC> : &k_sweep2<M_RESTRICT, T, TC>;
    if (kind == K_PROLONG) return &k_prolong<DIM, T, TC>;
    return nullptr;
}

template <int DIM, class T>
KFn pick(int kind, int mode, int prec_c) {
    if (kind == K_SWEEP) {
        switch (mode) {
            case M_JACOBI: return DIM == 3 ? &k_sweep3<M_JACOBI, T, T> : &k_sweep2<M_JACOBI, T, T>;
            case M_ZERO2: return DIM == 3 ? &k_sweep3<M_ZERO2, T, T> : &k_sweep2<M_ZERO2, T, T>;
            case M_ZERO1: return DIM == 3 ? &k_sweep3<M_ZERO1, T, T> : &k_sweep2<M_ZERO1, T, T>;
            default: break;
        }
    }
    if (kind == K_UPDATE) return &k_update<DIM, T>;
    if (kind == K_SCALE) return &k_scale_cast<DIM, T>;
    switch (prec_c) {
        case MG_FP64: return pick_tc<DIM, T, double>(kind, mode);
        case MG_FP32: return pick_tc<DIM, T, float>(kind, mode);
        case MG_FP16: return pick_tc<DIM, T, __half>(kind, mode);
        case MG_BF16: return pick_tc<DIM, T, __nv_bfloat16>(kind, mode);
    }
    return nullptr;
}

template <class T>
int launch_kernel_t(int dim, int kind, int mode, int prec_c, const KArgs& a, const MarchShape& s, void* stream) {
    KFn f = dim == 3 ? pick<3, T>(kind, mode, prec_c) : pick<2, T>(kind, mode, prec_c);
    if (!f) return (int)cudaErrorInvalidValue;
    if (s.smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
        if (e != cudaSuccess) return (int)e;
    }
    f<<<dim3(s.gx, s.gy, s.gz), dim3(s.tx, s.ty), s.smem, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

}  // namespace mgi
