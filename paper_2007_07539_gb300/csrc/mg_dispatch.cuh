// Kernel selection for the stencil march of one fine storage type T.
// Each mg_k_<type>.cu includes this file once and defines launch_march_<type>.
#pragma once
#include "mg_march.cuh"

namespace mgi {

using MarchFn = void (*)(KArgs);

template <int DIM, int MODE, int LD, class T, class TC>
constexpr MarchFn march_ptr() {
    if constexpr (DIM == 3) return &k_march3<MODE, LD, T, TC>;
    else return &k_march2<MODE, LD, T, TC>;
}

template <int DIM, class T, class TC>
MarchFn pick_tc(int mode, int loader) {
    if (mode == M_JACOBI && loader == L_PROLONG) return march_ptr<DIM, M_JACOBI, L_PROLONG, T, TC>();
    if (mode == M_RESTRICT && loader == L_PLAIN) return march_ptr<DIM, M_RESTRICT, L_PLAIN, T, TC>();
    return nullptr;
}

template <int DIM, class T>
MarchFn pick(int mode, int loader, int prec_c) {
    if (mode == M_JACOBI && loader == L_PLAIN) return march_ptr<DIM, M_JACOBI, L_PLAIN, T, T>();
    if (mode == M_ZERO2 && loader == L_PLAIN) return march_ptr<DIM, M_ZERO2, L_PLAIN, T, T>();
    if (mode == M_ZERO2 && loader == L_SCALED) return march_ptr<DIM, M_ZERO2, L_SCALED, T, T>();
    if (mode == M_ZERO1 && loader == L_PLAIN) return march_ptr<DIM, M_ZERO1, L_PLAIN, T, T>();
    if (mode == M_ZERO1 && loader == L_SCALED) return march_ptr<DIM, M_ZERO1, L_SCALED, T, T>();
    if (mode == M_UPDATE && loader == L_PLAIN) return march_ptr<DIM, M_UPDATE, L_PLAIN, T, T>();
    switch (prec_c) {
        case MG_FP64: return pick_tc<DIM, T, double>(mode, loader);
        case MG_FP32: return pick_tc<DIM, T, float>(mode, loader);
        case MG_FP16: return pick_tc<DIM, T, __half>(mode, loader);
        case MG_BF16: return pick_tc<DIM, T, __nv_bfloat16>(mode, loader);
    }
    return nullptr;
}

template <class T>
int launch_march_t(int dim, int mode, int loader, int prec_c, const KArgs& a, int gx, int gy, int gz,
                   int ty, size_t smem, void* stream) {
    MarchFn f = dim == 3 ? pick<3, T>(mode, loader, prec_c) : pick<2, T>(mode, loader, prec_c);
    if (!f) return (int)cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
    }
    f<<<dim3(gx, gy, gz), dim3(32, ty), smem, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

}  // namespace mgi
