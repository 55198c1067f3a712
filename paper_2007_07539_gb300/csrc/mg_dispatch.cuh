// Kernel selection for one fine storage type T.  Each mg_k_<type>.cu includes
// this file once and defines launch_kernel_<type>.
#pragma once
#include "mg_march.cuh"

namespace mgi {

using KFn = void (*)(KArgs);
using KFn3 = void (*)(KArgs, SweepMaps);  // 3D sweeps (TMA descriptors by value)
using FKB = void (*)(const KItem*, const int*);  // batched kernels over KItem work lists

// Q1 variants (mode | M_FEM): one row per warp; M_ZERO1 (c = w D^-1 g) does
// not apply the operator and shares the finite-difference kernel.
template <class T>
KFn3 pick_sweep3_q1(int mode, int prec_c, int rpw) {
    if (rpw != 1) return nullptr;
    switch (mode & M_BASE) {
        case M_JACOBI: return &k_sweep3<M_JACOBI, T, T, 1, 1>;
        case M_ZERO2: return &k_sweep3<M_ZERO2, T, T, 1, 1>;
        case M_ZERO1: return &k_sweep3<M_ZERO1, T, T, 1>;
        case M_RESTRICT:
            switch (prec_c) {
                case MG_FP64: return &k_sweep3<M_RESTRICT, T, double, 1, 1>;
                case MG_FP32: return &k_sweep3<M_RESTRICT, T, float, 1, 1>;
                case MG_FP16: return &k_sweep3<M_RESTRICT, T, __half, 1, 1>;
                case MG_BF16: return &k_sweep3<M_RESTRICT, T, __nv_bfloat16, 1, 1>;
            }
    }
    return nullptr;
}

template <class T>
KFn3 pick_sweep3(int mode, int prec_c, int rpw) {
    if (mode & M_FEM) return pick_sweep3_q1<T>(mode, prec_c, rpw);
    switch (mode) {
        case M_JACOBI: return rpw == 2 ? &k_sweep3<M_JACOBI, T, T, 2> : &k_sweep3<M_JACOBI, T, T, 1>;
        case M_ZERO2: return rpw == 2 ? &k_sweep3<M_ZERO2, T, T, 2> : &k_sweep3<M_ZERO2, T, T, 1>;
        case M_ZERO1: return rpw == 2 ? &k_sweep3<M_ZERO1, T, T, 2> : &k_sweep3<M_ZERO1, T, T, 1>;
        case M_PRE:  // one-pass pre-smoothing + residual-restriction
            if (rpw != 1) return nullptr;
            switch (prec_c) {
                case MG_FP64: return &k_pre3<T, double>;
                case MG_FP32: return &k_pre3<T, float>;
                case MG_FP16: return &k_pre3<T, __half>;
                case MG_BF16: return &k_pre3<T, __nv_bfloat16>;
            }
            return nullptr;
        case M_RESTRICT:  // one row per warp (two rows per warp measured no faster here)
            if (rpw != 1) return nullptr;
            switch (prec_c) {
                case MG_FP64: return &k_sweep3<M_RESTRICT, T, double, 1>;
                case MG_FP32: return &k_sweep3<M_RESTRICT, T, float, 1>;
                case MG_FP16: return &k_sweep3<M_RESTRICT, T, __half, 1>;
                case MG_BF16: return &k_sweep3<M_RESTRICT, T, __nv_bfloat16, 1>;
            }
    }
    return nullptr;
}

template <int DIM, class T, class TC>
KFn pick_tc(int kind, int mode) {
    if (kind == K_SWEEP && (mode & M_BASE) == M_RESTRICT && DIM == 2)
        return (mode & M_FEM) ? &k_sweep2<M_RESTRICT, T, TC, 1> : &k_sweep2<M_RESTRICT, T, TC, 0>;
    if (kind == K_PROLONG) return &k_prolong<DIM, T, TC>;
    return nullptr;
}

template <int DIM, class T>
KFn pick(int kind, int mode, int prec_c) {
    const bool q1 = (mode & M_FEM) != 0;
    if (kind == K_SWEEP && DIM == 2) {
        switch (mode & M_BASE) {
            case M_JACOBI: return q1 ? &k_sweep2<M_JACOBI, T, T, 1> : &k_sweep2<M_JACOBI, T, T, 0>;
            case M_ZERO2: return q1 ? &k_sweep2<M_ZERO2, T, T, 1> : &k_sweep2<M_ZERO2, T, T, 0>;
            case M_ZERO1: return &k_sweep2<M_ZERO1, T, T, 0>;
            default: break;
        }
    }
    if (kind == K_UPDATE) {
        if (!std::is_same<T, double>::value && (mode & M_SA))
            return q1 ? &k_update<DIM, T, 1, 1> : &k_update<DIM, T, 0, 1>;
        return q1 ? &k_update<DIM, T, 1> : &k_update<DIM, T, 0>;
    }
    if (kind == K_SCALE) return &k_scale_cast<DIM, T>;
    switch (prec_c) {
        case MG_FP64: return pick_tc<DIM, T, double>(kind, mode);
        case MG_FP32: return pick_tc<DIM, T, float>(kind, mode);
        case MG_FP16: return pick_tc<DIM, T, __half>(kind, mode);
        case MG_BF16: return pick_tc<DIM, T, __nv_bfloat16>(kind, mode);
    }
    return nullptr;
}

// The direct small-level kernels (3D, finite differences): rpw 0.
template <class T>
KFn pick_direct3(int mode, int prec_c) {
    switch (mode) {
        case M_JACOBI: return &k_dsweep3<M_JACOBI, T>;
        case M_ZERO2: return &k_dsweep3<M_ZERO2, T>;
        case M_ZERO1: return &k_dsweep3<M_ZERO1, T>;
        case M_RESTRICT:
            switch (prec_c) {
                case MG_FP64: return &k_drestrict3<T, double>;
                case MG_FP32: return &k_drestrict3<T, float>;
                case MG_FP16: return &k_drestrict3<T, __half>;
                case MG_BF16: return &k_drestrict3<T, __nv_bfloat16>;
            }
    }
    return nullptr;
}
template <class T>
FKB pick_direct3_batch(int mode, int prec_c) {
    switch (mode) {
        case M_JACOBI: return &k_dsweep3_batch<M_JACOBI, T>;
        case M_ZERO2: return &k_dsweep3_batch<M_ZERO2, T>;
        case M_ZERO1: return &k_dsweep3_batch<M_ZERO1, T>;
        case M_RESTRICT:
            switch (prec_c) {
                case MG_FP64: return &k_drestrict3_batch<T, double>;
                case MG_FP32: return &k_drestrict3_batch<T, float>;
                case MG_FP16: return &k_drestrict3_batch<T, __half>;
                case MG_BF16: return &k_drestrict3_batch<T, __nv_bfloat16>;
            }
    }
    return nullptr;
}

template <class T>
int launch_kernel_t(int dim, int kind, int mode, int prec_c, const KArgs& a, const MarchShape& s,
                    const SweepMaps* maps, void* stream) {
    if (dim == 3 && kind == K_SWEEP && s.rpw == 0) {
        KFn f = pick_direct3<T>(mode, prec_c);
        if (!f) return (int)cudaErrorInvalidValue;
        f<<<s.gx, s.tx, 0, (cudaStream_t)stream>>>(a);
        return (int)cudaGetLastError();
    }
    if (dim == 3 && kind == K_SWEEP) {
        KFn3 f3 = pick_sweep3<T>(mode, prec_c, s.rpw);
        if (!f3 || !maps) return (int)cudaErrorInvalidValue;
        if (s.smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(f3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
            if (e != cudaSuccess) return (int)e;
        }
        f3<<<dim3(s.gx, s.gy, s.gz), dim3(s.tx, s.ty), s.smem, (cudaStream_t)stream>>>(a, *maps);
        return (int)cudaGetLastError();
    }
    KFn f = dim == 3 ? pick<3, T>(kind, mode, prec_c) : pick<2, T>(kind, mode, prec_c);
    if (!f) return (int)cudaErrorInvalidValue;
    if (s.smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
        if (e != cudaSuccess) return (int)e;
    }
    f<<<dim3(s.gx, s.gy, s.gz), dim3(s.tx, s.ty), s.smem, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

// Batched launch of one step kind for many instances (3D): items is a device
// array of SweepItem (sweeps) or KItem (update, scale-cast, prolongation).
template <class T>
int launch_batch_t(int kind, int mode, int prec_c, int rpw, const void* items, const int* cta_item, int ncta, int ty,
                   size_t smem, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (kind == K_SWEEP && rpw == 0) {  // direct small-level kernels: KItem work lists
        FKB f = pick_direct3_batch<T>(mode, prec_c);
        if (!f) return (int)cudaErrorInvalidValue;
        f<<<ncta, 256, 0, st>>>(static_cast<const KItem*>(items), cta_item);
        return (int)cudaGetLastError();
    }
    if (kind == K_SWEEP) {
        using FB = void (*)(const SweepItem*, const int*);
        FB f = nullptr;
        if (mode & M_FEM) {  // Q1: one row per warp
            if (rpw != 1) return (int)cudaErrorInvalidValue;
            switch (mode & M_BASE) {
                case M_JACOBI: f = &k_sweep3_batch<M_JACOBI, T, T, 1, 1>; break;
                case M_ZERO2: f = &k_sweep3_batch<M_ZERO2, T, T, 1, 1>; break;
                case M_ZERO1: f = &k_sweep3_batch<M_ZERO1, T, T, 1>; break;
                case M_RESTRICT:
                    switch (prec_c) {
                        case MG_FP64: f = &k_sweep3_batch<M_RESTRICT, T, double, 1, 1>; break;
                        case MG_FP32: f = &k_sweep3_batch<M_RESTRICT, T, float, 1, 1>; break;
                        case MG_FP16: f = &k_sweep3_batch<M_RESTRICT, T, __half, 1, 1>; break;
                        case MG_BF16: f = &k_sweep3_batch<M_RESTRICT, T, __nv_bfloat16, 1, 1>; break;
                    }
                    break;
            }
        } else
        switch (mode) {
            case M_JACOBI: f = rpw == 2 ? &k_sweep3_batch<M_JACOBI, T, T, 2> : &k_sweep3_batch<M_JACOBI, T, T, 1>; break;
            case M_ZERO2: f = rpw == 2 ? &k_sweep3_batch<M_ZERO2, T, T, 2> : &k_sweep3_batch<M_ZERO2, T, T, 1>; break;
            case M_ZERO1: f = rpw == 2 ? &k_sweep3_batch<M_ZERO1, T, T, 2> : &k_sweep3_batch<M_ZERO1, T, T, 1>; break;
            case M_PRE:
                switch (prec_c) {
                    case MG_FP64: f = &k_pre3_batch<T, double>; break;
                    case MG_FP32: f = &k_pre3_batch<T, float>; break;
                    case MG_FP16: f = &k_pre3_batch<T, __half>; break;
                    case MG_BF16: f = &k_pre3_batch<T, __nv_bfloat16>; break;
                }
                break;
            case M_RESTRICT:
                if (rpw != 1) return (int)cudaErrorInvalidValue;
                switch (prec_c) {
                    case MG_FP64: f = &k_sweep3_batch<M_RESTRICT, T, double, 1>; break;
                    case MG_FP32: f = &k_sweep3_batch<M_RESTRICT, T, float, 1>; break;
                    case MG_FP16: f = &k_sweep3_batch<M_RESTRICT, T, __half, 1>; break;
                    case MG_BF16: f = &k_sweep3_batch<M_RESTRICT, T, __nv_bfloat16, 1>; break;
                }
                break;
        }
        if (!f) return (int)cudaErrorInvalidValue;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return (int)e;
        }
        f<<<ncta, dim3(32, ty), smem, st>>>(static_cast<const SweepItem*>(items), cta_item);
        return (int)cudaGetLastError();
    }
    using FK = void (*)(const KItem*, const int*);
    FK f = nullptr;
    if (kind == K_UPDATE) {
        if (!std::is_same<T, double>::value && (mode & M_SA))
            f = (mode & M_FEM) ? &k_update_batch<3, T, 1, 1> : &k_update_batch<3, T, 0, 1>;
        else
            f = (mode & M_FEM) ? &k_update_batch<3, T, 1> : &k_update_batch<3, T, 0>;
    }
    else if (kind == K_SCALE) f = &k_scale_cast_batch<3, T>;
    else if (kind == K_PROLONG) {
        switch (prec_c) {
            case MG_FP64: f = &k_prolong_batch<3, T, double>; break;
            case MG_FP32: f = &k_prolong_batch<3, T, float>; break;
            case MG_FP16: f = &k_prolong_batch<3, T, __half>; break;
            case MG_BF16: f = &k_prolong_batch<3, T, __nv_bfloat16>; break;
        }
    }
    if (!f) return (int)cudaErrorInvalidValue;
    f<<<ncta, 256, 0, st>>>(static_cast<const KItem*>(items), cta_item);
    return (int)cudaGetLastError();
}

// CTAs of this kernel resident per SM for the given block size and dynamic
// shared memory (registers, shared memory and warp slots), 0 if unknown.
template <class F>
int occupancy_f(F f, int threads, size_t smem) {
    if (!f) return 0;
    if (smem > 48 * 1024 && cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}
template <class T>
int occupancy_t(int dim, int kind, int mode, int prec_c, int threads, size_t smem, int rpw) {
    if (dim == 3 && kind == K_SWEEP) return occupancy_f(pick_sweep3<T>(mode, prec_c, rpw), threads, smem);
    return occupancy_f(dim == 3 ? pick<3, T>(kind, mode, prec_c) : pick<2, T>(kind, mode, prec_c), threads, smem);
}

}  // namespace mgi
