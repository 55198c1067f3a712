// mg_axpy: y <- a x + y on device vectors of one storage type, the vector
// kernel behind the bandwidth-versus-size study of Sec. 8.2 (Fig. 6): the
// paper measures how an AXPY in FP16 (half2), FP32 (float, float2, float4)
// and FP64 reaches its bandwidth only for large vectors, which is why the
// coarse levels of a multigrid cycle run below the HBM roofline.  Here every
// type moves 16 bytes per thread per access (8 FP16 / BF16, 4 FP32 or 2 FP64
// values: the widest vector loads; FP16 arithmetic in half2 pairs, the
// others in their own type), over a grid-stride loop sized to the SM count.
#include <cuda_runtime.h>

#include <string>

#include "mg_device.cuh"
#include "mg_host.h"

namespace {

template <class T>
__global__ void __launch_bounds__(256) k_axpy(long long nvec, float a32, double a64, const uint4* __restrict__ x,
                                              uint4* __restrict__ y) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nvec; i += (long long)gridDim.x * blockDim.x) {
        const uint4 xv = __ldg(x + i);
        uint4 yv = y[i];
        if constexpr (sizeof(T) == 8) {
            double2 xd = *reinterpret_cast<const double2*>(&xv), yd = *reinterpret_cast<double2*>(&yv);
            yd.x = fma(a64, xd.x, yd.x);
            yd.y = fma(a64, xd.y, yd.y);
            yv = *reinterpret_cast<uint4*>(&yd);
        } else if constexpr (sizeof(T) == 4) {
            float4 xf = *reinterpret_cast<const float4*>(&xv), yf = *reinterpret_cast<float4*>(&yv);
            yf.x = __fmaf_rn(a32, xf.x, yf.x); yf.y = __fmaf_rn(a32, xf.y, yf.y);
            yf.z = __fmaf_rn(a32, xf.z, yf.z); yf.w = __fmaf_rn(a32, xf.w, yf.w);
            yv = *reinterpret_cast<uint4*>(&yf);
        } else if constexpr (std::is_same<T, __half>::value) {
            const __half2 ah = __float2half2_rn(a32);
            __half2* yh = reinterpret_cast<__half2*>(&yv);
            const __half2* xh = reinterpret_cast<const __half2*>(&xv);
#pragma unroll
            for (int k = 0; k < 4; ++k) yh[k] = __hfma2(ah, xh[k], yh[k]);
        } else {
            const __nv_bfloat162 ab = __float2bfloat162_rn(a32);
            __nv_bfloat162* yb = reinterpret_cast<__nv_bfloat162*>(&yv);
            const __nv_bfloat162* xb = reinterpret_cast<const __nv_bfloat162*>(&xv);
#pragma unroll
            for (int k = 0; k < 4; ++k) yb[k] = __hfma2(ab, xb[k], yb[k]);
        }
        y[i] = yv;
    }
}

}  // namespace

extern "C" mg_status mg_axpy(int32_t prec, int64_t n, double a, const void* x, void* y, void* stream) {
    if (prec < MG_FP64 || prec > MG_BF16 || n < 0 || (n > 0 && (!x || !y))) {
        mgi_set_error("mg_axpy: bad arguments");
        return MG_ERR_INVALID;
    }
    const int64_t per = 16 / (int64_t)mgi::elem_size(prec);
    if (n % per != 0 || (reinterpret_cast<uintptr_t>(x) & 15) || (reinterpret_cast<uintptr_t>(y) & 15)) {
        mgi_set_error("mg_axpy: n must be a multiple of 16 bytes of values and x, y 16-byte aligned");
        return MG_ERR_INVALID;
    }
    const long long nvec = n / per;
    if (nvec == 0) return MG_OK;
    const int threads = 256;
    const long long want = (nvec + threads - 1) / threads;
    const int blocks = (int)std::min<long long>(want, 152LL * 8);
    cudaStream_t s = (cudaStream_t)stream;
    const uint4* xv = static_cast<const uint4*>(x);
    uint4* yv = static_cast<uint4*>(y);
    switch (prec) {
        case MG_FP64: k_axpy<double><<<blocks, threads, 0, s>>>(nvec, (float)a, a, xv, yv); break;
        case MG_FP32: k_axpy<float><<<blocks, threads, 0, s>>>(nvec, (float)a, a, xv, yv); break;
        case MG_FP16: k_axpy<__half><<<blocks, threads, 0, s>>>(nvec, (float)a, a, xv, yv); break;
        default: k_axpy<__nv_bfloat16><<<blocks, threads, 0, s>>>(nvec, (float)a, a, xv, yv); break;
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        mgi_set_error(std::string("mg_axpy: ") + cudaGetErrorString(e));
        return MG_ERR_CUDA;
    }
    return MG_OK;
}
