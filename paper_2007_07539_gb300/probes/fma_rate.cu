// FP64 / FP32 FMA rate probe (the arithmetic roof of the FP64 refinement
// update): every thread runs K independent FMA chains for a fixed number of
// steps; rate = threads * K * steps / time over 5 timed launches after one
// warm-up.  One output write per thread keeps the work live.  Grid: 8 CTAs
// of 256 threads per SM.  Standalone (not part of libmgfp.so):
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o fma_rate fma_rate.cu && ./fma_rate
#include <cstdio>
#include <cuda_runtime.h>

template <class T, int K>
__global__ void k_fma(T* out, int iters, T a, T b) {
    T v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = fma(v[k], a, b);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) s += v[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T, int K>
double rate(int blocks, int threads, int iters) {
    T* out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) return -1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma<T, K><<<blocks, threads>>>(out, iters, (T)0.999, (T)1e-6);  // warm-up
    cudaEventRecord(e0);
    for (int r = 0; r < 5; ++r) k_fma<T, K><<<blocks, threads>>>(out, iters, (T)0.999, (T)1e-6);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaFree(out);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess) return -1;
    return 5.0 * blocks * threads * (double)K * iters / (ms * 1e-3);
}

int main() {
    int sms = 0, clk = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);  // kHz
    const int blocks = sms * 8, threads = 256;
    const double f64 = rate<double, 8>(blocks, threads, 1 << 14);
    const double f32 = rate<float, 8>(blocks, threads, 1 << 16);
    std::printf("{\"sms\": %d, \"max_clock_khz\": %d, \"fp64_fma_per_s\": %.4e, \"fp32_fma_per_s\": %.4e, "
                "\"fp64_fma_per_clk_per_sm\": %.3f, \"fp32_fma_per_clk_per_sm\": %.3f}\n",
                sms, clk, f64, f32, f64 / (sms * clk * 1e3), f32 / (sms * clk * 1e3));
    return f64 > 0 && f32 > 0 ? 0 : 1;
}
