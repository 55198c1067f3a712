// mg_residual_norms_noalloc: the FP64 residual norms ||b - A u||_2,
// ||b - A u||_inf and ||b||_2 of caller-owned contiguous device arrays,
// computed without allocating any device memory.
//
// It is for callers that must not call cudaMalloc / cudaFree at the point
// where they need the norms: for example a host application that has already
// reserved (nearly) all device memory for its own pool, or a latency-critical
// service loop where an allocation would implicitly synchronise the device and
// stall the work of other streams.  Instead of per-call buffers, the per-CTA
// partial sums live in one file-scope static __device__ array (kMaxBlocks * 4
// doubles = 2 MiB), which every device that loads this library holds until
// the process exits.
//
// Sharing rules: all calls on a device use the same array and it keeps the
// contents of the last call.  Each call writes every slot it later reads, so
// nothing has to be cleared between calls, but two calls whose kernels overlap
// on the GPU (e.g. issued on different streams) race on the array and give
// wrong norms: serialise them.  The first call on a device looks up the
// array's device address (cudaGetSymbolAddress) with that device current; make
// that first call before any stream capture is active.  The address is kept
// per device together with the identity of the CUDA context it belongs to:
// after cudaDeviceReset (a new primary context) the next call on that device
// looks the address up again, so it too should come before any capture.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "mg_device.cuh"
#include "mg_host.h"
#include "mg_noalloc.h"

namespace {

constexpr int kPointsPerBlock = 8192;
constexpr int kThreads = 256;
constexpr int kMaxBlocks = 65536;  // largest accepted n^d: 65536 * 8192 = 536,870,912 points
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_norm_scratch[kMaxBlocks * 4];

std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};  // context identity the address belongs to (0: none)

// Per-CTA partials of a fixed block of kPointsPerBlock points (contiguous
// layout, explicit boundary checks): {sum r^2, max |r| key, sum b^2, 0}.
// Fixed work per CTA and fixed-order reductions make the result independent
// of the GPU's size and scheduling.
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_resnorm_partials(int n, double h2inv, const double* __restrict__ b,
                                                               const double* __restrict__ u, long long npts,
                                                               double* __restrict__ part) {
    double sr = 0.0, sb = 0.0;
    unsigned long long mr = 0ull;
    const long long p0 = (long long)blockIdx.x * kPointsPerBlock;
    const long long p1 = p0 + kPointsPerBlock < npts ? p0 + kPointsPerBlock : npts;
    for (long long p = p0 + threadIdx.x; p < p1; p += kThreads) {
        const int i = (int)(p % n);
        const int j = (int)((p / n) % n);
        const int k = DIM == 3 ? (int)(p / ((long long)n * n)) : 0;
        const long long sy = n, sz = (long long)n * n;
        double nb = 0.0;
        if (i > 0) nb += __ldg(u + p - 1);
        if (i < n - 1) nb += __ldg(u + p + 1);
        if (j > 0) nb += __ldg(u + p - sy);
        if (j < n - 1) nb += __ldg(u + p + sy);
        if (DIM == 3) {
            if (k > 0) nb += __ldg(u + p - sz);
            if (k < n - 1) nb += __ldg(u + p + sz);
        }
        const double bv = __ldg(b + p);
        const double r = fma(-h2inv, fma(2.0 * DIM, __ldg(u + p), -nb), bv);
        sr = fma(r, r, sr);
        sb = fma(bv, bv, sb);
        const unsigned long long key = mgi::abs_key(r);
        mr = mgi::key_max(mr, key);
    }
    __shared__ double s1[kThreads / 32], s2[kThreads / 32];
    __shared__ unsigned long long s3[kThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    sr = mgi::warp_sum(sr);
    sb = mgi::warp_sum(sb);
    mr = mgi::warp_max(mr);
    if (lane == 0) { s1[w] = sr; s2[w] = sb; s3[w] = mr; }
    __syncthreads();
    if (w == 0) {
        sr = lane < kThreads / 32 ? s1[lane] : 0.0;
        sb = lane < kThreads / 32 ? s2[lane] : 0.0;
        mr = lane < kThreads / 32 ? s3[lane] : 0ull;
        sr = mgi::warp_sum(sr);
        sb = mgi::warp_sum(sb);
        mr = mgi::warp_max(mr);
        if (lane == 0) {
            double* q = part + 4LL * blockIdx.x;
            q[0] = sr;
            q[1] = __longlong_as_double((long long)mr);
            q[2] = sb;
            q[3] = 0.0;
        }
    }
}

// One CTA: fixed-order reduction of the partials into norms[0..2].
__global__ void __launch_bounds__(1024) k_resnorm_final(const double* __restrict__ part, int nblocks,
                                                        double* __restrict__ norms) {
    double sr = 0.0, sb = 0.0;
    unsigned long long mr = 0ull;
    for (int q = threadIdx.x; q < nblocks; q += blockDim.x) {
        sr += part[4LL * q];
        const unsigned long long m = (unsigned long long)__double_as_longlong(part[4LL * q + 1]);
        mr = m > mr ? m : mr;
        sb += part[4LL * q + 2];
    }
    __shared__ double s1[32], s2[32];
    __shared__ unsigned long long s3[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    sr = mgi::warp_sum(sr);
    sb = mgi::warp_sum(sb);
    mr = mgi::warp_max(mr);
    if (lane == 0) { s1[w] = sr; s2[w] = sb; s3[w] = mr; }
    __syncthreads();
    if (w == 0) {
        sr = lane < nw ? s1[lane] : 0.0;
        sb = lane < nw ? s2[lane] : 0.0;
        mr = lane < nw ? s3[lane] : 0ull;
        sr = mgi::warp_sum(sr);
        sb = mgi::warp_sum(sb);
        mr = mgi::warp_max(mr);
        if (lane == 0) {
            norms[0] = sqrt(sr);
            norms[1] = __longlong_as_double((long long)mr);
            norms[2] = sqrt(sb);
        }
    }
}

// mgi::noalloc_ptr_class of a pointer on the current device `dev`
int ptr_class(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return mgi::noalloc_ptr_class((int)a.type, a.device, dev);
}

// Unique identity of the calling thread's current CUDA context (cuCtxGetId,
// fetched through the runtime's driver entry point; never reused within the
// process), 0 if unavailable.
unsigned long long current_ctx_id() {
    using GetCur = int (*)(void**);
    using GetId = int (*)(void*, unsigned long long*);
    static GetCur get_cur = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = reinterpret_cast<GetCur>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
        cudaGetLastError();
    });
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (!get_cur || !get_id || get_cur(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

}  // namespace

extern "C" mg_status mg_residual_norms_noalloc(int32_t dim, int32_t n, const double* b, const double* u,
                                               double* norms, void* cuda_stream) {
    if (dim != 2 && dim != 3) { mgi_set_error("dim must be 2 or 3"); return MG_ERR_INVALID; }
    if (n < 1) { mgi_set_error("n must be >= 1"); return MG_ERR_INVALID; }
    if (!b || !u || !norms) { mgi_set_error("NULL argument"); return MG_ERR_INVALID; }
    const long long npts = dim == 3 ? (long long)n * n * n : (long long)n * n;
    const long long nblocks = (npts + kPointsPerBlock - 1) / kPointsPerBlock;
    if (nblocks > kMaxBlocks) {
        mgi_set_error("n^d = " + std::to_string(npts) + " points exceeds the static scratch limit of " +
                      std::to_string((long long)kMaxBlocks * kPointsPerBlock) + " points");
        return MG_ERR_INVALID;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        mgi_set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return MG_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        mgi_set_error("device ordinal " + std::to_string(dev) + " is beyond the " + std::to_string(kMaxDevices) +
                      " devices this entry point keeps scratch addresses for");
        return MG_ERR_INVALID;
    }
    const void* ptrs[3] = {b, u, norms};
    for (const void* q : ptrs) {
        const int c = ptr_class(q, dev);
        if (c == 1) { mgi_set_error("b, u and norms must be device (or managed) pointers"); return MG_ERR_INVALID; }
        if (c == 2) {
            mgi_set_error("b, u and norms must be memory of the current device " + std::to_string(dev));
            return MG_ERR_INVALID;
        }
    }
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        const unsigned long long ctx = current_ctx_id();
        if (!g_scratch_addr[dev] || ctx != g_scratch_ctx[dev]) {  // once per device (and context), that device current
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_norm_scratch);
            if (e != cudaSuccess) {
                mgi_set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
                return MG_ERR_CUDA;
            }
            g_scratch_addr[dev] = static_cast<double*>(p);
            g_scratch_ctx[dev] = ctx;
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const double h2inv = (double)(n + 1) * (double)(n + 1);
    if (dim == 3) k_resnorm_partials<3><<<(unsigned)nblocks, kThreads, 0, s>>>(n, h2inv, b, u, npts, scratch);
    else k_resnorm_partials<2><<<(unsigned)nblocks, kThreads, 0, s>>>(n, h2inv, b, u, npts, scratch);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_resnorm_final<<<1, 1024, 0, s>>>(scratch, (int)nblocks, norms);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        mgi_set_error(std::string("launch: ") + cudaGetErrorString(e));
        return MG_ERR_CUDA;
    }
    return MG_OK;
}
