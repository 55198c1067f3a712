// Small kernels of libmgfp: base-level solve, stand-alone prolongation,
// FP64 residual b - A u with norms, norm finalisation and the IR control
// state, and packing between the caller's contiguous layout and the padded
// device layout.  Also the launch-geometry rule of the stencil march.
#include <algorithm>
#include <cmath>
#include <cudaTypedefs.h>
#include <map>
#include <mutex>
#include <tuple>

#include "mg_compact.cuh"
#include "mg_final.cuh"
#include "mg_march.cuh"

namespace mgi {

int launch_kernel_f64(int, int, int, int, const KArgs&, const MarchShape&, const SweepMaps*, void*);
int launch_kernel_f32(int, int, int, int, const KArgs&, const MarchShape&, const SweepMaps*, void*);
int launch_kernel_f16(int, int, int, int, const KArgs&, const MarchShape&, const SweepMaps*, void*);
int launch_kernel_bf16(int, int, int, int, const KArgs&, const MarchShape&, const SweepMaps*, void*);
int occupancy_f64(int, int, int, int, int, size_t, int);
int launch_kernel_batch_f64(int, int, int, int, const void*, const int*, int, int, size_t, void*);
int launch_kernel_batch_f32(int, int, int, int, const void*, const int*, int, int, size_t, void*);
int launch_kernel_batch_f16(int, int, int, int, const void*, const int*, int, int, size_t, void*);
int launch_kernel_batch_bf16(int, int, int, int, const void*, const int*, int, int, size_t, void*);

int launch_kernel_batch(int kind, int mode, int prec, int prec_c, int rpw, const void* items, const int* cta_item,
                        int ncta, int ty, size_t smem, void* stream) {
    switch (prec) {
        case MG_FP64: return launch_kernel_batch_f64(kind, mode, prec_c, rpw, items, cta_item, ncta, ty, smem, stream);
        case MG_FP32: return launch_kernel_batch_f32(kind, mode, prec_c, rpw, items, cta_item, ncta, ty, smem, stream);
        case MG_FP16: return launch_kernel_batch_f16(kind, mode, prec_c, rpw, items, cta_item, ncta, ty, smem, stream);
        case MG_BF16: return launch_kernel_batch_bf16(kind, mode, prec_c, rpw, items, cta_item, ncta, ty, smem, stream);
    }
    return (int)cudaErrorInvalidValue;
}
int occupancy_f32(int, int, int, int, int, size_t, int);
int occupancy_f16(int, int, int, int, int, size_t, int);
int occupancy_bf16(int, int, int, int, int, size_t, int);

size_t elem_size(int prec) {
    switch (prec) {
        case MG_FP64: return 8;
        case MG_FP32: return 4;
        default: return 2;
    }
}

int launch_kernel(int dim, int kind, int mode, int prec, int prec_c, const KArgs& a, const MarchShape& s,
                  const SweepMaps* maps, void* stream) {
    switch (prec) {
        case MG_FP64: return launch_kernel_f64(dim, kind, mode, prec_c, a, s, maps, stream);
        case MG_FP32: return launch_kernel_f32(dim, kind, mode, prec_c, a, s, maps, stream);
        case MG_FP16: return launch_kernel_f16(dim, kind, mode, prec_c, a, s, maps, stream);
        case MG_BF16: return launch_kernel_bf16(dim, kind, mode, prec_c, a, s, maps, stream);
    }
    return (int)cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- autotuned tile shapes
namespace {
std::mutex g_tile_mu;
std::map<std::tuple<int, int, int, int, int>, TileChoice> g_tile;
}  // namespace
void tile_choice_set(int dim, int kind, int mode, int prec, int n, const TileChoice* c) {
    std::lock_guard<std::mutex> lk(g_tile_mu);
    const auto key = std::make_tuple(dim, kind, mode, prec, n);
    if (c) g_tile[key] = *c;
    else g_tile.erase(key);
}
bool tile_choice_get(int dim, int kind, int mode, int prec, int n, TileChoice* c) {
    std::lock_guard<std::mutex> lk(g_tile_mu);
    auto it = g_tile.find(std::make_tuple(dim, kind, mode, prec, n));
    if (it == g_tile.end()) return false;
    *c = it->second;
    return true;
}
// Sweeps per launch of a 3D level's pre-smoothing, chosen by the autotuner:
// kept with the tile shapes under the pseudo kernel kind -1 (mode = the coarse type).
void fuse_choice_set(int prec, int prec_c, int n, int fused) {
    const TileChoice c{fused, 0};
    tile_choice_set(3, -1, prec_c, prec, n, &c);
}
int fuse_choice_get(int prec, int prec_c, int n) {
    TileChoice c;
    return tile_choice_get(3, -1, prec_c, prec, n, &c) ? c.rpw : -1;
}

// Resident CTAs per SM of a kernel, from the runtime's occupancy calculator
// (cached: the answer depends only on the arguments), else from shared memory.
static int resident_ctas(int dim, int kind, int mode, int prec, int prec_c, int threads, size_t smem, int rpw = 1) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int, int, int, size_t, int>, int> cache;
    const auto key = std::make_tuple(dim, kind, mode, prec, prec_c, threads, smem, rpw);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    int nb = 0;
    switch (prec) {
        case MG_FP64: nb = occupancy_f64(dim, kind, mode, prec_c, threads, smem, rpw); break;
        case MG_FP32: nb = occupancy_f32(dim, kind, mode, prec_c, threads, smem, rpw); break;
        case MG_FP16: nb = occupancy_f16(dim, kind, mode, prec_c, threads, smem, rpw); break;
        default: nb = occupancy_bf16(dim, kind, mode, prec_c, threads, smem, rpw); break;
    }
    if (nb <= 0) nb = std::max(1, std::min(4, (int)(220 * 1024 / (smem + 1024))));
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = nb;
    return nb;
}

// ---------------------------------------------------------------- TMA descriptors
// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    });
    return fn;
}

int make_sweep_map(CUtensorMap* m, int prec, const Geom& geo, const void* x0, int rows, bool halo) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return (int)cudaErrorNotSupported;
    const size_t esz = elem_size(prec);
    const size_t ub = esz == 2 ? 4 : 8;  // bytes per unit
    const CUtensorMapDataType dt = esz == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT32 : CU_TENSOR_MAP_DATA_TYPE_UINT64;
    const cuuint64_t dims[3] = {(cuuint64_t)(geo.P * esz / ub), (cuuint64_t)geo.n + 1, (cuuint64_t)geo.n + 2};
    const cuuint64_t strides[2] = {(cuuint64_t)geo.P * esz, (cuuint64_t)geo.S * esz};
    const cuuint32_t box[3] = {(cuuint32_t)((halo ? kSweepRowBytes : 512) / ub), (cuuint32_t)rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    void* gaddr = const_cast<char*>(static_cast<const char*>(x0)) - geo.S * (long long)esz;  // plane -1
    const CUresult r = enc(m, dt, 3, gaddr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : (int)cudaErrorInvalidValue;
}

static int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }
static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

constexpr int kSMs = 152;

// Picks the march length L for `units` fine planes (rows in 2D) to march over
// in spans of L * step_mult (the restriction's CTAs take 2TK of them, for TK
// coarse planes) and `tiles` CTAs per span: each CTA also reads the two planes
// next to its range, and a grid that ends in a partial wave idles SMs, so L
// maximises  (waves / ceil(waves)) * L / (L + 2)  over L in [lo, hi].
static int pick_march_len(int units, long long tiles, int resident, int lo, int hi, int step_mult) {
    double best = -1.0;
    int bestL = lo;
    for (int L = lo; L <= hi; ++L) {
        const int span = L * step_mult;
        const long long nb = tiles * cdiv(units, span);
        const double waves = (double)nb / (double)(kSMs * resident);
        const double eff = waves / std::ceil(waves) * (double)span / (double)(span + 2);
        if (eff > best + 1e-9) { best = eff; bestL = L; }
    }
    return bestL;
}

// Launch geometry.  Sweeps (3D): CTAs of 8 warps over 8 rows (16 rows, two
// per warp, once n >= 16) of one 512-byte x-chunk, marching over z through a
// 6-stage TMA ring; restriction: 2TJ+1 fine rows per CTA (TJ coarse rows) and
// 2TK+1 fine planes per range, one fine
// row / plane shared with the neighbouring tile, x-chunks overlapping by one
// vector.  2D: one x-chunk per warp, 4 warps per CTA, marching over rows.
// Streaming kernels (update, scale-cast, prolongation): 256 threads, one
// thread per vector of a padded row.
MarchShape kernel_shape(int dim, int kind, int mode, int prec, int n, int P, int tz_hint) {
    const int V = (int)(16 / elem_size(prec));
    const int CW = 32 * V;
    const size_t cs = prec == MG_FP64 ? 8 : 4;
    const int VH = V / 2 > 0 ? V / 2 : 1;
    MarchShape s{};
    s.tx = 32;
    s.gz = 1;
    if (kind != K_SWEEP) {
        const int per = kind == K_UPDATE ? kUpdQ : V;
        // prolongation: one thread per vector of a pair of rows (and planes)
        const long long np = (n - 1) / 2 + 1;
        const long long rows = kind == K_PROLONG ? (dim == 3 ? np * np : np) : (dim == 3 ? (long long)n * n : n);
        s.tx = 256;
        s.ty = 1;
        s.gx = cdiv(rows * (P / per), 256);
        if (kind == K_UPDATE) s.gx = std::min(s.gx, 4 * kSMs);  // grid-stride: one partial per CTA
        if (kind == K_SCALE) s.gx = std::min(s.gx, 8 * kSMs);   // grid-stride
        s.gy = 1;
        s.smem = 0;
        return s;
    }
    const int bmode = mode & M_BASE;
    const bool q1 = (mode & M_FEM) != 0;  // Q1 sweeps keep one row per warp
    const bool need_g = bmode == M_JACOBI || bmode == M_RESTRICT;
    if (dim == 3 && !q1 && bmode != M_PRE) {  // small levels: the direct kernels (same results)
        TileChoice tc;
        // default: direct sweeps up to kDirectMaxN, direct restriction (one thread per coarse
        // point, latency-bound) only below that
        const bool direct = tile_choice_get(dim, kind, mode, prec, n, &tc)
                                ? tc.rpw == 0
                                : n <= (bmode == M_RESTRICT ? kDirectMaxN / 2 : kDirectMaxN);
        if (direct) {
            s.rpw = 0;
            s.tx = 256;
            s.ty = 1;
            const long long units = bmode == M_RESTRICT ? (long long)((n - 1) / 2) * ((n - 1) / 2) * ((n - 1) / 2)
                                                        : (long long)(P / V) * n * n;
            s.gx = (int)std::max<long long>(1, cdiv(units, 256));
            s.gy = 1;
            s.smem = 0;
            return s;
        }
    }
    if (bmode == M_RESTRICT || bmode == M_PRE) {
        const int nc = (n - 1) / 2;
        s.xstep = P > CW ? CW - V : CW;
        const int nchunks = P > CW ? 1 + cdiv(P - CW, CW - V) : 1;
        if (dim == 3) {
            // TJ coarse rows per CTA from 2TJ+1 fine rows, one per warp
            s.rpw = 1;
            const int TJ = clampi(nc, 1, 4);
            s.ty = 2 * TJ + 1;
            const int rows = s.ty;
            s.ystep = 2 * TJ;
            s.gx = nchunks;
            s.gy = cdiv(nc, TJ);
            s.smem = bmode == M_PRE ? (size_t)pre3_smem(rows, rows * 32 * VH * (int)cs)
                                   : (size_t)sweep3_smem(rows, true, (q1 ? 1 : 2) * rows * 32 * VH * (int)cs,
                                                         sweep3_stages(M_RESTRICT, s.rpw));
            const int res = resident_ctas(dim, kind, mode, prec, prec, s.tx * s.ty, s.smem, s.rpw);
            TileChoice tc;
            if (tz_hint <= 0 && tile_choice_get(dim, kind, mode, prec, n, &tc)) tz_hint = tc.zlen;
            int TK = tz_hint > 0 ? tz_hint : pick_march_len(2 * nc, (long long)s.gx * s.gy, res, 2, 16, 2);
            TK = clampi(TK, 1, nc);
            s.zlen = 2 * TK + 1;
            s.zstep = 2 * TK;
            s.gz = cdiv(nc, TK);
        } else {
            const int W = clampi(nchunks, 1, 4);
            s.ty = W;
            s.gx = cdiv(nchunks, W);
            s.smem = (size_t)W * 6 * 2 * kRowBytes;
            int TK = tz_hint > 0 ? tz_hint : pick_march_len(2 * nc, s.gx, 8, 4, 32, 2);
            TK = clampi(TK, 1, nc);
            s.zlen = 2 * TK + 1;
            s.zstep = 2 * TK;
            s.gy = cdiv(nc, TK);
        }
        return s;
    }
    s.xstep = CW;
    const int nchunks = cdiv(P, CW);
    if (dim == 3) {
        // two rows per warp (16-row tiles) once the level has 16 rows: the
        // per-plane work of a warp (waits, barrier, copy issue, addressing)
        // is shared by twice the points
        s.ty = clampi(n, 1, 8);
        s.rpw = n >= 16 && !q1 ? 2 : 1;
        TileChoice tc;
        const bool tuned = tile_choice_get(dim, kind, mode, prec, n, &tc);
        if (tuned) {
            s.rpw = n >= 16 && !q1 ? clampi(tc.rpw, 1, 2) : 1;
            if (tz_hint <= 0) tz_hint = tc.zlen;
        }
        s.ystep = s.ty * s.rpw;
        s.gx = nchunks;
        s.gy = cdiv(n, s.ystep);
        s.smem = (size_t)sweep3_smem(s.ystep, need_g, 0, sweep3_stages(bmode, s.rpw));
        const int res = resident_ctas(dim, kind, mode, prec, prec, s.tx * s.ty, s.smem, s.rpw);
        int zl = tz_hint > 0 ? tz_hint : pick_march_len(n, (long long)s.gx * s.gy, res, 4, 40, 1);
        zl = clampi(zl, 1, n);
        s.zlen = zl;
        s.zstep = zl;
        s.gz = cdiv(n, zl);
    } else {
        const int W = clampi(nchunks, 1, 4);
        s.ty = W;
        s.gx = cdiv(nchunks, W);
        s.smem = (size_t)W * 6 * (need_g ? 2 : 1) * kRowBytes;
        int zl = tz_hint > 0 ? tz_hint : pick_march_len(n, s.gx, 8, 4, 64, 1);
        zl = clampi(zl, 1, n);
        s.zlen = zl;
        s.zstep = zl;
        s.gy = cdiv(n, zl);
    }
    return s;
}

// ---------------------------------------------------------------- base-level solve
// c = A0^-1 g with the dense FP64 inverse computed on the host at setup
// (exact solve on the coarsest level, Sec. 4.2); accumulation in FP64, the
// result rounded to the level's storage type.
template <class T>
__global__ void k_coarse_solve(const double* __restrict__ minv, int m, const T* __restrict__ g, T* __restrict__ c,
                               int n, int P, long long S, int dim, const DevState* st, int gate) {
    if (gate && st->phase != 0) return;
    extern __shared__ double gs[];
    for (int q = threadIdx.x; q < m; q += blockDim.x) {
        int i = q % n, j = (q / n) % n, k = q / (n * n);
        long long o = (dim == 3 ? (long long)k * S : 0LL) + (long long)j * P + i;
        gs[q] = (double)ld1(g + o);
    }
    __syncthreads();
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= m) return;
    double s = 0.0;
    const double* row = minv + (long long)p * m;
    for (int q = 0; q < m; ++q) s = fma(row[q], gs[q], s);
    int i = p % n, j = (p / n) % n, k = p / (n * n);
    long long o = (dim == 3 ? (long long)k * S : 0LL) + (long long)j * P + i;
    st1(c + o, s);
}

int launch_coarse_solve(int prec, const double* inv, int m, const void* g, void* c, const Geom& geo,
                        const DevState* st, int gate, void* stream) {
    dim3 grid((m + 255) / 256), block(256);
    size_t sm = (size_t)m * sizeof(double);
    cudaStream_t s = (cudaStream_t)stream;
    switch (prec) {
        case MG_FP64:
            k_coarse_solve<double><<<grid, block, sm, s>>>(inv, m, (const double*)g, (double*)c, geo.n, geo.P, geo.S, geo.dim, st, gate);
            break;
        case MG_FP32:
            k_coarse_solve<float><<<grid, block, sm, s>>>(inv, m, (const float*)g, (float*)c, geo.n, geo.P, geo.S, geo.dim, st, gate);
            break;
        case MG_FP16:
            k_coarse_solve<__half><<<grid, block, sm, s>>>(inv, m, (const __half*)g, (__half*)c, geo.n, geo.P, geo.S, geo.dim, st, gate);
            break;
        case MG_BF16:
            k_coarse_solve<__nv_bfloat16><<<grid, block, sm, s>>>(inv, m, (const __nv_bfloat16*)g, (__nv_bfloat16*)c, geo.n, geo.P, geo.S, geo.dim, st, gate);
            break;
        default: return (int)cudaErrorInvalidValue;
    }
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------- base solve by CG
// One CTA: g is gathered from its padded array into compact shared arrays,
// cg_base runs there, and x is scattered to c.  Shared memory: A p in the
// arithmetic type, then x, g, r, p in the level type (m <= 4096 points).
template <int DIM, class T>
__global__ void __launch_bounds__(1024) k_coarse_cg(const T* __restrict__ g, T* __restrict__ c, int n, int P,
                                                    long long S, int op, double alpha, double tol, int maxit,
                                                    const DevState* st, int gate) {
    using C = typename Tr<T>::C;
    if (gate && st->phase != 0) return;
    extern __shared__ __align__(16) unsigned char smc[];
    const int m = DIM == 3 ? n * n * n : n * n;
    C* q = reinterpret_cast<C*>(smc);
    T* x = reinterpret_cast<T*>(q + m);
    T* gs = x + m;
    T* r = gs + m;
    T* p = r + m;
    const unsigned long long mn = ((1ull << 40) + (unsigned long long)n - 1) / (unsigned long long)n;
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
        int i, j, k;
        decode<DIM>(t, n, mn, i, j, k);
        gs[t] = g[(DIM == 3 ? (long long)k * S : 0LL) + (long long)j * P + i];
    }
    __syncthreads();
    cg_base<DIM, T>(n, mn, op, (C)alpha, (C)op_beta_d<DIM>(op), gs, x, r, p, q, tol, maxit);
    __syncthreads();
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
        int i, j, k;
        decode<DIM>(t, n, mn, i, j, k);
        c[(DIM == 3 ? (long long)k * S : 0LL) + (long long)j * P + i] = x[t];
    }
}

template <int DIM, class T>
static int launch_coarse_cg_t(const void* g, void* c, const Geom& geo, int op, double tol, int maxit,
                              const DevState* st, int gate, cudaStream_t s) {
    using C = typename Tr<T>::C;
    const int m = DIM == 3 ? geo.n * geo.n * geo.n : geo.n * geo.n;
    const size_t smem = (size_t)m * (sizeof(C) + 4 * sizeof(T));
    auto f = &k_coarse_cg<DIM, T>;
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
    }
    f<<<1, 1024, smem, s>>>((const T*)g, (T*)c, geo.n, geo.P, geo.S, op, op_alpha(op, DIM, geo.n), tol, maxit, st,
                            gate);
    return (int)cudaGetLastError();
}

int launch_coarse_cg(int prec, int op, const void* g, void* c, const Geom& geo, double tol, int maxit,
                     const DevState* st, int gate, void* stream) {
    const cudaStream_t s = (cudaStream_t)stream;
    const bool d3 = geo.dim == 3;
    switch (prec) {
        case MG_FP64: return d3 ? launch_coarse_cg_t<3, double>(g, c, geo, op, tol, maxit, st, gate, s)
                                : launch_coarse_cg_t<2, double>(g, c, geo, op, tol, maxit, st, gate, s);
        case MG_FP32: return d3 ? launch_coarse_cg_t<3, float>(g, c, geo, op, tol, maxit, st, gate, s)
                                : launch_coarse_cg_t<2, float>(g, c, geo, op, tol, maxit, st, gate, s);
        case MG_FP16: return d3 ? launch_coarse_cg_t<3, __half>(g, c, geo, op, tol, maxit, st, gate, s)
                                : launch_coarse_cg_t<2, __half>(g, c, geo, op, tol, maxit, st, gate, s);
        case MG_BF16: return d3 ? launch_coarse_cg_t<3, __nv_bfloat16>(g, c, geo, op, tol, maxit, st, gate, s)
                                : launch_coarse_cg_t<2, __nv_bfloat16>(g, c, geo, op, tol, maxit, st, gate, s);
    }
    return (int)cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- FP16 level rescale
// Restriction into a rescaled FP16 level (DSH_MG, Sec. 6), after the
// restriction kernel has written the coarse residual x in FP32: (1) per-CTA
// max |x| over the interior; (2) every CTA reduces those kRescaleCtas
// partials in the same order, takes the shift k of rescale_shift, and casts
// g = fp16(x 2^k) (one rounding: the product is exact); CTA 0 stores 2^-k.
template <int DIM>
__global__ void __launch_bounds__(256) k_absmax(const float* __restrict__ x, int n, int P, long long S,
                                                float* __restrict__ part, const DevState* st, int gate) {
    if (gate && st->phase != 0) return;
    const int npts = DIM == 3 ? n * n * n : n * n;
    float m = 0.0f;
    for (int oc = blockIdx.x * blockDim.x + threadIdx.x; oc < npts; oc += gridDim.x * blockDim.x) {
        const int q = oc / n;
        const int i = oc - q * n;
        const int k = DIM == 3 ? q / n : 0;
        const int j = q - k * n;
        m = fmaxf(m, fabsf(x[offs<DIM>(i, j, k, P, S)]));
    }
    m = block_max<float>(m);
    if (threadIdx.x == 0) part[blockIdx.x] = m;
}

template <int DIM>
__global__ void __launch_bounds__(256) k_rescale_cast(const float* __restrict__ x, __half* __restrict__ g, int n,
                                                      int P, long long S, const float* __restrict__ part, int sig,
                                                      double* __restrict__ scale, const DevState* st, int gate) {
    if (gate && st->phase != 0) return;
    float m = 0.0f;
    for (int t = threadIdx.x; t < kRescaleCtas; t += blockDim.x) m = fmaxf(m, part[t]);
    const int k = rescale_shift<float>(block_max<float>(m), sig);
    if (blockIdx.x == 0 && threadIdx.x == 0) *scale = pow2d(-k);
    const float f = pow2f(k);
    const int npts = DIM == 3 ? n * n * n : n * n;
    for (int oc = blockIdx.x * blockDim.x + threadIdx.x; oc < npts; oc += gridDim.x * blockDim.x) {
        const int q = oc / n;
        const int i = oc - q * n;
        const int kz = DIM == 3 ? q / n : 0;
        const int j = q - kz * n;
        const long long o = offs<DIM>(i, j, kz, P, S);
        g[o] = __float2half_rn(x[o] * f);
    }
}

int launch_rescale(const float* x, void* g, const Geom& geo, float* part, int sig, double* scale,
                   const DevState* st, int gate, void* stream) {
    const cudaStream_t s = (cudaStream_t)stream;
    if (geo.dim == 3) {
        k_absmax<3><<<kRescaleCtas, 256, 0, s>>>(x, geo.n, geo.P, geo.S, part, st, gate);
        k_rescale_cast<3><<<kRescaleCtas, 256, 0, s>>>(x, (__half*)g, geo.n, geo.P, geo.S, part, sig, scale, st, gate);
    } else {
        k_absmax<2><<<kRescaleCtas, 256, 0, s>>>(x, geo.n, geo.P, geo.S, part, st, gate);
        k_rescale_cast<2><<<kRescaleCtas, 256, 0, s>>>(x, (__half*)g, geo.n, geo.P, geo.S, part, sig, scale, st, gate);
    }
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------- FP64 residual (IR step 1)
// r = b - A u in FP64 with per-CTA partials {sum r^2, max |r|, sum b^2, 0};
// optionally copies u to the caller's contiguous array.  One thread per point.
template <int DIM, bool init_copy>
__device__ __forceinline__ void residual64_body(const RArgs& a, int cta, int ncta) {
    if (a.gate == 1 && a.st->phase != 1) return;
    if (a.gate == 2 && !a.st->dirty) return;
    const double* bsrc = a.b ? a.b : a.st->b;
    double* uout = a.use_st_uout ? a.st->uout : a.uout;
    const int npts = DIM == 3 ? a.n * a.n * a.n : a.n * a.n;
    double sr = 0.0, sb = 0.0;
    unsigned long long mr = 0ull;
    // grid-stride over the interior points (contiguous order): fixed
    // per-CTA sets, so the partial sums are accumulated in a fixed order
    for (int oc = cta * blockDim.x + threadIdx.x; oc < npts; oc += ncta * blockDim.x) {
        const int q = oc / a.n;
        const int i = oc - q * a.n;
        const int k = DIM == 3 ? q / a.n : 0;
        const int j = q - k * a.n;
        const long long o = offs<DIM>(i, j, k, a.P, a.S);
        const double bv = __ldg(bsrc + oc);
        double r;
        if constexpr (init_copy) {
            r = bv;  // u = 0: r = b
        } else {
            const double* u = a.u + o;
            const double uc = __ldg(u);
            if (a.op == 1) {  // Q1: r = b - alpha (beta u - W) (the pads and ghost planes are zero)
                double s1 = 0.0, s2 = 0.0;  // weight-1 and weight-2 neighbour sums
#pragma unroll
                for (int dk = (DIM == 3 ? -1 : 0); dk <= (DIM == 3 ? 1 : 0); ++dk)
#pragma unroll
                    for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
                        for (int di = -1; di <= 1; ++di) {
                            const int nz = (di != 0) + (dj != 0) + (dk != 0);
                            if (nz == 0 || (DIM == 3 && nz == 1)) continue;
                            const double v = __ldg(u + di + (long long)dj * a.P + (DIM == 3 ? (long long)dk * a.S : 0LL));
                            if (DIM == 3 && nz == 2) s2 += v;
                            else s1 += v;
                        }
                const double W = fma(2.0, s2, s1);
                r = fma(-a.h2inv, fma(DIM == 3 ? 32.0 : 8.0, uc, -W), bv);
            } else {
                double nb = __ldg(u - 1) + __ldg(u + 1) + __ldg(u - a.P) + __ldg(u + a.P);
                if (DIM == 3) nb += __ldg(u - a.S) + __ldg(u + a.S);
                r = fma(-a.h2inv, fma(2.0 * DIM, uc, -nb), bv);
            }
            if (uout) uout[oc] = uc;
        }
        if (a.r) a.r[o] = r;
        // FP64 instructions are scarce on this GPU: b^2 only when asked, and
        // once for r = b
        if (!init_copy) sr = fma(r, r, sr);
        if (init_copy || a.need_b) sb = fma(bv, bv, sb);
        const unsigned long long key = abs_key(r);
        mr = key_max(mr, key);
    }
    if (init_copy) sr = sb;
    __shared__ double s1[32], s2[32];
    __shared__ unsigned long long s3[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    sr = warp_sum(sr); sb = warp_sum(sb); mr = warp_max(mr);
    if (lane == 0) { s1[wid] = sr; s2[wid] = sb; s3[wid] = mr; }
    __syncthreads();
    if (wid == 0) {
        sr = lane < nw ? s1[lane] : 0.0;
        sb = lane < nw ? s2[lane] : 0.0;
        mr = lane < nw ? s3[lane] : 0ull;
        sr = warp_sum(sr); sb = warp_sum(sb); mr = warp_max(mr);
        if (lane == 0) {
            a.partials[4LL * cta + 0] = sr;
            a.partials[4LL * cta + 1] = __longlong_as_double((long long)mr);
            a.partials[4LL * cta + 2] = sb;
            a.partials[4LL * cta + 3] = 0.0;
        }
    }
}
template <int DIM, bool init_copy>
__global__ void __launch_bounds__(256) k_residual64(RArgs a) { residual64_body<DIM, init_copy>(a, blockIdx.x, gridDim.x); }
template <int DIM, bool init_copy>
__global__ void __launch_bounds__(256) k_residual64_batch(const RItem* __restrict__ items, const int* __restrict__ cta_item) {
    const RItem& it = items[cta_item[blockIdx.x]];
    residual64_body<DIM, init_copy>(it.a, blockIdx.x - it.cta_begin, it.ncta);
}

static void residual_grid(int dim, int n, dim3& grid, dim3& block) {
    const long long npts = dim == 3 ? (long long)n * n * n : (long long)n * n;
    block = dim3(256);
    grid = dim3((unsigned)std::min<long long>(cdiv(npts, 256), 8LL * kSMs));
}

int residual64_blocks(int dim, int n) {
    dim3 g, b;
    residual_grid(dim, n, g, b);
    return (int)(g.x * g.y * g.z);
}

int launch_residual64(int dim, const RArgs& a, int* nblocks, void* stream) {
    dim3 grid, block;
    residual_grid(dim, a.n, grid, block);
    if (nblocks) *nblocks = (int)(grid.x * grid.y * grid.z);
    if (dim == 3) k_residual64<3, false><<<grid, block, 0, (cudaStream_t)stream>>>(a);
    else k_residual64<2, false><<<grid, block, 0, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

int launch_init_rb(int dim, const Geom& geo, const double* b, double* r, double* partials, const DevState* st,
                   int* nblocks, void* stream) {
    RArgs a{};
    a.n = geo.n; a.P = geo.P; a.S = geo.S; a.b = b; a.r = r; a.partials = partials; a.st = st;
    dim3 grid, block;
    residual_grid(dim, a.n, grid, block);
    if (nblocks) *nblocks = (int)(grid.x * grid.y * grid.z);
    if (dim == 3) k_residual64<3, true><<<grid, block, 0, (cudaStream_t)stream>>>(a);
    else k_residual64<2, true><<<grid, block, 0, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}


__global__ void k_finalize(int kind, DevState* st, const double* __restrict__ partials, int nblocks) {
    finalize_body(kind, st, partials, nblocks);
}
// Batched: one CTA per instance.
__global__ void k_finalize_batch(int kind, const FinItem* __restrict__ items) {
    const FinItem& it = items[blockIdx.x];
    finalize_body(kind, it.st, it.partials, it.nblocks);
}
int launch_finalize_batch(int kind, const FinItem* items, int nitems, void* stream) {
    k_finalize_batch<<<nitems, 1024, 0, (cudaStream_t)stream>>>(kind, items);
    return (int)cudaGetLastError();
}

int launch_finalize(int kind, DevState* st, const double* partials, int nblocks, void* stream) {
    k_finalize<<<1, 1024, 0, (cudaStream_t)stream>>>(kind, st, partials, nblocks);
    return (int)cudaGetLastError();
}

// Evicts L2 by reading a buffer larger than it (the autotuner's cold-cache
// timing): clean lines replace whatever the cache held, with no write-back
// traffic left to overlap the next kernel, as a memset flush would leave.
// The sum feeds a store only under a condition the contents never meet, so
// the loads stay.
__global__ void __launch_bounds__(256) k_l2_evict(const uint4* __restrict__ p, long long n16, unsigned* sink) {
    unsigned acc = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (long long)gridDim.x * blockDim.x) {
        const uint4 v = __ldcg(p + i);
        acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
    if (acc == 0x9E3779B9u) atomicAdd(sink, 1u);
}
int launch_l2_evict(const void* buf, size_t bytes, unsigned* sink, void* stream) {
    k_l2_evict<<<8 * kSMs, 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<const uint4*>(buf), (long long)(bytes / 16), sink);
    return (int)cudaGetLastError();
}

// Holds the stream for about ns nanoseconds (one thread sleeping on the
// global timer; at most 2^16 sleeps of at most 1 us each, so it always ends).
// The per-kernel profile launches it ahead of each step so that the host has
// enqueued the step's kernels and events before the device reaches them: the
// event pairs then time the kernels, not the host's enqueue gaps.
__global__ void k_hold(long long ns) {
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (int i = 0; i < (1 << 16); ++i) {
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if ((long long)(t - t0) >= ns) return;
        __nanosleep(1000);
    }
}
int launch_hold(long long ns, void* stream) {
    k_hold<<<1, 1, 0, (cudaStream_t)stream>>>(ns);
    return (int)cudaGetLastError();
}

// Sets the condition of the device-side IR loop (a WHILE node of the solve
// graph).  The body-count limit ends the loop even if the state never leaves
// phases 0/1, so the graph always terminates.
__global__ void k_loop_condition(DevState* st, cudaGraphConditionalHandle h, int limit) {
    const int loops = st->loops + 1;
    st->loops = loops;
    const bool more = (st->phase == 0 || st->phase == 1) && loops < limit;
    if (!more && (st->phase == 0 || st->phase == 1)) {  // body-count limit hit: stop as not converged
        st->phase = 3;
        st->status = MG_ERR_NOT_CONVERGED;
    }
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

// Batched: the loop runs while any instance is iterating or has its true-
// residual check pending; every instance counts the body's iterations.
__global__ void k_loop_condition_batch(DevState* const* sts, int n, cudaGraphConditionalHandle h, int limit) {
    bool more = false;
    for (int i = 0; i < n; ++i) {
        DevState* st = sts[i];
        const int loops = st->loops + 1;
        st->loops = loops;
        if (st->phase == 0 || st->phase == 1) {
            if (loops < limit) {
                more = true;
            } else {
                st->phase = 3;
                st->status = MG_ERR_NOT_CONVERGED;
            }
        }
    }
    cudaGraphSetConditional(h, more ? 1u : 0u);
}
int launch_loop_condition_batch(DevState* const* sts, int n, unsigned long long handle, int limit, void* stream) {
    k_loop_condition_batch<<<1, 1, 0, (cudaStream_t)stream>>>(sts, n, (cudaGraphConditionalHandle)handle, limit);
    return (int)cudaGetLastError();
}
int launch_residual64_batch(int dim, bool init_copy, const RItem* items, const int* cta_item, int ncta, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (dim == 3) {
        if (init_copy) k_residual64_batch<3, true><<<ncta, 256, 0, s>>>(items, cta_item);
        else k_residual64_batch<3, false><<<ncta, 256, 0, s>>>(items, cta_item);
    } else {
        if (init_copy) k_residual64_batch<2, true><<<ncta, 256, 0, s>>>(items, cta_item);
        else k_residual64_batch<2, false><<<ncta, 256, 0, s>>>(items, cta_item);
    }
    return (int)cudaGetLastError();
}
int residual64_ctas(int dim, int n) {
    dim3 grid, block;
    residual_grid(dim, n, grid, block);
    return (int)grid.x;
}

int launch_loop_condition(DevState* st, unsigned long long handle, int limit, void* stream) {
    k_loop_condition<<<1, 1, 0, (cudaStream_t)stream>>>(st, (cudaGraphConditionalHandle)handle, limit);
    return (int)cudaGetLastError();
}

__global__ void k_pack_u0(int dim, int n, int P, long long S, const DevState* st, double* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= n || j >= n) return;
    const long long o = (dim == 3 ? (long long)k * S : 0LL) + (long long)j * P + i;
    const long long oc = dim == 3 ? ((long long)k * n + j) * n + i : (long long)j * n + i;
    dst[o] = st->uout[oc];
}

int launch_pack_u0(int dim, const Geom& geo, const DevState* st, double* u_padded, void* stream) {
    dim3 block(64, 4), grid((unsigned)cdiv(geo.n, 64), (unsigned)cdiv(geo.n, 4), (unsigned)(dim == 3 ? geo.n : 1));
    k_pack_u0<<<grid, block, 0, (cudaStream_t)stream>>>(dim, geo.n, geo.P, geo.S, st, u_padded);
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------- packing
template <class T>
__global__ void k_pack(int dim, int n, int P, long long S, const T* __restrict__ src, T* __restrict__ dst, int unpack) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= n || j >= n) return;
    const long long o = (dim == 3 ? (long long)k * S : 0LL) + (long long)j * P + i;
    const long long oc = dim == 3 ? ((long long)k * n + j) * n + i : (long long)j * n + i;
    if (unpack) dst[oc] = src[o];
    else dst[o] = src[oc];
}

static int pack_any(int dim, int prec, const Geom& geo, const void* src, void* dst, int unpack, void* stream) {
    dim3 block(64, 4), grid((unsigned)cdiv(geo.n, 64), (unsigned)cdiv(geo.n, 4), (unsigned)(dim == 3 ? geo.n : 1));
    cudaStream_t s = (cudaStream_t)stream;
    switch (elem_size(prec)) {
        case 8: k_pack<unsigned long long><<<grid, block, 0, s>>>(dim, geo.n, geo.P, geo.S, (const unsigned long long*)src, (unsigned long long*)dst, unpack); break;
        case 4: k_pack<unsigned><<<grid, block, 0, s>>>(dim, geo.n, geo.P, geo.S, (const unsigned*)src, (unsigned*)dst, unpack); break;
        default: k_pack<unsigned short><<<grid, block, 0, s>>>(dim, geo.n, geo.P, geo.S, (const unsigned short*)src, (unsigned short*)dst, unpack); break;
    }
    return (int)cudaGetLastError();
}

int launch_pack(int dim, int prec, const Geom& geo, const void* src_contig, void* dst_padded, void* stream) {
    return pack_any(dim, prec, geo, src_contig, dst_padded, 0, stream);
}
int launch_unpack(int dim, int prec, const Geom& geo, const void* src_padded, void* dst_contig, void* stream) {
    return pack_any(dim, prec, geo, src_padded, dst_contig, 1, stream);
}

}  // namespace mgi
