// Stencil "march" kernels of libmgfp.
//
// One template covers every grid pass of the method that applies the
// 5/7-point operator A_l (Sec. 5):
//   M_JACOBI    damped Jacobi sweep (Sec. 4.2 smoother; Alg. 1 steps 1, 5)
//   M_ZERO2     the first two sweeps of a pre-smoothing that starts from c = 0
//               (Alg. 1 step 1 with a zero initial guess), fused in one pass
//   M_ZERO1     one sweep from c = 0 (c = omega D^-1 g)
//   M_RESTRICT  residual g - A c and its full-weighting restriction to the
//               next coarser level with the precision change (Alg. 1 step 2)
//   M_UPDATE    Alg. 2 lines 6-7 fused (the paper's UpdateResiduum_Correction):
//               u += alpha c, r -= alpha A c in FP64, with norm partials
// and three ways of producing the marched vector ("loaders"):
//   L_PLAIN     the stored level vector
//   L_SCALED    the cast of the scaled FP64 residual, r * inv rounded to the
//               level type (Alg. 2 line 4), also stored as the level's g
//   L_PROLONG   c + P c_coarse: prolongation and correction (Alg. 1 step 4)
//               fused into the first post-smoothing sweep
//
// Work decomposition (3D): a CTA of TY warps owns TY consecutive rows of a
// 32*V-wide x-chunk (V = elements per 16-byte vector: 8 for FP16/BF16, 4 for
// FP32, 2 for FP64) and marches over a z-range.  Each lane keeps its vector
// of planes z-1, z, z+1 in registers (coalesced 128-bit loads, one new plane
// per step), the y-neighbours come from a double-buffered shared-memory tile
// of plane z with one halo row above and below, and the x-neighbours from
// warp shuffles (plus one scalar halo load at each chunk edge).  In 2D a warp
// owns an x-chunk and marches over rows; no shared memory is needed.
// Arithmetic is FP32 for FP16/BF16/FP32 levels and FP64 for FP64 levels.
#pragma once
#include "mg_device.cuh"

namespace mgi {

template <int DIM>
__device__ __forceinline__ long long offs(int x, int y, int z, int P, long long S) {
    return DIM == 3 ? (long long)z * S + (long long)y * P + x : (long long)y * P + x;
}

// Multiplication by inv split as 2^E * m, m in [1, 2): the exponent is added
// to the FP64 bit pattern with an integer add (exact), the significand product
// is done in FP32.  Used to scale and cast the FP64 residual without FP64
// instructions.
struct ScaleK {
    double inv;
    long long eadd;
    float mant;
};
__device__ __forceinline__ ScaleK make_scale(double inv) {
    ScaleK k;
    k.inv = inv;
    long long b = __double_as_longlong(inv);
    int E = (int)((b >> 52) & 0x7FF) - 1023;
    k.eadd = (long long)E << 52;
    k.mant = f64_to_f32_trunc(__longlong_as_double((b & 0x000FFFFFFFFFFFFFll) | 0x3FF0000000000000ll));
    return k;
}
__device__ __forceinline__ float scaled_f32(double r, const ScaleK& k) {
    long long b = __double_as_longlong(r);
    long long ex = b & 0x7FF0000000000000ll;
    if (ex == 0) return 0.0f;
    if (ex == 0x7FF0000000000000ll) return f64_to_f32_trunc(r);
    return __fmul_rn(f64_to_f32_trunc(__longlong_as_double(b + k.eadd)), k.mant);
}

template <class T> struct ScaledVal {
    __device__ static float get(double r, const ScaleK& k) { return rnd(scaled_f32(r, k), (const T*)nullptr); }
};
template <> struct ScaledVal<double> {
    __device__ static double get(double r, const ScaleK& k) { return r * k.inv; }
};

// ---------------------------------------------------------------- loaders
template <int DIM, int LD, class T, class TC> struct Load {
    using C = typename Tr<T>::C;
    static constexpr int V = Tr<T>::V;

    // Prolongation P c_coarse added to v (fine x even, V consecutive points).
    __device__ static void add_prolong_vec(const KArgs& a, int x, int y, int z, C (&v)[V]) {
        const TC* cc = reinterpret_cast<const TC*>(a.coarse);
        int Jl, Jh, Kl = 0, Kh = 0;
        C w = 1;
        if (y & 1) { Jl = Jh = (y - 1) >> 1; } else { Jl = (y >> 1) - 1; Jh = y >> 1; w *= (C)0.5; }
        if (DIM == 3) {
            if (z & 1) { Kl = Kh = (z - 1) >> 1; } else { Kl = (z >> 1) - 1; Kh = z >> 1; w *= (C)0.5; }
        }
        const int I0 = (x >> 1) - 1;
        C s[V / 2 + 1];
#pragma unroll
        for (int k = 0; k <= V / 2; ++k) s[k] = 0;
        for (int K = Kl; K <= Kh; ++K)
            for (int J = Jl; J <= Jh; ++J) {
                const TC* row = cc + (DIM == 3 ? (long long)K * a.Sc : 0LL) + (long long)J * a.Pc + I0;
#pragma unroll
                for (int k = 0; k <= V / 2; ++k) s[k] += (C)ld1(row + k);
            }
#pragma unroll
        for (int i = 0; i < V; ++i) {
            C p = (i & 1) ? s[(i + 1) >> 1] : (C)0.5 * (s[i >> 1] + s[(i >> 1) + 1]);
            v[i] += w * p;
        }
    }
    __device__ static C prolong_one(const KArgs& a, int x, int y, int z) {
        const TC* cc = reinterpret_cast<const TC*>(a.coarse);
        int Jl, Jh, Kl = 0, Kh = 0, Il, Ih;
        C w = 1;
        if (y & 1) { Jl = Jh = (y - 1) >> 1; } else { Jl = (y >> 1) - 1; Jh = y >> 1; w *= (C)0.5; }
        if (x & 1) { Il = Ih = (x - 1) >> 1; } else { Il = (x >> 1) - 1; Ih = x >> 1; w *= (C)0.5; }
        if (DIM == 3) {
            if (z & 1) { Kl = Kh = (z - 1) >> 1; } else { Kl = (z >> 1) - 1; Kh = z >> 1; w *= (C)0.5; }
        }
        C s = 0;
        for (int K = Kl; K <= Kh; ++K)
            for (int J = Jl; J <= Jh; ++J)
                for (int I = Il; I <= Ih; ++I)
                    s += (C)ld1(cc + (DIM == 3 ? (long long)K * a.Sc : 0LL) + (long long)J * a.Pc + I);
        return w * s;
    }

    __device__ static void vec(const KArgs& a, const ScaleK& sk, int x, int y, int z, bool ok, C (&v)[V]) {
        if (!ok) {
#pragma unroll
            for (int i = 0; i < V; ++i) v[i] = 0;
            return;
        }
        const long long o = offs<DIM>(x, y, z, a.P, a.S);
        if (LD == L_SCALED) {
            const double* rp = a.r64 + o;
#pragma unroll
            for (int i = 0; i < V; i += 2) {
                double2 t = __ldg(reinterpret_cast<const double2*>(rp + i));
                v[i] = ScaledVal<T>::get(t.x, sk);
                v[i + 1] = ScaledVal<T>::get(t.y, sk);
            }
        } else {
            ldv(reinterpret_cast<const T*>(a.src) + o, v);
            if (LD == L_PROLONG) add_prolong_vec(a, x, y, z, v);
        }
    }
    __device__ static C one(const KArgs& a, const ScaleK& sk, int x, int y, int z) {
        const long long o = offs<DIM>(x, y, z, a.P, a.S);
        if (LD == L_SCALED) return ScaledVal<T>::get(__ldg(a.r64 + o), sk);
        C v = ld1(reinterpret_cast<const T*>(a.src) + o);
        if (LD == L_PROLONG) v += prolong_one(a, x, y, z);
        return v;
    }
};

// ---------------------------------------------------------------- exact A c for the FP64 update
// S = 2d c0 - (sum of neighbours), exactly, returned as FP64 in the units
// given by *scale (2^-24 for FP16 inputs, 1 otherwise) with a residual part.
template <class T> struct ExactStencil;

template <> struct ExactStencil<__half> {
    static constexpr bool kTwoTerm = false;
    // FP16 values: exact integer arithmetic in units of 2^-24 (see h_split).
    // NB = 2d neighbours; |H| < 2^26 and |L| < 2^21, so both sums are exact.
    template <int NB>
    __device__ static void sum(float c0, const float (&nb)[NB], double& s, double& s2) {
        const float MAGIC = 12582912.0f;
        HSplit q = h_split(c0);
        int H = NB * q.hi;
        float L = __fmul_rn((float)NB, q.lo);
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            HSplit t = h_split(nb[j]);
            H -= t.hi;
            L = __fsub_rn(L, t.lo);
        }
        int Li = __float_as_int(__fadd_rn(L, MAGIC)) - __float_as_int(MAGIC);
        long long Sint = ((long long)H << 18) + (long long)Li;
        s = i64_to_f64(Sint, -24);
        s2 = 0.0;
    }
};
template <class T> struct ExactStencil {
    static constexpr bool kTwoTerm = true;
    // FP32/BF16 values: double-float sum with error-free transformations.
    template <int NB>
    __device__ static void sum(float c0, const float (&nb)[NB], double& s, double& s2) {
        float p = __fmul_rn((float)NB, c0);
        float e = __fmaf_rn((float)NB, c0, -p);
        float acc = p;
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            float t, err;
            two_sum(acc, -nb[j], t, err);
            acc = t;
            e = __fadd_rn(e, err);
        }
        s = f32_to_f64(acc);
        s2 = f32_to_f64(e);
    }
};
template <> struct ExactStencil<double> {
    static constexpr bool kTwoTerm = false;
    template <int NB>
    __device__ static void sum(double c0, const double (&nb)[NB], double& s, double& s2) {
        double t = 0.0;
#pragma unroll
        for (int j = 0; j < NB; ++j) t += nb[j];
        s = fma((double)NB, c0, -t);
        s2 = 0.0;
    }
};

__device__ __forceinline__ double to_f64(float v) { return f32_to_f64(v); }
__device__ __forceinline__ double to_f64(double v) { return v; }

// ---------------------------------------------------------------- per-point epilogue helpers
template <int MODE, class C>
__device__ __forceinline__ C point_value(C c0, C nb, C g, C c1, C c2, C c3, C h2inv, C twod, C om) {
    if (MODE == M_JACOBI) return c1 * c0 + c2 * nb + c3 * g;            // c + w D^-1 (g - A c)
    if (MODE == M_ZERO2) return c3 * (((C)2 - om) * c0 + c2 * nb);       // two sweeps from 0, c0 = g
    if (MODE == M_ZERO1) return c3 * c0;                                   // one sweep from 0
    return g - h2inv * (twod * c0 - nb);                                   // residual g - A c
}

template <int DIM>
__device__ __forceinline__ void write_partials(double nsum, unsigned long long nmax, double* partials,
                                               int nwarps, int lane, int w) {
    __shared__ double rs[32];
    __shared__ unsigned long long rm[32];
    nsum = warp_sum(nsum);
    nmax = warp_max(nmax);
    if (lane == 0) { rs[w] = nsum; rm[w] = nmax; }
    __syncthreads();
    if (w == 0) {
        double s = lane < nwarps ? rs[lane] : 0.0;
        unsigned long long m = lane < nwarps ? rm[lane] : 0ull;
        s = warp_sum(s);
        m = warp_max(m);
        if (lane == 0) {
            const long long bid = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
            partials[2 * bid] = s;
            partials[2 * bid + 1] = __longlong_as_double((long long)m);
        }
    }
}

// Alg. 2 lines 6-7 on one vector of V points: FP64 loads/stores of u and r.
template <int DIM, class T, class C, int V>
__device__ __forceinline__ void update_vec(const KArgs& a, long long o, int x, const C (&c0)[V], C left, C right,
                                           const C (&cm)[V], const C (&cp)[V], const C (&ym)[V],
                                           const C (&yp)[V], double alpha, double beta, double& nsum,
                                           unsigned long long& nmax) {
    double* up = a.u64 + o;
    double* rp = a.rw64 + o;
    double uu[V], rr[V];
#pragma unroll
    for (int i = 0; i < V; i += 2) {
        double2 tu = *reinterpret_cast<const double2*>(up + i);
        double2 tr = *reinterpret_cast<const double2*>(rp + i);
        uu[i] = tu.x; uu[i + 1] = tu.y; rr[i] = tr.x; rr[i + 1] = tr.y;
    }
#pragma unroll
    for (int i = 0; i < V; ++i) {
        if (x + i < a.n) {
            C xm = i ? c0[i - 1] : left;
            C xp = i < V - 1 ? c0[i + 1] : right;
            double s, s2;
            if (DIM == 3) {
                const C nb[6] = {xm, xp, cm[i], cp[i], ym[i], yp[i]};
                ExactStencil<T>::template sum<6>(c0[i], nb, s, s2);
            } else {
                const C nb[4] = {xm, xp, cm[i], cp[i]};
                ExactStencil<T>::template sum<4>(c0[i], nb, s, s2);
            }
            double r = fma(-beta, s, rr[i]);
            if (ExactStencil<T>::kTwoTerm) r = fma(-beta, s2, r);
            rr[i] = r;
            uu[i] = fma(alpha, to_f64(c0[i]), uu[i]);
            nsum = fma(r, r, nsum);
            unsigned long long k = abs_key(r);
            nmax = k > nmax ? k : nmax;
        }
    }
#pragma unroll
    for (int i = 0; i < V; i += 2) {
        *reinterpret_cast<double2*>(up + i) = make_double2(uu[i], uu[i + 1]);
        *reinterpret_cast<double2*>(rp + i) = make_double2(rr[i], rr[i + 1]);
    }
}

// ---------------------------------------------------------------- 3D march
template <int MODE, int LD, class T, class TC>
__global__ void __launch_bounds__(384) k_march3(const KArgs a) {
    using C = typename Tr<T>::C;
    constexpr int V = Tr<T>::V;
    constexpr int CW = 32 * V;
    constexpr int VH = V / 2 > 0 ? V / 2 : 1;
    using LDR = Load<3, LD, T, TC>;
    if (a.gate && a.st->phase != 0) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TY = blockDim.y, lane = threadIdx.x, w = threadIdx.y;
    C* planes = reinterpret_cast<C*>(smem_raw);
    C* flush = planes + 2 * (TY + 2) * CW;
    const int x0 = blockIdx.x * a.xstep, x = x0 + lane * V;
    const int y0 = blockIdx.y * a.ystep, y = y0 + w;
    const int zb = blockIdx.z * a.zstep;
    const int ze = min(zb + a.zlen, a.n);
    const bool lane_in = x < a.P, row_in = y < a.n, act = lane_in && row_in;
    ScaleK sk;
    if (LD == L_SCALED) sk = make_scale(a.st ? a.st->inv : a.inv_explicit);
    const C h2inv = (C)a.h2inv, om = (C)a.omega, twod = (C)6;
    const C c1 = (C)1 - om, c2 = om / twod, c3 = om / (twod * h2inv);
    const T* gp = reinterpret_cast<const T*>(a.g);
    T* dp = reinterpret_cast<T*>(a.dst);
    double alpha = 0.0, beta = 0.0;
    if (MODE == M_UPDATE) {
        alpha = a.st ? a.st->alpha : a.a_step;
        beta = alpha * a.h2inv;
    }
    C cm[V], c0[V], cp[V], acc[VH];
#pragma unroll
    for (int k = 0; k < VH; ++k) acc[k] = 0;
    double nsum = 0.0;
    unsigned long long nmax = 0ull;
    LDR::vec(a, sk, x, y, zb - 1, act, cm);
    LDR::vec(a, sk, x, y, zb, act, c0);
    if (LD == L_SCALED && act && zb < ze) stv(reinterpret_cast<T*>(a.gside) + offs<3>(x, y, zb, a.P, a.S), c0);
    for (int z = zb; z < ze; ++z) {
        LDR::vec(a, sk, x, y, z + 1, act, cp);
        if (LD == L_SCALED && act && z + 1 < ze)
            stv(reinterpret_cast<T*>(a.gside) + offs<3>(x, y, z + 1, a.P, a.S), cp);
        C* buf = planes + (z & 1) * (TY + 2) * CW;
#pragma unroll
        for (int i = 0; i < V; ++i) buf[(w + 1) * CW + lane * V + i] = c0[i];
        if (w == 0) {
            C hv[V];
            LDR::vec(a, sk, x, y0 - 1, z, lane_in, hv);
#pragma unroll
            for (int i = 0; i < V; ++i) buf[lane * V + i] = hv[i];
        }
        if (w == TY - 1) {
            C hv[V];
            LDR::vec(a, sk, x, y0 + TY, z, lane_in && y0 + TY <= a.n, hv);
#pragma unroll
            for (int i = 0; i < V; ++i) buf[(TY + 1) * CW + lane * V + i] = hv[i];
        }
        C xl = 0, xr = 0;
        if (lane == 0 && row_in) xl = LDR::one(a, sk, x0 - 1, y, z);
        if (lane == 31 && row_in && x0 + CW < a.P) xr = LDR::one(a, sk, x0 + CW, y, z);
        __syncthreads();
        C ym[V], yp[V];
#pragma unroll
        for (int i = 0; i < V; ++i) {
            ym[i] = buf[w * CW + lane * V + i];
            yp[i] = buf[(w + 2) * CW + lane * V + i];
        }
        C left = __shfl_up_sync(kFull, c0[V - 1], 1);
        C right = __shfl_down_sync(kFull, c0[0], 1);
        if (lane == 0) left = xl;
        if (lane == 31) right = xr;
        const long long o = offs<3>(x, y, z, a.P, a.S);
        if constexpr (MODE == M_UPDATE) {
            if (act) update_vec<3, T, C, V>(a, o, x, c0, left, right, cm, cp, ym, yp, alpha, beta, nsum, nmax);
        } else {
            C g[V];
            if (MODE == M_JACOBI || MODE == M_RESTRICT) {
                if (act) ldv(gp + o, g);
                else {
#pragma unroll
                    for (int i = 0; i < V; ++i) g[i] = 0;
                }
            }
            C out[V];
#pragma unroll
            for (int i = 0; i < V; ++i) {
                C nb = (i ? c0[i - 1] : left) + (i < V - 1 ? c0[i + 1] : right) + cm[i] + cp[i] + ym[i] + yp[i];
                C gi = (MODE == M_JACOBI || MODE == M_RESTRICT) ? g[i] : (C)0;
                C v = point_value<MODE, C>(c0[i], nb, gi, c1, c2, c3, h2inv, twod, om);
                out[i] = (x + i < a.n && row_in) ? v : (C)0;
            }
            if constexpr (MODE != M_RESTRICT) {
                if (act) stv(dp + o, out);
            } else {
                C rn = __shfl_down_sync(kFull, out[0], 1);
                if (lane == 31) rn = 0;
                C q[VH];
#pragma unroll
                for (int k = 0; k < VH; ++k) {
                    C r2 = (2 * k + 2 < V) ? out[(2 * k + 2) % V] : rn;
                    q[k] = (C)0.25 * out[2 * k] + (C)0.5 * out[2 * k + 1] + (C)0.25 * r2;
                }
                const int t = z - zb;
                if (t & 1) {
#pragma unroll
                    for (int k = 0; k < VH; ++k) acc[k] += (C)0.5 * q[k];
                } else {
                    if (t >= 2) {
                        C* fl = flush + (w * 32 + lane) * VH;
#pragma unroll
                        for (int k = 0; k < VH; ++k) fl[k] = acc[k] + (C)0.25 * q[k];
                        __syncthreads();
                        if ((w & 1) == 0 && w + 2 < TY) {
                            const int J = (y0 >> 1) + (w >> 1), K = (zb >> 1) + (t >> 1) - 1;
                            const C* f0 = flush + (w * 32 + lane) * VH;
                            const C* f1 = f0 + 32 * VH;
                            const C* f2 = f1 + 32 * VH;
                            const int I0 = (x0 + lane * V) >> 1;
                            if (lane_in && J < a.nc && K < a.nc && (lane < 31 || x0 + CW >= a.P)) {
                                TC* cd = reinterpret_cast<TC*>(a.dst) + (long long)K * a.Sc + (long long)J * a.Pc;
#pragma unroll
                                for (int k = 0; k < VH; ++k)
                                    if (I0 + k < a.nc)
                                        st1(cd + I0 + k, (C)0.25 * f0[k] + (C)0.5 * f1[k] + (C)0.25 * f2[k]);
                            }
                        }
                    }
#pragma unroll
                    for (int k = 0; k < VH; ++k) acc[k] = (C)0.25 * q[k];
                }
            }
        }
#pragma unroll
        for (int i = 0; i < V; ++i) { cm[i] = c0[i]; c0[i] = cp[i]; }
    }
    if constexpr (MODE == M_UPDATE) write_partials<3>(nsum, nmax, a.partials, TY, lane, w);
}

// ---------------------------------------------------------------- 2D march
template <int MODE, int LD, class T, class TC>
__global__ void __launch_bounds__(256) k_march2(const KArgs a) {
    using C = typename Tr<T>::C;
    constexpr int V = Tr<T>::V;
    constexpr int CW = 32 * V;
    constexpr int VH = V / 2 > 0 ? V / 2 : 1;
    using LDR = Load<2, LD, T, TC>;
    if (a.gate && a.st->phase != 0) return;
    const int W = blockDim.y, lane = threadIdx.x, w = threadIdx.y;
    const int x0 = (blockIdx.x * W + w) * a.xstep, x = x0 + lane * V;
    const bool lane_in = x0 < a.P && x < a.P;
    const int yb = blockIdx.y * a.zstep;
    const int ye = min(yb + a.zlen, a.n);
    ScaleK sk;
    if (LD == L_SCALED) sk = make_scale(a.st ? a.st->inv : a.inv_explicit);
    const C h2inv = (C)a.h2inv, om = (C)a.omega, twod = (C)4;
    const C c1 = (C)1 - om, c2 = om / twod, c3 = om / (twod * h2inv);
    const T* gp = reinterpret_cast<const T*>(a.g);
    T* dp = reinterpret_cast<T*>(a.dst);
    double alpha = 0.0, beta = 0.0;
    if (MODE == M_UPDATE) {
        alpha = a.st ? a.st->alpha : a.a_step;
        beta = alpha * a.h2inv;
    }
    C cm[V], c0[V], cp[V], acc[VH];
    const C zero[V] = {};
#pragma unroll
    for (int k = 0; k < VH; ++k) acc[k] = 0;
    double nsum = 0.0;
    unsigned long long nmax = 0ull;
    LDR::vec(a, sk, x, yb - 1, 0, lane_in, cm);
    LDR::vec(a, sk, x, yb, 0, lane_in, c0);
    if (LD == L_SCALED && lane_in && yb < ye) stv(reinterpret_cast<T*>(a.gside) + offs<2>(x, yb, 0, a.P, a.S), c0);
    for (int y = yb; y < ye; ++y) {
        LDR::vec(a, sk, x, y + 1, 0, lane_in, cp);
        if (LD == L_SCALED && lane_in && y + 1 < ye)
            stv(reinterpret_cast<T*>(a.gside) + offs<2>(x, y + 1, 0, a.P, a.S), cp);
        C xl = 0, xr = 0;
        if (lane == 0 && x0 < a.P) xl = LDR::one(a, sk, x0 - 1, y, 0);
        if (lane == 31 && x0 + CW < a.P) xr = LDR::one(a, sk, x0 + CW, y, 0);
        C left = __shfl_up_sync(kFull, c0[V - 1], 1);
        C right = __shfl_down_sync(kFull, c0[0], 1);
        if (lane == 0) left = xl;
        if (lane == 31) right = xr;
        const long long o = offs<2>(x, y, 0, a.P, a.S);
        if constexpr (MODE == M_UPDATE) {
            if (lane_in) update_vec<2, T, C, V>(a, o, x, c0, left, right, cm, cp, zero, zero, alpha, beta, nsum, nmax);
        } else {
            C g[V];
            if (MODE == M_JACOBI || MODE == M_RESTRICT) {
                if (lane_in) ldv(gp + o, g);
                else {
#pragma unroll
                    for (int i = 0; i < V; ++i) g[i] = 0;
                }
            }
            C out[V];
#pragma unroll
            for (int i = 0; i < V; ++i) {
                C nb = (i ? c0[i - 1] : left) + (i < V - 1 ? c0[i + 1] : right) + cm[i] + cp[i];
                C gi = (MODE == M_JACOBI || MODE == M_RESTRICT) ? g[i] : (C)0;
                C v = point_value<MODE, C>(c0[i], nb, gi, c1, c2, c3, h2inv, twod, om);
                out[i] = (x + i < a.n) ? v : (C)0;
            }
            if constexpr (MODE != M_RESTRICT) {
                if (lane_in) stv(dp + o, out);
            } else {
                C rn = __shfl_down_sync(kFull, out[0], 1);
                if (lane == 31) rn = 0;
                C q[VH];
#pragma unroll
                for (int k = 0; k < VH; ++k) {
                    C r2 = (2 * k + 2 < V) ? out[(2 * k + 2) % V] : rn;
                    q[k] = (C)0.25 * out[2 * k] + (C)0.5 * out[2 * k + 1] + (C)0.25 * r2;
                }
                const int t = y - yb;
                if (t & 1) {
#pragma unroll
                    for (int k = 0; k < VH; ++k) acc[k] += (C)0.5 * q[k];
                } else {
                    if (t >= 2) {
                        const int J = (yb >> 1) + (t >> 1) - 1;
                        const int I0 = (x0 + lane * V) >> 1;
                        if (lane_in && J < a.nc && (lane < 31 || x0 + CW >= a.P)) {
                            TC* cd = reinterpret_cast<TC*>(a.dst) + (long long)J * a.Pc;
#pragma unroll
                            for (int k = 0; k < VH; ++k)
                                if (I0 + k < a.nc) st1(cd + I0 + k, acc[k] + (C)0.25 * q[k]);
                        }
                    }
#pragma unroll
                    for (int k = 0; k < VH; ++k) acc[k] = (C)0.25 * q[k];
                }
            }
        }
#pragma unroll
        for (int i = 0; i < V; ++i) { cm[i] = c0[i]; c0[i] = cp[i]; }
    }
    if constexpr (MODE == M_UPDATE) write_partials<2>(nsum, nmax, a.partials, W, lane, w);
}

}  // namespace mgi
