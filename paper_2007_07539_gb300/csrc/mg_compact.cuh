// Single-CTA building blocks on compact level arrays (x fastest, n^d values,
// no pads; the zero boundary is a bounds check): index decoding, block-wide
// reductions, the power-of-two rescale rule of FP16 levels and the conjugate
// gradient base solver.  Used by the coarse-tail kernel and by the base-level
// kernels of hierarchies without a tail.
#pragma once
#include <type_traits>

#include "mg_device.cuh"

namespace mgi {

// p / n through mn = ceil(2^40 / n) (division by an invariant integer with a
// fixed-point reciprocal): the error p (mn - 2^40/n) / 2^40 < p / 2^40 stays
// below 1/n, so the quotient is exact, for every p < 2^40 / n (here p < 2^20,
// n < 2^10)
__device__ __forceinline__ int divn(int p, unsigned long long mn) {
    return (int)(((unsigned long long)(unsigned)p * mn) >> 40);
}
// (i, j, k) of compact point p
template <int DIM>
__device__ __forceinline__ void decode(int p, int n, unsigned long long mn, int& i, int& j, int& k) {
    const int q = divn(p, mn);
    i = p - q * n;
    if (DIM == 3) {
        k = divn(q, mn);
        j = q - k * n;
    } else {
        j = q;
        k = 0;
    }
}

template <class T>
__device__ __forceinline__ typename Tr<T>::C cget(const T* a, int p) {
    if constexpr (std::is_same<T, __half>::value) return __half2float(a[p]);
    else if constexpr (std::is_same<T, __nv_bfloat16>::value) return __bfloat162float(a[p]);
    else return a[p];
}

// sum of the 2*DIM axis neighbours of compact point p; zero outside the grid.
// get(q) returns the value of point q in the arithmetic type C.
template <int DIM, class C, class G>
__device__ __forceinline__ C cnbsum_f(const G& get, int p, int n, int i, int j, int k) {
    C s = 0;
    if (i > 0) s += get(p - 1);
    if (i < n - 1) s += get(p + 1);
    if (j > 0) s += get(p - n);
    if (j < n - 1) s += get(p + n);
    if (DIM == 3) {
        if (k > 0) s += get(p - n * n);
        if (k < n - 1) s += get(p + n * n);
    }
    return s;
}
template <int DIM, class T>
__device__ __forceinline__ typename Tr<T>::C cnbsum(const T* a, int p, int n, int i, int j, int k) {
    return cnbsum_f<DIM, typename Tr<T>::C>([&](int q) { return cget(a, q); }, p, n, i, j, k);
}

// W of the Q1 operator at compact point p: weight 1 on the 8 neighbours (2D);
// 2 on the 12 edge and 1 on the 8 corner neighbours, 0 on the 6 faces (3D)
template <int DIM, class C, class G>
__device__ __forceinline__ C cwsum_q1_f(const G& get, int p, int n, int i, int j, int k) {
    C s1 = 0, s2 = 0;  // weight-1 and weight-2 sums
#pragma unroll
    for (int dk = (DIM == 3 ? -1 : 0); dk <= (DIM == 3 ? 1 : 0); ++dk)
#pragma unroll
        for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
            for (int di = -1; di <= 1; ++di) {
                const int nz = (di != 0) + (dj != 0) + (dk != 0);
                if (nz == 0 || (DIM == 3 && nz == 1)) continue;
                if (i + di < 0 || i + di >= n || j + dj < 0 || j + dj >= n || k + dk < 0 || k + dk >= (DIM == 3 ? n : 1))
                    continue;
                const C v = get(p + di + dj * n + dk * n * n);
                if (DIM == 3 && nz == 2) s2 += v;
                else s1 += v;
            }
    return (C)2 * s2 + s1;
}
template <int DIM, class T>
__device__ __forceinline__ typename Tr<T>::C cwsum_q1(const T* a, int p, int n, int i, int j, int k) {
    return cwsum_q1_f<DIM, typename Tr<T>::C>([&](int q) { return cget(a, q); }, p, n, i, j, k);
}
// beta of operator op (the centre weight of beta I - W)
template <int DIM>
__device__ __forceinline__ int op_beta_d(int op) { return op == 1 ? (DIM == 3 ? 32 : 8) : 2 * DIM; }
// W of operator op (0: the 2d axis neighbours, 1: Q1)
template <int DIM, class T>
__device__ __forceinline__ typename Tr<T>::C cwsum(int op, const T* a, int p, int n, int i, int j, int k) {
    return op == 1 ? cwsum_q1<DIM, T>(a, p, n, i, j, k) : cnbsum<DIM, T>(a, p, n, i, j, k);
}
template <int DIM, class C, class G>
__device__ __forceinline__ C cwsum_f(int op, const G& get, int p, int n, int i, int j, int k) {
    return op == 1 ? cwsum_q1_f<DIM, C>(get, p, n, i, j, k) : cnbsum_f<DIM, C>(get, p, n, i, j, k);
}

// Block-wide sum / max; every thread receives the result.  Fixed reduction
// tree (lane shuffles, then the warps' values in warp order): the same inputs
// give the same bits on every run.  All threads of the CTA must call.
template <class C>
__device__ __forceinline__ C block_sum(C v) {
    __shared__ C red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    v = (int)(threadIdx.x & 31) < (int)(blockDim.x >> 5) ? red[threadIdx.x & 31] : (C)0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    __syncthreads();  // red is reused by the next call
    return v;
}
template <class C>
__device__ __forceinline__ C block_max(C v) {
    __shared__ C red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(kFull, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    v = (int)(threadIdx.x & 31) < (int)(blockDim.x >> 5) ? red[threadIdx.x & 31] : (C)0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(kFull, v, o));
    __syncthreads();
    return v;
}

// ---- residual rescaling into an FP16 level (DSH_MG, Sec. 6)
// The shift k with m 2^k in [2^(sig-1), 2^sig) for the max-norm m of the
// restricted residual: the residual is multiplied by 2^k before the cast to
// FP16 (exact, a power of two) and the correction prolongated back from that
// level by 2^-k.  k = 0 for m = 0 or a non-finite m; |k| <= 126 so that both
// powers are normal FP32 numbers.
template <class C>
__device__ __forceinline__ int rescale_shift(C m, int sig) {
    if (!(m > (C)0) || !(m <= (C)3.0e38)) return 0;
    int e = 0;
    if constexpr (std::is_same<C, double>::value) (void)frexp(m, &e);
    else (void)frexpf(m, &e);  // m = f 2^e, f in [1/2, 1)
    return min(126, max(-126, sig - e));
}
// 2^k as IEEE binary32 / binary64 bit patterns, |k| <= 126
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }
__device__ __forceinline__ double pow2d(int k) { return __longlong_as_double((long long)(k + 1023) << 52); }

// ---- conjugate gradients on the base level (Sec. 6: CG base solver)
// A = alpha (beta I - W) of operator op on n^DIM compact points, from x = 0:
// x, r, p are stored in the level type T, A p (q) and the dot products are
// taken in the arithmetic type C.  Stops when
// ||r||_2 <= tol ||g||_2 (recursively updated r) or after maxit steps, or when
// p^T A p is not positive (breakdown, also for g = 0).  Called by every thread
// of one CTA; returns the steps taken.
template <int DIM, class T>
__device__ int cg_base(int n, unsigned long long mn, int op, typename Tr<T>::C alpha, typename Tr<T>::C beta,
                       const T* __restrict__ g, T* __restrict__ x, T* __restrict__ r, T* __restrict__ p,
                       typename Tr<T>::C* __restrict__ q, double tol, int maxit) {
    using C = typename Tr<T>::C;
    const int N = DIM == 3 ? n * n * n : n * n;
    C rr = 0;
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
        x[t] = T(0.0f);
        st1(r + t, cget(g, t));
        p[t] = r[t];
        const C v = cget(r, t);
        rr += v * v;
    }
    rr = block_sum<C>(rr);  // also orders the writes above before the first A p
    const C thr = (C)(tol * tol) * rr;
    int it = 0;
    while (it < maxit && rr > thr) {
        C pq = 0;
        for (int t = threadIdx.x; t < N; t += blockDim.x) {
            int i, j, k;
            decode<DIM>(t, n, mn, i, j, k);
            const C pv = cget(p, t);
            const C qv = alpha * (beta * pv - cwsum<DIM, T>(op, p, t, n, i, j, k));
            q[t] = qv;
            pq += pv * qv;
        }
        pq = block_sum<C>(pq);
        if (!(pq > (C)0)) break;
        const C a = rr / pq;
        C rn = 0;
        for (int t = threadIdx.x; t < N; t += blockDim.x) {
            st1(x + t, cget(x, t) + a * cget(p, t));
            st1(r + t, cget(r, t) - a * q[t]);
            const C v = cget(r, t);
            rn += v * v;
        }
        rn = block_sum<C>(rn);
        const C b = rn / rr;
        for (int t = threadIdx.x; t < N; t += blockDim.x) st1(p + t, cget(r, t) + b * cget(p, t));
        rr = rn;
        ++it;
        __syncthreads();  // p is read at the neighbours by the next A p
    }
    return it;
}

}  // namespace mgi
