// IR control of libmgfp: the fixed-order reduction of the residual-norm
// partials and the stopping test / next scale of Alg. 2, shared by the
// stand-alone finalisation kernel and the IR update, whose last CTA runs it.
#pragma once
#include <cmath>

#include "mg_device.cuh"

namespace mgi {

// ---------------------------------------------------------------- norms and IR control
// Reduces per-CTA partials in a fixed order (deterministic), then applies the
// stopping test of Alg. 2 and sets alpha for the next step's residual scaling:
// alpha = ||r||_inf / sigma (scaling 1), ||r||_2 / sigma (scaling 2) or 1.
// kind: FIN_INIT after r = b - A u0, FIN_STEP after an update (partials of
// stride 2), FIN_GUARD after the true residual, 3 = report only.
__device__ __forceinline__ void finalize_body(int kind, DevState* st, const double* __restrict__ partials, int nblocks) {
    // gating (uniform across the block): a step's finalisation only while
    // iterating, the true-residual check only when it is pending, the report
    // only when u changed since it was last copied out
    if (kind == FIN_STEP && st->phase != 0) return;
    if (kind == FIN_GUARD && st->phase != 1) return;
    if (kind == FIN_REPORT && !st->dirty) return;
    const int stride = kind == FIN_STEP ? 2 : 4;
    double sr = 0.0, sb = 0.0;
    unsigned long long mr = 0ull;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        sr += partials[(long long)stride * b];
        unsigned long long m = (unsigned long long)__double_as_longlong(partials[(long long)stride * b + 1]);
        mr = m > mr ? m : mr;
        if (stride == 4) sb += partials[(long long)stride * b + 2];
    }
    __shared__ double s1[32], s2[32];
    __shared__ unsigned long long s3[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    sr = warp_sum(sr); sb = warp_sum(sb); mr = warp_max(mr);
    if (lane == 0) { s1[wid] = sr; s2[wid] = sb; s3[wid] = mr; }
    __syncthreads();
    if (wid != 0) return;
    sr = lane < nw ? s1[lane] : 0.0;
    sb = lane < nw ? s2[lane] : 0.0;
    mr = lane < nw ? s3[lane] : 0ull;
    sr = warp_sum(sr); sb = warp_sum(sb); mr = warp_max(mr);
    if (lane != 0) return;
    const double rn = sqrt(sr);
    const double rinf = __longlong_as_double((long long)mr);
    // scale-ahead: did this step's update write the next g (with inv_pred, no overflow)?
    const bool ahead_ok = kind == FIN_STEP && st->scale_ahead && !st->gover && st->inv_pred > 0.0;
    const double inv_used = st->inv_pred;
    st->gover = 0;
    st->g_ready = 0;
    if (kind == FIN_INIT) {
        st->bnorm2 = sqrt(sb);
        st->tol_abs = st->tol_mode == 0 ? st->tol * st->bnorm2 : st->tol;
        st->iter = 0;
        st->guard_restarts = 0;
        st->stag = 0;
        st->status = MG_OK;
        st->dirty = 1;
    }
    const double bn = st->bnorm2;
    const double rel = bn > 0.0 ? rn / bn : rn;
    if (kind == FIN_REPORT) {  // report only: u has been copied out
        st->rel_true = rel;
        st->dirty = 0;
        return;
    }
    if (kind == FIN_STEP) {
        st->iter += 1;
        st->dirty = 1;
        st->stag = (rn >= 0.999 * st->rnorm2) ? st->stag + 1 : 0;
    }
    if (kind == FIN_GUARD) st->dirty = 0;
    st->rnorm2 = rn;
    st->rnorminf = rinf;
    const int it = st->iter < kMaxHist ? st->iter : kMaxHist;
    st->hist[it] = rel;
    if (kind == FIN_GUARD) st->rel_true = rel;
    if (!isfinite(rn) || !isfinite(rinf)) {
        st->phase = 3;
        st->status = MG_ERR_NUMERIC;
        return;
    }
    if (rn <= st->tol_abs) {
        if (kind == FIN_GUARD || !st->guard) {
            st->phase = 2;
            st->status = MG_OK;
            return;
        }
        st->phase = 1;
        return;
    }
    if (kind == FIN_GUARD) st->guard_restarts += 1;
    if (st->iter >= st->max_iter || st->stag >= 5) {
        st->phase = 3;
        st->status = MG_ERR_NOT_CONVERGED;
        return;
    }
    double alpha = 1.0, inv = 1.0;
    if (st->scaling == 1) { alpha = rinf / st->sigma; inv = st->sigma / rinf; }
    else if (st->scaling == 2) { alpha = rn / st->sigma; inv = st->sigma / rn; }
    if (ahead_ok) {  // g = cast(r inv_used) is in place: alpha = 1 / inv_used (powers of two, exact)
        int e = 0;
        (void)frexp(inv_used, &e);
        alpha = ldexp(1.0, 1 - e);
        inv = inv_used;
        st->g_ready = 1;
    }
    st->alpha = alpha;
    st->inv = inv;
    if (st->scale_ahead && rinf > 0.0) {  // the next update's scale: sigma / 2^e, 2^e > ||r||_inf >= 2^(e-1)
        int e = 0;
        (void)frexp(rinf, &e);
        st->inv_pred = ldexp(st->sigma, -e);
    }
    st->phase = 0;
}

}  // namespace mgi
