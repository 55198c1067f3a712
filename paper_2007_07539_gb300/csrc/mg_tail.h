// Coarse-tail program: the stages of the multigrid cycle on the coarsest
// levels, executed in order by one CTA (or one thread-block cluster) with every
// tail level held in shared memory (kernels: mg_tail_body.cuh; launches:
// mg_tail.cu).
#pragma once
#include "mg_internal.h"

namespace mgi {

constexpr int kTailThreads = 1024;
constexpr long long kTailMaxPoints = 8192;     // single-CTA tail: levels with n^d up to this
constexpr long long kTailMaxPointsCl = 1 << 15;  // cluster tail: levels with n^d up to this
constexpr size_t kTailMaxSmem = 200 * 1024;    // shared-memory budget of the tail's level arrays (per CTA)
constexpr int kTailMaxOps = 16384;
constexpr int kTailMaxCluster = 16;            // CTAs of a cluster tail
constexpr int kTailWholeShift = 30;            // chunk shift of a single-CTA tail (one chunk)

enum TailKind : int {
    TK_SWEEP = 0,     // Jacobi family (mode M_JACOBI / M_ZERO2 / M_ZERO1) on level n
    TK_RESID = 1,     // scratch r = g - A c (arithmetic type)
    TK_RESTRICT = 2,  // coarse g = R r (cast to the coarse storage type)
    TK_PROLONG = 3,   // c += P c_coarse
    TK_COARSE = 4,    // c = A0^-1 g (mode 0: dense inverse; mode 1: CG, scratch at src)
    TK_ZERO = 5,      // c = 0
    TK_LOAD = 6,      // shared array <- padded global array
    TK_STORE = 7      // padded global array <- shared array
};

// One stage.  src / g / dst / coarse are byte offsets into the kernel's
// dynamic shared memory, where level arrays are compact (x fastest, n^d
// values, no pads); gptr is the padded global array of TK_LOAD / TK_STORE.
// mn / mnc are ceil(2^40 / n) and ceil(2^40 / nc): q = (p * mn) >> 40 is p / n
// for every point p of a tail level, p < 2^15 (division by an invariant integer
// through a fixed-point reciprocal, exact because p * (mn - 2^40 / n) < p <
// 2^40 / n for n < 2^10).
struct TailOp {
    int kind, mode, prec, prec_c;
    int n, nc, P, S;
    int src, g, dst, coarse;
    unsigned long long mn, mnc;
    int sslot;  // TK_RESTRICT / TK_PROLONG into / from a rescaled FP16 level: byte offset of its scale, else -1
    int scr2;   // TK_RESTRICT with sslot >= 0: byte offset of the coarse-value scratch
    int rsig;   // TK_RESTRICT with sslot >= 0: target max-norm 2^rsig (power-of-two range)
    int cgmax;  // TK_COARSE mode 1 (CG): step limit
    int op;     // operator: 0 finite differences, 1 Q1 elements
    int sh;     // chunk shift of level n: point p lives in CTA p >> sh of the cluster
    int shc;    // chunk shift of the coarser level nc
    int pad_;
    void* gptr;
    double h2inv;
    double omega;
    double cgtol;  // TK_COARSE mode 1: relative residual tolerance
    SweepCoef cf;  // host-computed sweep coefficients of level n
};
static_assert(sizeof(TailOp) % 8 == 0, "TailOp is copied as 8-byte words");
constexpr int kTailOpWords = (int)(sizeof(TailOp) / 8);
constexpr int kTailChunk = 32;  // stages staged in shared memory at a time

inline unsigned long long tail_magic(int n) { return ((1ull << 40) + (unsigned long long)n - 1) / (unsigned long long)n; }

// One instance of a batched tail launch (one CTA, or one cluster, each; gated
// on its state).
struct TailItem {
    const TailOp* prog;
    const double* minv;
    const DevState* st;
    int nops, m0;
};
int launch_tail_batch(int dim, int uniform_prec, const TailItem* items, int nitems, size_t smem, int cs,
                      void* stream);

// The tail kernels of one dimension, one CTA (CL false) or a cluster (CL
// true), for a uniform tail storage type or -1 (mixed precisions); each
// (DIM, CL) is instantiated in its own translation unit.
using TailFn = void (*)(const TailOp*, int, const double*, int, const DevState*, int, int, TailOp);
using TailBatchFn = void (*)(const TailItem*, int);
template <int DIM, bool CL>
TailFn tail_kernel(int uniform_prec);
template <int DIM, bool CL>
TailBatchFn tail_batch_kernel(int uniform_prec);

// uniform_prec: the storage type of every tail level (selects a kernel
// specialised for it), or -1 for a mixed-precision tail.
// cs: CTAs of the thread-block cluster that holds the tail levels (1: one CTA).
// first: host copy of prog[0] (or nullptr), passed by value so that a one-CTA
// tail starts its first load without waiting for the program's own fetch.
int launch_tail(int dim, int uniform_prec, const TailOp* prog, int nops, const double* minv, int m0,
                const DevState* st, int gate, size_t smem, int cs, void* stream, const TailOp* first = nullptr);
// Active clusters of cs tail CTAs with smem bytes each this device can hold (0: none / no device).
int tail_cluster_ok(int dim, int uniform_prec, int cs, size_t smem);

}  // namespace mgi
