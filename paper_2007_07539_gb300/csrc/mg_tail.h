// Coarse-tail program: the stages of the multigrid cycle on the coarsest
// levels, executed in order by one thread-block cluster (mg_tail.cu).
#pragma once
#include "mg_internal.h"

namespace mgi {

constexpr int kTailThreads = 1024;
constexpr long long kTailMaxPoints = 32768;  // levels with n^d up to this run in the tail
constexpr int kTailMaxOps = 16384;

enum TailKind : int { TK_SWEEP = 0, TK_RESID = 1, TK_RESTRICT = 2, TK_PROLONG = 3, TK_COARSE = 4, TK_ZERO = 5 };

struct TailOp {
    int kind, mode, prec, prec_c;
    int n, P;
    long long S;
    int nc, Pc;
    long long Sc;
    const void* src;
    const void* g;
    void* dst;
    const void* coarse;
    void* scratch;
    double h2inv;
    double omega;
};

int launch_tail(int dim, const TailOp* prog, int nops, const double* minv, int m0, const DevState* st, int gate,
                void* stream);
int tail_cluster_size(int dim);

}  // namespace mgi
