// Cluster coarse-tail kernels of 3D hierarchies (one translation unit
// per dimension and tail shape, so that they compile in parallel).
#include "mg_tail_body.cuh"

namespace mgi {
template TailFn tail_kernel<3, true>(int);
template TailBatchFn tail_batch_kernel<3, true>(int);
}  // namespace mgi
