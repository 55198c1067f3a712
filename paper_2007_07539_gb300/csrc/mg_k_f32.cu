// Stencil, update, scale-cast and prolongation kernels instantiated for the
// fine-level storage type float.
#include "mg_dispatch.cuh"

namespace mgi {
int launch_kernel_f32(int dim, int kind, int mode, int prec_c, const KArgs& a, const MarchShape& s,
                      const SweepMaps* maps, void* stream) {
    return launch_kernel_t<float>(dim, kind, mode, prec_c, a, s, maps, stream);
}
int occupancy_f32(int dim, int kind, int mode, int prec_c, int threads, size_t smem, int rpw) {
    return occupancy_t<float>(dim, kind, mode, prec_c, threads, smem, rpw);
}
int launch_kernel_batch_f32(int kind, int mode, int prec_c, int rpw, const void* items, const int* cta_item, int ncta,
                            int ty, size_t smem, void* stream) {
    return launch_batch_t<float>(kind, mode, prec_c, rpw, items, cta_item, ncta, ty, smem, stream);
}
}  // namespace mgi
