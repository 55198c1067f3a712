// Stencil march kernels instantiated for fine-level storage type __nv_bfloat16.
#include "mg_dispatch.cuh"

namespace mgi {
int launch_march_bf16(int dim, int mode, int loader, int prec_c, const KArgs& a, int gx, int gy, int gz,
                     int ty, size_t smem, void* stream) {
    return launch_march_t<__nv_bfloat16>(dim, mode, loader, prec_c, a, gx, gy, gz, ty, smem, stream);
}
}  // namespace mgi
