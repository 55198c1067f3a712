// Stencil march kernels instantiated for fine-level storage type __half.
#include "mg_dispatch.cuh"

namespace mgi {
int launch_march_f16(int dim, int mode, int loader, int prec_c, const KArgs& a, int gx, int gy, int gz,
                     int ty, size_t smem, void* stream) {
    return launch_march_t<__half>(dim, mode, loader, prec_c, a, gx, gy, gz, ty, smem, stream);
}
}  // namespace mgi
