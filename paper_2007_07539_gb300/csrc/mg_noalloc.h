// Host-side argument checks of mg_residual_norms_noalloc (header-only, so the
// host compiler can test them without a device).
#pragma once

namespace mgi {

// Where a pointer given to the no-allocation entry point may live, from the
// fields of cudaPointerAttributes (type: 0 unregistered, 1 host, 2 device,
// 3 managed; ptr_device: the device of a device allocation) and the device
// current at the call.  0: usable by kernels on the current device (its own
// device memory, or managed memory); 1: not device memory (host or unknown);
// 2: device memory of another device, which the kernels cannot read without
// peer access.
inline int noalloc_ptr_class(int type, int ptr_device, int current_device) {
    if (type == 3) return 0;
    if (type == 2) return ptr_device == current_device ? 0 : 2;
    return 1;
}

}  // namespace mgi
