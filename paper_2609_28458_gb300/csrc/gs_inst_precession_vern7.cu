// Kernel instantiations for the precession system with the Vern7 pair (forward plain and persistent,
// reverse plain and persistent, all precision modes).
#include "gs_kernels.cuh"

namespace gs {
GS_DEFINE_METHOD(precession, Precession, Vern7)

}  // namespace gs
