// Kernel instantiations for the precession system with the Tsit5 pair (forward plain and persistent,
// reverse plain and persistent, all precision modes).
#include "gs_kernels.cuh"

namespace gs {
GS_DEFINE_METHOD(precession, Precession, Tsit5)
GS_DEFINE_RHS(precession, Precession)
}  // namespace gs
