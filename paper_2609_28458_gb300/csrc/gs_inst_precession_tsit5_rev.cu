// Kernel instantiations for the precession system with the Tsit5 pair: reverse (discrete adjoint)
// plain and persistent, all precision modes.
#include "gs_kernels.cuh"

namespace gs {
GS_DEFINE_REVERSE(precession, Precession, Tsit5)

}  // namespace gs
