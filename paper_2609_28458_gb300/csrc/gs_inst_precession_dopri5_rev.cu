// Kernel instantiations for the precession system with the Dopri5 pair: reverse (discrete adjoint)
// plain and persistent, all precision modes.
#include "gs_kernels.cuh"

namespace gs {
GS_DEFINE_REVERSE(precession, Precession, Dopri5)

}  // namespace gs
