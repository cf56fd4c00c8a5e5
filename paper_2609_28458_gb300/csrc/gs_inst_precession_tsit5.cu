// Kernel instantiations for the precession system with the Tsit5 pair: forward plain and persistent
// and forward sensitivities, all precision modes (the reverse kernels are in the _rev unit).
#include "gs_kernels.cuh"

namespace gs {
GS_DEFINE_FORWARD_JVP(precession, Precession, Tsit5)
GS_DEFINE_RHS(precession, Precession)
}  // namespace gs
