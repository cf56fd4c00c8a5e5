// Kernel instantiations for the isochrone system with the Tsit5 pair (forward plain and persistent,
// reverse plain and persistent, all precision modes).
#include "gs_kernels.cuh"

namespace gs {
GS_DEFINE_METHOD(isochrone, Isochrone, Tsit5)
GS_DEFINE_RHS(isochrone, Isochrone)
}  // namespace gs
