// Kernel instantiations for the isochrone system (forward plain and persistent, reverse, rhs).
#include "gs_kernels.cuh"

namespace gs {
GS_DEFINE_SYSTEM(isochrone, Isochrone)
}  // namespace gs
