// Kernel instantiations for the precession system (forward plain and persistent, reverse, rhs).
#include "gs_kernels.cuh"

namespace gs {
GS_DEFINE_SYSTEM(precession, Precession)
}  // namespace gs
