// Kernel instantiations for the quintessence system (forward plain and persistent, reverse, rhs).
#include "gs_kernels.cuh"

namespace gs {
GS_DEFINE_SYSTEM(quintessence, Quintessence)
}  // namespace gs
