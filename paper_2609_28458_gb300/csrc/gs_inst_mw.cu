// Kernel instantiations for the mw system (forward plain and persistent, reverse, rhs).
#include "gs_kernels.cuh"

namespace gs {
GS_DEFINE_SYSTEM(mw, MilkyWay)
}  // namespace gs
