// Kernel instantiations for the loghalo system (forward plain and persistent, reverse, rhs).
#include "gs_kernels.cuh"

namespace gs {
GS_DEFINE_SYSTEM(loghalo, LogHalo)
}  // namespace gs
