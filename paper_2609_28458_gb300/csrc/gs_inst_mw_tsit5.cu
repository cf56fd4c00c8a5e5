// Kernel instantiations for the mw system with the Tsit5 pair (forward plain and persistent,
// reverse plain and persistent, all precision modes).
#include "gs_kernels.cuh"

namespace gs {
GS_DEFINE_METHOD(mw, MilkyWay, Tsit5)
GS_DEFINE_RHS(mw, MilkyWay)
}  // namespace gs
