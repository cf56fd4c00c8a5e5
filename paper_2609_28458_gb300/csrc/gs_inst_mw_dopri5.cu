// Kernel instantiations for the mw system with the Dopri5 pair (forward plain and persistent,
// reverse plain and persistent, all precision modes).
#include "gs_kernels.cuh"

namespace gs {
GS_DEFINE_METHOD(mw, MilkyWay, Dopri5)

}  // namespace gs
