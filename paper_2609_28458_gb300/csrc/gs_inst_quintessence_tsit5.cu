// Kernel instantiations for the quintessence system with the Tsit5 pair (forward plain and persistent,
// reverse plain and persistent, all precision modes).
#include "gs_kernels.cuh"

namespace gs {
GS_DEFINE_METHOD(quintessence, Quintessence, Tsit5)
GS_DEFINE_RHS(quintessence, Quintessence)
}  // namespace gs
