// Kernel instantiations for the precession system with the Vern7 pair: forward plain and persistent
// and forward sensitivities, all precision modes (the reverse kernels are in the _rev unit).
#include "gs_kernels.cuh"

namespace gs {
GS_DEFINE_FORWARD_JVP(precession, Precession, Vern7)

}  // namespace gs
