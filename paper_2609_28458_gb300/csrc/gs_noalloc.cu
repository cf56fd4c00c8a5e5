// gs_vjp_noalloc: the discrete-adjoint gradient for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or hand the library a workspace: code running inside another
// framework's memory pool that forbids foreign allocations, plug-ins loaded into a host that owns
// every device allocation, or a real-time loop where an allocation could stall or fail. For them this
// entry point keeps its scratch (work counters and the step tape) in a fixed array compiled into the
// library, so a call allocates nothing. The paper has no counterpart: it is an interface convenience.
//
// The array (GS_NOALLOC_SCRATCH_BYTES, 64 MiB) exists on every GPU that loads the library, from load
// until process exit. Host code cannot use the array's name as a device address, so the first call on
// each device looks the address up with cudaGetSymbolAddress (with that device current) and caches it;
// make that first call before any stream capture. All calls share the array and it keeps the previous
// call's contents: the call clears the counters that must start at zero, and every other byte it reads
// it has written first. Calls that overlap on the GPU (different streams, or different host threads
// on one device) race on the array; issue them one after another.
#include <cstdio>
#include <mutex>

#include <cuda_runtime.h>

#include "gs.h"

namespace gs {
int set_error(int code, const char* msg);  // defined in gs_api.cu
}

static __device__ __align__(256) unsigned char g_gs_noalloc_scratch[GS_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
void* g_scratch[kMaxDevices];
cudaError_t g_setup[kMaxDevices];
std::once_flag g_once[kMaxDevices];
}  // namespace

extern "C" int gs_vjp_noalloc(int32_t system, int64_t N, const double* y0, const double* params, const double* t0,
                              const double* t1, double rtol, double atol, int32_t K, const double* saveat,
                              const gs_options* opt, const double* dLdy, double* dLdy0, double* dLdparams,
                              double* y_out, int32_t* status, int32_t* n_accept, int32_t* n_reject,
                              void* cuda_stream) {
  char msg[256];
  int32_t d, p;
  if (gs_dims(system, &d, &p) != GS_OK) return GS_ERR_INVALID;  // gs_dims recorded the message
  if (!opt) return gs::set_error(GS_ERR_INVALID, "opt is NULL");
  if (opt->reuse_tape)
    return gs::set_error(GS_ERR_INVALID, "gs_vjp_noalloc re-runs the forward solve; reuse_tape must be 0");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    std::snprintf(msg, sizeof(msg), "cudaGetDevice: %s", cudaGetErrorString(e));
    return gs::set_error(GS_ERR_CUDA, msg);
  }
  if (dev < 0 || dev >= kMaxDevices) return gs::set_error(GS_ERR_INVALID, "device index above 63");
  // once per device, with that device current: the device address of the scratch array
  std::call_once(g_once[dev], [dev]() { g_setup[dev] = cudaGetSymbolAddress(&g_scratch[dev], g_gs_noalloc_scratch); });
  if (g_setup[dev] != cudaSuccess) {
    std::snprintf(msg, sizeof(msg), "cudaGetSymbolAddress of the scratch array: %s", cudaGetErrorString(g_setup[dev]));
    return gs::set_error(GS_ERR_CUDA, msg);
  }
  // the part before the tape pool (work counters, per-trajectory arrays and, with a checkpoint stride
  // above 1, the output attribution) plus one tape chunk must fit, the same test as gs_vjp's;
  // trajectories whose steps do not fit in the rest get GS_ST_TAPE_OVERFLOW. Sizes of 0 mean an
  // argument gs_vjp rejects (N < 0, K < 0, an unknown stride): it reports those itself.
  const size_t fixed = gs_workspace_bytes(system, N, K, opt, 1, 0.0);
  const size_t one_chunk = gs_tape_chunk_bytes(system, opt);
  if (N > 0 && fixed > 0 && one_chunk > 0 && fixed + one_chunk > size_t(GS_NOALLOC_SCRATCH_BYTES)) {
    std::snprintf(msg, sizeof(msg),
                  "N = %lld trajectories do not fit the %u-byte built-in scratch of gs_vjp_noalloc "
                  "(it needs %zu bytes with one tape chunk); use gs_vjp with a workspace",
                  (long long)N, (unsigned)GS_NOALLOC_SCRATCH_BYTES, fixed + one_chunk);
    return gs::set_error(GS_ERR_WORKSPACE, msg);
  }
  return gs_vjp(system, N, y0, params, t0, t1, rtol, atol, K, saveat, opt, dLdy, dLdy0, dLdparams, y_out, status,
                n_accept, n_reject, g_scratch[dev], size_t(GS_NOALLOC_SCRATCH_BYTES), cuda_stream);
}
