// Entry points shared between the library's translation units (not part of the C ABI).
#pragma once
#include <cstdint>

#include "gs.h"

namespace gs {

// Records an error message for gs_last_error and returns `code`.
int set_error(int code, const char* msg);

// gs_jvp restricted to the trajectories work[0 .. n_work - 1] (all N when work is null); the
// outputs of the others are left untouched. With n_work_dev set, the list's length is read on the
// device from *n_work_dev (at most n_work) when the kernel starts.
int jvp_on(int32_t system, int64_t N, const double* y0, const double* params, const double* t0, const double* t1,
           double rtol, double atol, int32_t K, const double* saveat, const gs_options* opt, int32_t m,
           const double* dy0, const double* dparams, double* y_out, double* S_out, int32_t* status, int32_t* n_accept,
           int32_t* n_reject, void* workspace, size_t workspace_bytes, void* cuda_stream, const int32_t* work,
           long long n_work, const unsigned int* n_work_dev);

}  // namespace gs
