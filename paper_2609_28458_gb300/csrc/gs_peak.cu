// gs_alu_probe: the GPU's plain-ALU multiply-add throughput, measured rather than derived from unit
// counts and a nominal clock. The paper has no counterpart: the benchmark divides each ALU-bound
// kernel's algorithmic flop rate by this number to report its fraction of the FP32 or FP64 peak.
//
// kind 0: FP32, 1: FP64, 2: FP32 with the packed two-lane multiply-add (FFMA2, sm_100 and later).
// Every thread runs kChains independent multiply-add chains, x <- x * a + b, for `iters` rounds,
// so the FMA pipe always has independent work in flight; the grid is `blocks_per_sm` blocks of 256
// threads per SM. Each block writes one sum, so the work cannot be optimised away, and nothing else
// touches memory.
#include <cuda_runtime.h>

#include "gs.h"

namespace gs {
int set_error(int code, const char* msg);  // defined in gs_api.cu
}

namespace {
constexpr int kChains = 8;
constexpr int kThreads = 256;

__device__ void block_sum(double v, double* sink) {
  __shared__ double part[kThreads];
  part[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kThreads; k++) t += part[k];
    sink[blockIdx.x] = t;
  }
}

template <class R>
__global__ void __launch_bounds__(kThreads) k_fma_probe(long long iters, R a, R b, double* sink) {
  R x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) x[c] = R(threadIdx.x + c) * R(1e-3);
#pragma unroll 16
  for (long long i = 0; i < iters; i++) {  // unrolled: the loop's own instructions stay a few percent
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = x[c] * a + b;
  }
  R s = R(0);
#pragma unroll
  for (int c = 0; c < kChains; c++) s += x[c];
  block_sum(double(s), sink);
}

// The same with the packed two-lane FP32 multiply-add of sm_100 and later (FFMA2): kChains chains of
// float2, two multiply-adds per instruction.
__global__ void __launch_bounds__(kThreads) k_fma2_probe(long long iters, float a, float b, double* sink) {
  float2 x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) x[c] = make_float2(float(threadIdx.x + c) * 1e-3f, float(threadIdx.x - c) * 1e-3f);
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll 16
  for (long long i = 0; i < iters; i++) {
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = __ffma2_rn(x[c], a2, b2);
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; c++) s += x[c].x + x[c].y;
  block_sum(double(s), sink);
}
}  // namespace

extern "C" int gs_alu_probe(int32_t kind, int64_t iters, int32_t blocks_per_sm, double* sink, int64_t* fma_count,
                            void* cuda_stream) {
  if (kind < 0 || kind > 2 || iters < 1 || blocks_per_sm < 1 || blocks_per_sm > 8 || !sink || !fma_count)
    return gs::set_error(GS_ERR_INVALID,
                         "gs_alu_probe: need kind 0..2, iters >= 1, 1 <= blocks_per_sm <= 8, sink and fma_count");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return gs::set_error(GS_ERR_CUDA, cudaGetErrorString(e));
  const int grid = sms * blocks_per_sm;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // a and b keep every chain bounded (|a| < 1): no overflow, no denormals
  if (kind == 1) k_fma_probe<double><<<grid, kThreads, 0, s>>>(iters, 0.9999, 1e-4, sink);
  else if (kind == 2) k_fma2_probe<<<grid, kThreads, 0, s>>>(iters, 0.9999f, 1e-4f, sink);
  else k_fma_probe<float><<<grid, kThreads, 0, s>>>(iters, 0.9999f, 1e-4f, sink);
  e = cudaGetLastError();
  if (e != cudaSuccess) return gs::set_error(GS_ERR_CUDA, cudaGetErrorString(e));
  *fma_count = int64_t(grid) * kThreads * kChains * iters * (kind == 2 ? 2 : 1);
  return GS_OK;
}
