// C ABI of libgs.so (declared in include/gs.h): argument checks, workspace layout and dispatch to
// the per-system launchers. Nothing here allocates device memory; every call is stream-ordered.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "gs.h"
#include "gs_internal.h"
#include "gs_kernels.cuh"

namespace gs {
GS_DECLARE_SYSTEM(isochrone)
GS_DECLARE_SYSTEM(mw)
GS_DECLARE_SYSTEM(precession)
GS_DECLARE_SYSTEM(quintessence)
GS_DECLARE_SYSTEM(loghalo)
}  // namespace gs

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int dims_of(int32_t sys, int32_t* d, int32_t* p) {
  switch (sys) {
    case GS_SYS_ISOCHRONE: *d = 6; *p = 0; return 0;
    case GS_SYS_MW: *d = 6; *p = 4; return 0;
    case GS_SYS_PRECESSION: *d = 9; *p = 3; return 0;
    case GS_SYS_QUINTESSENCE: *d = 3; *p = 4; return 0;
    case GS_SYS_LOGHALO: *d = 6; *p = 3; return 0;
    default: return 1;
  }
}

int order_of(int32_t method) { return method == GS_VERN7 ? 7 : 5; }

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// tape slot (checkpoint stride 1): the state at the step's start (FP64, df64 pairs, or its FP32 high
// part), then the times: t, tc, h as FP64 from the next 8-byte boundary (24 bytes; h negative for
// the last step), or th, tl, h, flag as FP32 from the next 16-byte boundary (16 bytes, PM 2 and 3);
// padded to 16 bytes
long long slot_bytes(int32_t d, int32_t prec) {
  const long long state = (prec == GS_FP64 || prec == GS_DF64 ? 8LL : 4LL) * d;
  if (prec == GS_FP32_DF || prec == GS_DF64) return (state + 15) / 16 * 16 + 16;  // FP32 tail th, tl, h, flag
  return ((state + 7) / 8 * 8 + 24 + 15) / 16 * 16;  // FP64 tail t, tc, signed h
}
// checkpoint stride S > 1 (not PM 3): kChunk step lengths (FP64, FP32 in PM 2), then kChunk / S
// checkpoints: state and first stage (FP64: 16 d bytes; FP32 modes: high part, low part and first
// stage, 12 d bytes) padded to 16 bytes, then the time (16 bytes)
long long ckpt_bytes(int32_t d, int32_t prec) {
  const long long state = (prec == GS_FP64 ? 16LL : 12LL) * d;
  return (state + 15) / 16 * 16 + 16;
}
long long chunk_bytes(int32_t d, int32_t prec, int32_t stride) {
  if (stride > 1)
    return gs::kChunkHeader + gs::kChunk * (prec == GS_FP32_DF ? 4LL : 8LL) + (gs::kChunk / stride) * ckpt_bytes(d, prec);
  return gs::kChunkHeader + gs::kChunk * slot_bytes(d, prec);
}
int32_t stride_of(const gs_options* opt) { return (opt && opt->ckpt_stride > 1) ? opt->ckpt_stride : 1; }

// workspace: header (work counters), head[N], n_rec[N], a work list order[N] with its bucket
// counters and the estimated costs cost[N] (longest-first ordering of the forward and reverse
// launches), the prepared starts of the persistent forward start[N] (rows of start_row bytes)
// [= total_fixed], with a checkpoint stride above 1 the output attribution emit[N, K], then the
// tape pool
struct Layout {
  size_t header, head, nrec, order, buckets, cost, start, total_fixed, emit, pool;
};
long long start_row(int32_t system, int32_t precision) {
  switch (system) {
    case GS_SYS_ISOCHRONE: return gs::start_row_isochrone(precision);
    case GS_SYS_MW: return gs::start_row_mw(precision);
    case GS_SYS_PRECESSION: return gs::start_row_precession(precision);
    case GS_SYS_QUINTESSENCE: return gs::start_row_quintessence(precision);
    default: return gs::start_row_loghalo(precision);
  }
}
Layout layout(int64_t N, int32_t K, int32_t stride, long long row) {
  Layout L;
  L.header = 0;
  L.head = 256;
  L.nrec = L.head + align256(size_t(N) * 4);
  L.order = L.nrec + align256(size_t(N) * 4);
  L.buckets = L.order + align256(size_t(N) * 4);
  L.cost = L.buckets + align256(size_t(gs::kOrderBuckets) * 4);
  L.start = L.cost + align256(size_t(N) * 4);
  L.total_fixed = L.start + align256(size_t(N) * size_t(row));
  L.emit = L.total_fixed;
  L.pool = L.emit + (stride > 1 ? align256(size_t(N) * size_t(K > 0 ? K : 0) * 4) : 0);
  return L;
}

// Ordering of a forward launch (gs_options.order): the work list needs the workspace's fixed part.
// (order and cost_hint are validated by check_common)
int set_order(gs::Problem& pb, const gs_options* opt, int64_t N, void* ws, size_t ws_bytes, long long row) {
  const Layout L = layout(N, 0, 1, row);
  bool use = false;
  if (opt->order == GS_ORDER_HINT || opt->order == GS_ORDER_ESTIMATE) use = true;
  if (opt->order == GS_ORDER_AUTO) use = opt->cost_hint != nullptr || N >= 32768;
  if (!use) return GS_OK;
  if (!ws || ws_bytes < L.total_fixed) {
    if (opt->order == GS_ORDER_AUTO) return GS_OK;  // as stored
    return fail(GS_ERR_WORKSPACE, "a longest-first order needs a workspace of gs_workspace_bytes(..., for_vjp = 0) "
                "= %zu bytes", L.total_fixed);
  }
  unsigned char* base = static_cast<unsigned char*>(ws);
  pb.cost_hint = (opt->order == GS_ORDER_ESTIMATE) ? nullptr : opt->cost_hint;
  pb.ord_cost = reinterpret_cast<float*>(base + L.cost);
  pb.ord_order = reinterpret_cast<int32_t*>(base + L.order);
  pb.ord_cnt = reinterpret_cast<unsigned int*>(base + L.buckets);
  return GS_OK;
}

// Prepared starts of a persistent forward launch (modes 0-2): when the workspace holds the fixed part,
// else the persistent kernel starts trajectories in place.
void set_start(gs::Problem& pb, int kernel, int64_t N, void* ws, size_t ws_bytes, long long row) {
  if (kernel != GS_KERNEL_PERSISTENT || row <= 0 || !ws) return;
  const Layout L = layout(N, 0, 1, row);
  if (ws_bytes < L.total_fixed) return;
  pb.start = static_cast<unsigned char*>(ws) + L.start;
  pb.start_row = row;
}


typedef cudaError_t (*launch_fn)(const gs::Problem&, const gs::LaunchCfg&);
#define GS_PICK(kind, sysname)                                  \
  (method == GS_TSIT5 ? gs::kind##_##sysname##_Tsit5            \
   : method == GS_DOPRI5 ? gs::kind##_##sysname##_Dopri5        \
                         : gs::kind##_##sysname##_Vern7)
launch_fn forward_of(int32_t sys, int32_t method) {
  switch (sys) {
    case GS_SYS_ISOCHRONE: return GS_PICK(forward, isochrone);
    case GS_SYS_MW: return GS_PICK(forward, mw);
    case GS_SYS_PRECESSION: return GS_PICK(forward, precession);
    case GS_SYS_QUINTESSENCE: return GS_PICK(forward, quintessence);
    default: return GS_PICK(forward, loghalo);
  }
}
typedef cudaError_t (*jvp_fn)(const gs::Problem&, const gs::LaunchCfg&, int);
jvp_fn jvp_of(int32_t sys, int32_t method) {
  switch (sys) {
    case GS_SYS_ISOCHRONE: return GS_PICK(jvp, isochrone);
    case GS_SYS_MW: return GS_PICK(jvp, mw);
    case GS_SYS_PRECESSION: return GS_PICK(jvp, precession);
    case GS_SYS_QUINTESSENCE: return GS_PICK(jvp, quintessence);
    default: return GS_PICK(jvp, loghalo);
  }
}
launch_fn reverse_of(int32_t sys, int32_t method) {
  switch (sys) {
    case GS_SYS_ISOCHRONE: return GS_PICK(reverse, isochrone);
    case GS_SYS_MW: return GS_PICK(reverse, mw);
    case GS_SYS_PRECESSION: return GS_PICK(reverse, precession);
    case GS_SYS_QUINTESSENCE: return GS_PICK(reverse, quintessence);
    default: return GS_PICK(reverse, loghalo);
  }
}
#undef GS_PICK

int check_common(int32_t sys, int64_t N, const double* y0, const double* params, const double* t0,
                 const double* t1, double rtol, double atol, int32_t K, const double* saveat,
                 const gs_options* opt, int32_t* d, int32_t* p) {
  if (dims_of(sys, d, p)) return fail(GS_ERR_INVALID, "unknown system id %d", sys);
  if (!opt) return fail(GS_ERR_INVALID, "opt is NULL");
  if (N < 0) return fail(GS_ERR_INVALID, "N < 0");
  if (N > (int64_t(1) << 31) - 4096) return fail(GS_ERR_INVALID, "N too large (max 2^31 - 4096)");
  if (K < 0) return fail(GS_ERR_INVALID, "K < 0");
  if (opt->method < 0 || opt->method > 2) return fail(GS_ERR_INVALID, "unknown method %d", opt->method);
  if (opt->precision < 0 || opt->precision > 3) return fail(GS_ERR_INVALID, "unknown precision %d", opt->precision);
  if (opt->precision == GS_DF64 && sys != GS_SYS_ISOCHRONE && sys != GS_SYS_PRECESSION && sys != GS_SYS_LOGHALO)
    return fail(GS_ERR_INVALID, "GS_DF64 is available for the isochrone, precession and log-halo systems");
  if (opt->kernel < 0 || opt->kernel > 2) return fail(GS_ERR_INVALID, "unknown kernel %d", opt->kernel);
  if (opt->order < GS_ORDER_AUTO || opt->order > GS_ORDER_HINT) return fail(GS_ERR_INVALID, "unknown order %d", opt->order);
  if (opt->order == GS_ORDER_HINT && !opt->cost_hint) return fail(GS_ERR_INVALID, "GS_ORDER_HINT needs cost_hint");
  if (opt->block_size < 0 || opt->block_size > 128 || (opt->block_size % 32) != 0)
    return fail(GS_ERR_INVALID, "block_size must be 0 or a multiple of 32 up to 128");
  if (!(rtol >= 0.0) || !(atol >= 0.0) || !(rtol + atol > 0.0) || !std::isfinite(rtol) || !std::isfinite(atol))
    return fail(GS_ERR_INVALID, "tolerances must be finite, non-negative and not both zero");
  if (!(opt->safety > 0.0) || !(opt->alpha_min > 0.0) || !(opt->alpha_max >= opt->alpha_min))
    return fail(GS_ERR_INVALID, "controller: need safety > 0 and 0 < alpha_min <= alpha_max");
  if (opt->max_steps < 0) return fail(GS_ERR_INVALID, "max_steps < 0");
  if (opt->warp_lanes < 0 || opt->warp_lanes > 32) return fail(GS_ERR_INVALID, "warp_lanes must be 0..32");
  {
    const int32_t cs = opt->ckpt_stride;
    if (cs != 0 && cs != 1 && cs != 2 && cs != 4 && cs != 8 && cs != 16 && cs != 32)
      return fail(GS_ERR_INVALID, "ckpt_stride must be 0, 1, 2, 4, 8, 16 or 32");
  }
  if (N > 0) {
    if (!y0 || !t0 || !t1) return fail(GS_ERR_INVALID, "y0, t0 and t1 must not be NULL");
    if (*p > 0 && !params) return fail(GS_ERR_INVALID, "params must not be NULL for this system");
    if (K > 0 && !saveat) return fail(GS_ERR_INVALID, "saveat must not be NULL when K > 0");
  }
  return GS_OK;
}

gs::Problem make_problem(int64_t N, const double* y0, const double* params, const double* t0, const double* t1,
                         double rtol, double atol, int32_t K, const double* saveat, const gs_options* opt) {
  gs::Problem pb;
  std::memset(&pb, 0, sizeof(pb));
  pb.N = N;
  pb.n_work = N;
  pb.K = K;
  pb.per_traj = opt->per_traj_saveat ? 1 : 0;
  pb.y0 = y0; pb.params = params; pb.t0 = t0; pb.t1 = t1; pb.saveat = saveat;
  pb.rtol = rtol; pb.atol = atol;
  pb.max_steps = opt->max_steps;
  pb.safety = opt->safety; pb.alpha_min = opt->alpha_min; pb.alpha_max = opt->alpha_max;
  pb.beta1 = opt->beta1 > 0.0 ? opt->beta1 : 1.0 / order_of(opt->method);
  pb.beta2 = opt->beta2;
  pb.h0 = opt->h0;
  pb.warp_lanes = opt->warp_lanes > 0 ? opt->warp_lanes : 32;
  pb.fsafety = float(pb.safety);
  pb.falpha_min = float(pb.alpha_min);
  pb.falpha_max = float(pb.alpha_max);
  pb.fbeta1 = float(pb.beta1);
  pb.fbeta2 = float(pb.beta2);
  return pb;
}

int set_tape(gs::Problem& pb, int32_t d, const gs_options* opt, int64_t N, int32_t K, void* ws, size_t ws_bytes,
             long long row) {
  if (opt->tape_capacity <= 0) return fail(GS_ERR_INVALID, "tape_capacity must be positive");
  const int32_t stride = stride_of(opt);
  if (stride > 1 && opt->precision == GS_DF64)
    return fail(GS_ERR_INVALID, "checkpoint strides above 1 are not available in GS_DF64");
  if (stride > 1 && opt->kernel == GS_KERNEL_PLAIN)
    return fail(GS_ERR_INVALID, "checkpoint strides above 1 run in the persistent kernels (kernel auto or persistent)");
  Layout L = layout(N, K, stride, row);
  const long long cb = chunk_bytes(d, opt->precision, stride);
  if (!ws) return fail(GS_ERR_WORKSPACE, "this call needs a workspace (see gs_workspace_bytes)");
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return fail(GS_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  if (ws_bytes < L.pool + size_t(cb))
    return fail(GS_ERR_WORKSPACE, "workspace of %zu bytes is smaller than the %zu needed for N = %lld", ws_bytes,
                size_t(L.pool + cb), (long long)N);
  unsigned char* base = static_cast<unsigned char*>(ws);
  pb.tape.stride = stride;
  pb.tape.emit = stride > 1 ? reinterpret_cast<int32_t*>(base + L.emit) : nullptr;
  pb.tape.verify = (stride > 1 && opt->ckpt_verify) ? reinterpret_cast<unsigned int*>(base + 16) : nullptr;
  pb.tape.pool = base + L.pool;
  pb.tape.chunk_bytes = cb;
  pb.tape.cap = opt->tape_capacity;
  pb.tape.pool_chunks = (long long)((ws_bytes - L.pool) / size_t(cb));
  if (pb.tape.pool_chunks > 0x7fffffffLL) pb.tape.pool_chunks = 0x7fffffffLL;
  pb.tape.pool_next = reinterpret_cast<unsigned long long*>(base + 8);
  pb.tape.head = reinterpret_cast<int32_t*>(base + L.head);
  pb.tape.n_rec = reinterpret_cast<int32_t*>(base + L.nrec);
  return GS_OK;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(GS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace

namespace gs {
// error reporting for entry points defined in other translation units
int set_error(int code, const char* msg) { return fail(code, "%s", msg); }
}  // namespace gs

extern "C" {

void gs_default_options(gs_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->method = GS_TSIT5;
  o->precision = GS_FP64;
  o->kernel = GS_KERNEL_AUTO;
  o->max_steps = 1000000;
  o->safety = 0.9;
  o->alpha_min = 0.2;
  o->alpha_max = 5.0;
  o->beta1 = 0.0;
  o->beta2 = 0.0;
  o->h0 = 0.0;
  o->tape_capacity = 1000000;
  o->sm_limit = 0;
  o->graph_safe = 0;
}

int gs_dims(int32_t system, int32_t* d, int32_t* p) {
  if (!d || !p) return fail(GS_ERR_INVALID, "d and p must not be NULL");
  if (dims_of(system, d, p)) return fail(GS_ERR_INVALID, "unknown system id %d", system);
  return GS_OK;
}

size_t gs_workspace_bytes(int32_t system, int64_t N, int32_t K, const gs_options* opt, int32_t for_vjp,
                          double steps_hint) {
  int32_t d, p;
  if (dims_of(system, &d, &p) || N < 0 || K < 0) return 0;
  const int32_t stride = stride_of(opt);
  Layout L = layout(N, K, stride, start_row(system, opt ? opt->precision : GS_FP64));
  if (!for_vjp) return L.total_fixed;
  if (!(steps_hint > 0.0)) return L.pool;
  const double chunks = double(N) * (std::ceil(steps_hint / gs::kChunk) + 1.0) + 1.0;
  return L.pool + size_t(chunks) * size_t(chunk_bytes(d, opt ? opt->precision : GS_FP64, stride));
}

size_t gs_tape_chunk_bytes(int32_t system, const gs_options* opt) {
  int32_t d, p;
  if (dims_of(system, &d, &p)) return 0;
  const int32_t cs = opt ? opt->ckpt_stride : 0;
  if (cs != 0 && cs != 1 && cs != 2 && cs != 4 && cs != 8 && cs != 16 && cs != 32) return 0;
  return size_t(chunk_bytes(d, opt ? opt->precision : GS_FP64, stride_of(opt)));
}

int gs_solve(int32_t system, int64_t N, const double* y0, const double* params, const double* t0,
             const double* t1, double rtol, double atol, int32_t K, const double* saveat,
             const gs_options* opt, double* y_out, int32_t* status, int32_t* n_accept, int32_t* n_reject,
             void* workspace, size_t workspace_bytes, void* cuda_stream) {
  int32_t d, p;
  int rc = check_common(system, N, y0, params, t0, t1, rtol, atol, K, saveat, opt, &d, &p);
  if (rc) return rc;
  if (N > 0 && ((K > 0 && !y_out) || !status || !n_accept || !n_reject))
    return fail(GS_ERR_INVALID, "outputs must not be NULL");
  if (N == 0) return GS_OK;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  gs::Problem pb = make_problem(N, y0, params, t0, t1, rtol, atol, K, saveat, opt);
  pb.y_out = y_out; pb.status = status; pb.n_acc = n_accept; pb.n_rej = n_reject;
  const int kernel = opt->kernel == GS_KERNEL_AUTO ? GS_KERNEL_PERSISTENT : opt->kernel;
  const bool need_ws = kernel == GS_KERNEL_PERSISTENT || opt->record_tape;
  if (need_ws) {
    if (!workspace) return fail(GS_ERR_WORKSPACE, "the persistent kernel and tape recording need a workspace");
    if (workspace_bytes < 256) return fail(GS_ERR_WORKSPACE, "workspace smaller than 256 bytes");
    if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return fail(GS_ERR_WORKSPACE, "workspace must be 256-byte aligned");
    pb.queue = static_cast<unsigned int*>(workspace);
  }
  const long long row = start_row(system, opt->precision);
  if (opt->record_tape) {
    rc = set_tape(pb, d, opt, N, K, workspace, workspace_bytes, row);
    if (rc) return rc;
    pb.record = 1;
  }
  rc = set_order(pb, opt, N, workspace, workspace_bytes, row);
  if (rc) return rc;
  if (need_ws) set_start(pb, kernel, N, workspace, workspace_bytes, row);
  if (need_ws) {
    cudaError_t e = cudaMemsetAsync(workspace, 0, 256, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  }
  gs::LaunchCfg c{opt->method, opt->precision, kernel, opt->block_size, s, opt->sm_limit};
  cudaError_t e = forward_of(system, opt->method)(pb, c);
  if (e != cudaSuccess) return cuda_fail(e, "forward launch");
  return GS_OK;
}

int gs_vjp(int32_t system, int64_t N, const double* y0, const double* params, const double* t0,
           const double* t1, double rtol, double atol, int32_t K, const double* saveat, const gs_options* opt,
           const double* dLdy, double* dLdy0, double* dLdparams, double* y_out, int32_t* status,
           int32_t* n_accept, int32_t* n_reject, void* workspace, size_t workspace_bytes, void* cuda_stream) {
  int32_t d, p;
  int rc = check_common(system, N, y0, params, t0, t1, rtol, atol, K, saveat, opt, &d, &p);
  if (rc) return rc;
  if (N > 0 && ((K > 0 && !dLdy) || !dLdy0 || (p > 0 && !dLdparams) || !status || !n_accept || !n_reject))
    return fail(GS_ERR_INVALID, "dLdy, dLdy0, dLdparams, status and step counts must not be NULL");
  if (N == 0) return GS_OK;
  if (!opt->reuse_tape && K > 0 && !y_out)
    return fail(GS_ERR_INVALID, "y_out must not be NULL when the forward solve is re-run");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  gs::Problem pb = make_problem(N, y0, params, t0, t1, rtol, atol, K, saveat, opt);
  pb.y_out = y_out; pb.status = status; pb.n_acc = n_accept; pb.n_rej = n_reject;
  const long long row = start_row(system, opt->precision);
  rc = set_tape(pb, d, opt, N, K, workspace, workspace_bytes, row);
  if (rc) return rc;
  rc = set_order(pb, opt, N, workspace, workspace_bytes, row);  // of the forward re-solve
  if (rc) return rc;
  pb.queue = static_cast<unsigned int*>(workspace);
  pb.dLdy = dLdy; pb.dLdy0 = dLdy0; pb.dLdp = dLdparams;
  const int kernel = opt->kernel == GS_KERNEL_AUTO ? GS_KERNEL_PERSISTENT : opt->kernel;
  gs::LaunchCfg c{opt->method, opt->precision, kernel, opt->block_size, s, opt->sm_limit};
  if (!opt->reuse_tape) {
    cudaError_t e = cudaMemsetAsync(workspace, 0, 256, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    set_start(pb, kernel, N, workspace, workspace_bytes, row);
    pb.record = 1;
    e = forward_of(system, opt->method)(pb, c);
    if (e != cudaSuccess) return cuda_fail(e, "forward launch");
  }
  pb.record = 0;
  pb.start = nullptr;
  // the reverse pass takes its work-queue counter from header bytes [4, 8)
  pb.queue = reinterpret_cast<unsigned int*>(static_cast<unsigned char*>(workspace) + 4);
  if (kernel == GS_KERNEL_PERSISTENT) {
    cudaError_t e0 = cudaMemsetAsync(pb.queue, 0, 4, s);
    if (e0 != cudaSuccess) return cuda_fail(e0, "cudaMemsetAsync");
  }
  if (opt->order != GS_ORDER_NATURAL) {  // longest-first order of the reverse pass, by the recorded step counts
    const Layout L = layout(N, K, stride_of(opt), row);
    unsigned char* base = static_cast<unsigned char*>(workspace);
    int32_t* order = reinterpret_cast<int32_t*>(base + L.order);
    const cudaError_t e1 = gs::build_order((long long)N, nullptr, pb.tape.n_rec,
                                           reinterpret_cast<unsigned int*>(base + L.buckets), order, s);
    if (e1 != cudaSuccess) return cuda_fail(e1, "order launch");
    pb.work = order;
    pb.n_work = N;
    pb.ord_order = nullptr;
  }
  cudaError_t e = reverse_of(system, opt->method)(pb, c);
  if (e != cudaSuccess) return cuda_fail(e, "reverse launch");
  return GS_OK;
}

int gs_jvp(int32_t system, int64_t N, const double* y0, const double* params, const double* t0,
           const double* t1, double rtol, double atol, int32_t K, const double* saveat, const gs_options* opt,
           int32_t m, const double* dy0, const double* dparams, double* y_out, double* S_out, int32_t* status,
           int32_t* n_accept, int32_t* n_reject, void* workspace, size_t workspace_bytes, void* cuda_stream) {
  return gs::jvp_on(system, N, y0, params, t0, t1, rtol, atol, K, saveat, opt, m, dy0, dparams, y_out, S_out, status,
                    n_accept, n_reject, workspace, workspace_bytes, cuda_stream, nullptr, N, nullptr);
}

}  // extern "C"

namespace gs {

int jvp_on(int32_t system, int64_t N, const double* y0, const double* params, const double* t0, const double* t1,
           double rtol, double atol, int32_t K, const double* saveat, const gs_options* opt, int32_t m,
           const double* dy0, const double* dparams, double* y_out, double* S_out, int32_t* status, int32_t* n_accept,
           int32_t* n_reject, void* workspace, size_t workspace_bytes, void* cuda_stream, const int32_t* work,
           long long n_work, const unsigned int* n_work_dev) {
  int32_t d, p;
  int rc = check_common(system, N, y0, params, t0, t1, rtol, atol, K, saveat, opt, &d, &p);
  if (rc) return rc;
  if (m < 1) return fail(GS_ERR_INVALID, "m (number of sensitivity directions) must be >= 1");
  if (opt->precision == GS_FP32_STAGES || opt->precision == GS_DF64)
    return fail(GS_ERR_INVALID, "gs_jvp runs in GS_FP64 or GS_FP32_DF");
  if (N > 0 && ((K > 0 && (!y_out || !S_out)) || !status || !n_accept || !n_reject))
    return fail(GS_ERR_INVALID, "y_out, S_out, status and step counts must not be NULL");
  if (N == 0) return GS_OK;
  if (!workspace || workspace_bytes < 256 || reinterpret_cast<uintptr_t>(workspace) % 256 != 0)
    return fail(GS_ERR_WORKSPACE, "gs_jvp needs a 256-byte aligned workspace of at least 256 bytes");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  gs::Problem pb = make_problem(N, y0, params, t0, t1, rtol, atol, K, saveat, opt);
  pb.y_out = y_out; pb.status = status; pb.n_acc = n_accept; pb.n_rej = n_reject;
  pb.queue = static_cast<unsigned int*>(workspace);
  pb.dy0 = dy0; pb.dp = dparams; pb.S_out = S_out; pb.m_total = m;
  if (work) {
    if (n_work < 0 || n_work > N) return fail(GS_ERR_INVALID, "work list of %lld entries for N = %lld", n_work, (long long)N);
    pb.work = work;
    pb.n_work = n_work;
    pb.n_work_dev = n_work_dev;  // at most n_work entries (checked by the writer of the list)
  } else {
    rc = set_order(pb, opt, N, workspace, workspace_bytes, start_row(system, opt->precision));
    if (rc) return rc;
  }
  const int group = opt->method == GS_VERN7 ? 1 : 4;
  gs::LaunchCfg c{opt->method, opt->precision, GS_KERNEL_PERSISTENT, opt->block_size, s, opt->sm_limit};
  for (int32_t off = 0; off < m;) {
    const int32_t left = m - off;
    const int mt = left >= 4 && group >= 4 ? 4 : (left >= 2 && group >= 2 ? 2 : 1);
    pb.m_off = off;
    cudaError_t e = cudaMemsetAsync(workspace, 0, 256, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    e = jvp_of(system, opt->method)(pb, c, mt);
    if (e != cudaSuccess) return cuda_fail(e, "jvp launch");
    off += mt;
  }
  return GS_OK;
}

}  // namespace gs

extern "C" {

int gs_rhs(int32_t system, int32_t precision, int64_t M, const double* t, const double* y, const double* params,
           const double* w, double* f, double* gy, double* gp, void* cuda_stream) {
  int32_t d, p;
  if (dims_of(system, &d, &p)) return fail(GS_ERR_INVALID, "unknown system id %d", system);
  if (precision < 0 || precision > 2) return fail(GS_ERR_INVALID, "unknown precision %d", precision);
  if (M < 0) return fail(GS_ERR_INVALID, "M < 0");
  if (M == 0) return GS_OK;
  if (!t || !y || (p > 0 && !params)) return fail(GS_ERR_INVALID, "t, y (and params) must not be NULL");
  if ((gy || gp) && !w) return fail(GS_ERR_INVALID, "w must not be NULL when a VJP is requested");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e;
  switch (system) {
    case GS_SYS_ISOCHRONE: e = gs::rhs_isochrone(precision, M, t, y, params, w, f, gy, gp, s); break;
    case GS_SYS_MW: e = gs::rhs_mw(precision, M, t, y, params, w, f, gy, gp, s); break;
    case GS_SYS_PRECESSION: e = gs::rhs_precession(precision, M, t, y, params, w, f, gy, gp, s); break;
    case GS_SYS_QUINTESSENCE: e = gs::rhs_quintessence(precision, M, t, y, params, w, f, gy, gp, s); break;
    default: e = gs::rhs_loghalo(precision, M, t, y, params, w, f, gy, gp, s); break;
  }
  if (e != cudaSuccess) return cuda_fail(e, "rhs launch");
  return GS_OK;
}

const char* gs_last_error(void) { return g_err.c_str(); }

const char* gs_version(void) { return "gs-gb300 0.1 (sm_103a)"; }

}  // extern "C"
