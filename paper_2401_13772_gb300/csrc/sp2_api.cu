// C ABI of the SP2 solver: argument checks, per-(device, stream) workspace
// cache, the device-driven iteration loop (a CUDA graph with a WHILE node)
// and readback of the solve state.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <utility>

#include "progress_sp2.h"
#include "sp2_common.cuh"
#include "sp2_launch.h"
#include "sp2_slices.cuh"

namespace {

thread_local std::string g_err = "";

progress_status_t fail(progress_status_t s, const char* what) {
  g_err = what;
  return s;
}

progress_status_t cuda_fail(cudaError_t e, const char* where) {
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
  g_err = buf;
  cudaGetLastError();  // clear a sticky-free error so later calls start clean
  return e == cudaErrorMemoryAllocation ? PROGRESS_ENOMEM : PROGRESS_ECUDA;
}

#define CK(call, where)                              \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

struct Workspace {
  int device = -1;
  cudaStream_t stream = nullptr;
  int ld_cap = 0;       // ld the matrix buffers were sized for
  int x64_cap = 0;      // ld of the FP64 ping-pong buffers (0 = none)
  int slices_cap = 0;   // slices per set that are allocated
  int digits_cap = 0;   // ld of the digit planes (0 = none)
  size_t flags_cap = 0; // bytes of each tile-flag array (thresholded SP2)
  sp2::DevBuffers buf{};
  sp2::State* h_state = nullptr;  // pinned host mirror for readback
  cudaStream_t cap_stream = nullptr;
  // cached loop graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int g_ld = -1, g_prec = -1, g_fmt = -1, g_df = -1, g_oz = -1, g_tile = -1;
  float g_tau = -1.0f;
};

std::mutex g_mu;
std::map<std::pair<int, cudaStream_t>, Workspace*> g_ws;

void free_graph(Workspace* w) {
  if (w->exec) cudaGraphExecDestroy(w->exec);
  if (w->graph) cudaGraphDestroy(w->graph);
  w->exec = nullptr;
  w->graph = nullptr;
  w->g_ld = w->g_prec = w->g_fmt = w->g_df = w->g_oz = w->g_tile = -1;
  w->g_tau = -1.0f;
}

void free_matrices(Workspace* w) {
  for (int k = 0; k < 2; ++k) {
    if (w->buf.x64[k]) cudaFree(w->buf.x64[k]);
    w->buf.x64[k] = nullptr;
    for (int i = 0; i < 3; ++i) {
      if (w->buf.sl[k][i]) cudaFree(w->buf.sl[k][i]);
      w->buf.sl[k][i] = nullptr;
    }
  }
  for (int d = 0; d < 5; ++d) {
    if (w->buf.dg[d]) cudaFree(w->buf.dg[d]);
    w->buf.dg[d] = nullptr;
  }
  if (w->buf.partials) cudaFree(w->buf.partials);
  w->buf.partials = nullptr;
  w->buf.max_partials = 0;
  w->x64_cap = w->slices_cap = w->ld_cap = w->digits_cap = 0;
  for (int k = 0; k < 2; ++k) {
    if (w->buf.tflags[k]) cudaFree(w->buf.tflags[k]);
    w->buf.tflags[k] = nullptr;
  }
  w->flags_cap = 0;
}

// Tile-flag arrays of thresholded SP2 for order ld.
progress_status_t ensure_flags(Workspace* w, int ld) {
  const size_t t = (size_t)(ld / 128);
  if (w->flags_cap >= t * t && w->buf.tflags[0]) return PROGRESS_OK;
  CK(cudaStreamSynchronize(w->stream), "cudaStreamSynchronize");
  free_graph(w);  // the loop graph holds the old pointers
  for (int k = 0; k < 2; ++k) {
    if (w->buf.tflags[k]) cudaFree(w->buf.tflags[k]);
    w->buf.tflags[k] = nullptr;
  }
  w->flags_cap = 0;
  for (int k = 0; k < 2; ++k) CK(cudaMalloc(&w->buf.tflags[k], t * t), "tile flag allocation");
  w->flags_cap = t * t;
  return PROGRESS_OK;
}

void free_workspace(Workspace* w) {
  free_graph(w);
  free_matrices(w);
  if (w->buf.st) cudaFree(w->buf.st);
  if (w->h_state) cudaFreeHost(w->h_state);
  if (w->cap_stream) cudaStreamDestroy(w->cap_stream);
  delete w;
}

progress_status_t get_workspace(cudaStream_t s, Workspace** out) {
  int dev = 0;
  CK(cudaGetDevice(&dev), "cudaGetDevice");
  std::lock_guard<std::mutex> lk(g_mu);
  auto key = std::make_pair(dev, s);
  auto it = g_ws.find(key);
  if (it != g_ws.end()) {
    *out = it->second;
    return PROGRESS_OK;
  }
  Workspace* w = new Workspace();
  w->device = dev;
  w->stream = s;
  cudaError_t e = cudaMalloc(&w->buf.st, sizeof(sp2::State));
  if (e == cudaSuccess) e = cudaMallocHost(&w->h_state, sizeof(sp2::State));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&w->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemset(w->buf.st, 0, sizeof(sp2::State));
  if (e != cudaSuccess) {
    free_workspace(w);
    return cuda_fail(e, "workspace allocation");
  }
  g_ws[key] = w;
  *out = w;
  return PROGRESS_OK;
}

// Make sure the matrix buffers cover ld and the requested formats.
progress_status_t ensure_buffers(Workspace* w, int ld, bool need_x64, int nslices,
                                 bool need_digits = false) {
  const bool grow = ld > w->ld_cap || (need_x64 && w->x64_cap < ld) ||
                    (nslices > 0 && (w->slices_cap < nslices || w->ld_cap < ld)) ||
                    (need_digits && w->digits_cap < ld);
  if (!grow && w->buf.partials) return PROGRESS_OK;
  CK(cudaStreamSynchronize(w->stream), "cudaStreamSynchronize");
  const int new_ld = ld > w->ld_cap ? ld : w->ld_cap;
  const bool keep_x64 = w->x64_cap > 0;
  const bool keep_dg = w->digits_cap > 0;
  const int keep_sl = w->slices_cap;
  free_graph(w);
  free_matrices(w);
  const size_t elems = (size_t)new_ld * new_ld;
  const bool x64 = need_x64 || keep_x64;
  const bool dg = need_digits || keep_dg;
  const int ns = nslices > keep_sl ? nslices : keep_sl;
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    if (x64) e = cudaMalloc(&w->buf.x64[k], elems * sizeof(double));
    for (int i = 0; i < ns && e == cudaSuccess; ++i)
      e = cudaMalloc(&w->buf.sl[k][i], elems * sizeof(uint16_t));
  }
  if (dg && e == cudaSuccess) e = cudaMalloc(&w->buf.dg[0], 4 * elems * sizeof(uint16_t));
  if (dg && e == cudaSuccess) e = cudaMalloc(&w->buf.dg[4], elems * sizeof(uint16_t));
  int maxp = sp2::fp64_tile_count(new_ld);
  if (sp2::df64_tile_count(new_ld) > maxp) maxp = sp2::df64_tile_count(new_ld);
  const int sp = sp2::split_tile_count(new_ld);
  if (sp > maxp) maxp = sp;
  if (maxp < 152 * 8) maxp = 152 * 8;
  if (e == cudaSuccess) e = cudaMalloc(&w->buf.partials, (size_t)maxp * 2 * sizeof(double));
  if (e != cudaSuccess) {
    free_matrices(w);
    return cuda_fail(e, "workspace matrix allocation");
  }
  w->buf.max_partials = maxp;
  w->ld_cap = new_ld;
  w->x64_cap = x64 ? new_ld : 0;
  w->slices_cap = ns;
  w->digits_cap = dg ? new_ld : 0;
  return PROGRESS_OK;
}

bool is_mixed(int prec) { return prec == PROGRESS_MIXED_FP16 || prec == PROGRESS_MIXED_BF16; }

int slice_fmt_of(int prec, int fixed) {
  const bool bf16 = prec == PROGRESS_MIXED_BF16;
  if (fixed) return bf16 ? sp2::kBF16x3F : sp2::kFP16x2F;
  return bf16 ? sp2::kBF16x3 : sp2::kFP16x2;
}

// Queue the product steps of one loop iteration on `s`.
progress_status_t queue_steps(Workspace* w, const sp2::SolveParams& p, unsigned long long cond,
                              cudaStream_t s) {
  if (p.prec == PROGRESS_FP64 || is_mixed(p.prec)) {
    if (p.oz) {
      CK(sp2::launch_digits(w->buf, p.ld, s), "digits launch");
      CK(sp2::launch_square_oz(w->buf, p.ld, p.slice_fmt, cond, s), "square_oz launch");
    } else if (p.df64)
      CK(sp2::launch_square_df64(w->buf, p.ld, p.slice_fmt, cond, s), "square_df64 launch");
    else
      CK(sp2::launch_square_fp64(w->buf, p.ld, p.slice_fmt, cond, s), "square_fp64 launch");
  }
  if (p.prec != PROGRESS_FP64)
    CK(sp2::launch_square_split(w->buf, p, cond, s), "square_split launch");
  return PROGRESS_OK;
}

progress_status_t build_graph(Workspace* w, const sp2::SolveParams& p) {
  if (w->exec && w->g_ld == p.ld && w->g_prec == p.prec && w->g_fmt == p.slice_fmt &&
      w->g_df == p.df64 && w->g_oz == p.oz && w->g_tau == p.tau && w->g_tile == p.split_tile)
    return PROGRESS_OK;
  free_graph(w);
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0), "cudaGraphCreate");
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(e, "cudaGraphConditionalHandleCreate");
  }
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(e, "cudaGraphAddNode(conditional)");
  }
  cudaGraph_t body = np.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(w->cap_stream, body, nullptr, nullptr, 0,
                                    cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(e, "cudaStreamBeginCaptureToGraph");
  }
  progress_status_t qs = queue_steps(w, p, (unsigned long long)h, w->cap_stream);
  cudaGraph_t captured = nullptr;
  e = cudaStreamEndCapture(w->cap_stream, &captured);
  if (qs != PROGRESS_OK || e != cudaSuccess) {
    cudaGraphDestroy(g);
    return qs != PROGRESS_OK ? qs : cuda_fail(e, "cudaStreamEndCapture");
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(e, "cudaGraphInstantiate");
  }
  w->graph = g;
  w->exec = exec;
  w->g_ld = p.ld;
  w->g_prec = p.prec;
  w->g_fmt = p.slice_fmt;
  w->g_df = p.df64;
  w->g_oz = p.oz;
  w->g_tau = p.tau;
  w->g_tile = p.split_tile;
  return PROGRESS_OK;
}

int round_up(int64_t n, int m) { return (int)((n + m - 1) / m * m); }

void fill_info(const sp2::State& s, progress_info_t* info) {
  memset(info, 0, sizeof *info);
  info->status = s.status;
  info->iters = s.iter;
  info->converged = s.converged;
  for (int i = 0; i < 3; ++i) info->phase_iters[i] = s.phase_iters[i];
  info->emin = s.emin;
  info->emax = s.emax;
  info->trace = s.t1;
  info->idempotency = s.idem;
  for (int i = 0; i < 4; ++i) info->bits[i] = s.bits[i];
  info->kblocks = s.kblocks;
}

progress_status_t query(Workspace* w, progress_info_t* info) {
  CK(cudaMemcpyAsync(w->h_state, w->buf.st, sizeof(sp2::State), cudaMemcpyDeviceToHost,
                     w->stream),
     "state readback");
  CK(cudaStreamSynchronize(w->stream), "cudaStreamSynchronize");
  fill_info(*w->h_state, info);
  if (w->h_state->status != PROGRESS_OK) {
    const int s = w->h_state->status;
    g_err = s == PROGRESS_ENOCONV   ? "SP2 did not converge within maxiter"
            : s == PROGRESS_ETIMEOUT ? "a bounded device-side wait gave up (D is not valid)"
                                     : "SP2 iterate left [0,1] (bad bounds or input)";
    return (progress_status_t)w->h_state->status;
  }
  return PROGRESS_OK;
}

}  // namespace

namespace sp2 {
void set_last_error(const char* what) { g_err = what; }
}  // namespace sp2

extern "C" {

void progress_opts_default(progress_opts_t* o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->prec = PROGRESS_FP64;
  o->rule = PROGRESS_RULE_NEARER;
  o->fp64_prefix = 12;
  o->maxiter = 100;
  o->emin = NAN;
  o->emax = NAN;
  o->loop_mode = 0;
}

const char* progress_last_error(void) { return g_err.c_str(); }

const char* progress_version(void) { return "0.1.0"; }

progress_status_t progress_gershgorin_bounds(const double* dH, int64_t n, double* d_emin,
                                             double* d_emax, void* stream) {
  if (n < 1 || !dH || !d_emin || !d_emax)
    return fail(PROGRESS_EINVAL, "gershgorin: n < 1 or NULL pointer");
  cudaStream_t s = (cudaStream_t)stream;
  Workspace* w = nullptr;
  progress_status_t st = get_workspace(s, &w);
  if (st != PROGRESS_OK) return st;
  if (!w->buf.partials) {
    st = ensure_buffers(w, 128, false, 0);
    if (st != PROGRESS_OK) return st;
  }
  sp2::SolveParams p;
  memset(&p, 0, sizeof p);
  p.n = n;
  p.ld = 0;
  p.emin_override = NAN;
  p.emax_override = NAN;
  CK(sp2::launch_init(w->buf, p, s), "init launch");
  CK(sp2::launch_gershgorin(dH, n, w->buf, d_emin, d_emax, s), "gershgorin launch");
  return PROGRESS_OK;
}

progress_status_t progress_sp2_dense_ex(const double* dH, int64_t n, int64_t nocc, double tol,
                                        double* dD, const progress_opts_t* opts,
                                        progress_info_t* info, void* stream) {
  progress_opts_t o;
  if (opts) {
    o = *opts;
  } else {
    progress_opts_default(&o);
  }
  if (n < 0 || n > (1 << 16)) return fail(PROGRESS_EINVAL, "n must be in [0, 65536]");
  if (nocc < 0 || nocc > n) return fail(PROGRESS_EINVAL, "nocc must be in [0, n]");
  if (!(tol >= 0.0)) return fail(PROGRESS_EINVAL, "tol must be >= 0");
  if (o.prec < PROGRESS_FP64 || o.prec > PROGRESS_DF64)
    return fail(PROGRESS_EINVAL, "unknown precision mode");
  if (o.fp64_impl < 0 || o.fp64_impl > 3) return fail(PROGRESS_EINVAL, "fp64_impl must be 0..3");
  // FP64-accurate products of the MIXED modes: tensor-core digit products
  // (3; the default up to n = 8192), double-float (2; the default above),
  // native FP64 (1); the DF64 mode is double-float throughout
  const bool mixed = o.prec == PROGRESS_MIXED_FP16 || o.prec == PROGRESS_MIXED_BF16;
  if (mixed && o.fp64_impl == 3 && n > sp2::oz_max_order())
    return fail(PROGRESS_EUNSUPPORTED, "digit products (fp64_impl 3) need n <= 8192");
  const int oz = (mixed && (o.fp64_impl == 3 || (o.fp64_impl == 0 && n <= sp2::oz_max_order())))
                     ? 1 : 0;
  const int df64 = (o.prec == PROGRESS_DF64 || (mixed && o.fp64_impl != 1)) ? 1 : 0;
  if (o.prec == PROGRESS_DF64) o.prec = PROGRESS_FP64;
  // the all-split bf16 mode is the all-split mode with bf16 slices
  const bool split_bf16 = o.prec == PROGRESS_FP32_SPLIT_BF16;
  if (split_bf16) o.prec = PROGRESS_FP32_SPLIT;
  if (o.rule != PROGRESS_RULE_NEARER && o.rule != PROGRESS_RULE_PAPER)
    return fail(PROGRESS_EINVAL, "unknown branch rule");
  if (o.maxiter < 0 || o.maxiter > sp2::kMaxHist - 6)
    return fail(PROGRESS_EINVAL, "maxiter must be in [0, 250]");
  if (o.fp64_prefix < 0) return fail(PROGRESS_EINVAL, "fp64_prefix must be >= 0");
  if (o.loop_mode != 0 && o.loop_mode != 1) return fail(PROGRESS_EINVAL, "loop_mode must be 0 or 1");
  if (o.slice_fixed != 0 && o.slice_fixed != 1) return fail(PROGRESS_EINVAL, "slice_fixed must be 0 or 1");
  if (!(o.tau >= 0.0f) || !isfinite(o.tau)) return fail(PROGRESS_EINVAL, "tau must be finite and >= 0");
  if (o.wait_limit_us < 0) return fail(PROGRESS_EINVAL, "wait_limit_us must be >= 0");
  if (o.stall_test != 0 && o.stall_test != 1) return fail(PROGRESS_EINVAL, "stall_test must be 0 or 1");
  if (o.split_tile < 0 || o.split_tile > 2) return fail(PROGRESS_EINVAL, "split_tile must be 0, 1 or 2");
  if (o.prefix_full != 0 && o.prefix_full != 1) return fail(PROGRESS_EINVAL, "prefix_full must be 0 or 1");
  if (o.stall_test && (o.prec == PROGRESS_FP64 || o.prec == PROGRESS_DF64))
    return fail(PROGRESS_EINVAL, "stall_test needs a mode with tensor-core products");
  if (o.tau > 0.0f && (o.prec != PROGRESS_FP32_SPLIT || o.slice_fixed))
    return fail(PROGRESS_EINVAL,
                "tau > 0 needs prec FP32_SPLIT or FP32_SPLIT_BF16 with floating slices");
  if (!isnan(o.emin) || !isnan(o.emax)) {
    if (isnan(o.emin) || isnan(o.emax) || !(o.emax > o.emin))
      return fail(PROGRESS_EINVAL, "bounds override needs emin < emax (both set)");
  }
  if (n == 0) {
    if (info) memset(info, 0, sizeof *info);
    if (info) info->converged = 1;
    return PROGRESS_OK;
  }
  if (!dH || !dD) return fail(PROGRESS_EINVAL, "NULL matrix pointer");
  cudaStream_t s = (cudaStream_t)stream;
  if (o.prec != PROGRESS_FP64) {
    int dev = 0, major = 0;
    CK(cudaGetDevice(&dev), "cudaGetDevice");
    CK(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev),
       "cudaDeviceGetAttribute");
    if (major != 10) return fail(PROGRESS_EUNSUPPORTED, "split precision needs an sm_10x GPU");
  }
  Workspace* w = nullptr;
  progress_status_t st = get_workspace(s, &w);
  if (st != PROGRESS_OK) return st;
  const int ld = round_up(n, 128);
  const bool need_x64 = o.prec != PROGRESS_FP32_SPLIT;
  int fmt = slice_fmt_of(o.prec, o.slice_fixed);
  if (split_bf16) fmt = o.slice_fixed ? sp2::kBF16x3F : sp2::kBF16x3;
  const int nslices = o.prec == PROGRESS_FP64 ? 0 : sp2::fmt_slices(fmt);
  st = ensure_buffers(w, ld, need_x64, nslices, oz != 0);
  if (st != PROGRESS_OK) return st;
  if (o.tau > 0.0f) {
    st = ensure_flags(w, ld);
    if (st != PROGRESS_OK) return st;
  }

  sp2::SolveParams p;
  memset(&p, 0, sizeof p);
  p.n = n;
  p.ld = ld;
  p.nocc = nocc;
  p.rule = o.rule;
  p.maxiter = o.maxiter;
  p.prec = o.prec;
  p.fp64_prefix = o.fp64_prefix;
  p.slice_fmt = fmt;
  p.df64 = df64;
  p.oz = oz;
  p.tol = tol;
  p.emin_override = o.emin;
  p.emax_override = o.emax;
  p.tau = o.tau;
  p.wait_ns = o.wait_limit_us > 0 ? 1000ull * (unsigned long long)o.wait_limit_us
                                  : 2000000000ull;
  p.stall_test = o.stall_test;
  p.split_tile = o.split_tile;
  p.prefix_full = o.prefix_full;
  // round-off floor of the refinement: 2 n u with u the absolute accuracy of
  // one FP64-accurate product entry (digit products ~2^-40, double-float
  // ~2^-44, native FP64 ~2^-52; entries of X are at most 1)
  p.floor_acc = 2.0 * (double)n * (oz ? 9.094947017729282e-13 : df64 ? 5.684341886080802e-14
                                                                   : 2.220446049250313e-16);

  CK(sp2::launch_init(w->buf, p, s), "init launch");
  CK(sp2::launch_gershgorin(dH, n, w->buf, nullptr, nullptr, s), "gershgorin launch");
  CK(sp2::launch_x0(dH, w->buf, p, s), "x0 launch");
  if (p.tau > 0.0f) CK(sp2::launch_tile_flags(dH, n, ld, w->buf, s), "tile flag launch");
  if (o.loop_events[0]) CK(cudaEventRecord((cudaEvent_t)o.loop_events[0], s), "event record");
  if (o.loop_mode == 0) {
    st = build_graph(w, p);
    if (st != PROGRESS_OK) return st;
    CK(cudaGraphLaunch(w->exec, s), "cudaGraphLaunch");
  } else {
    for (int i = 0; i < o.maxiter + 1; ++i) {
      st = queue_steps(w, p, 0ull, s);
      if (st != PROGRESS_OK) return st;
    }
  }
  if (o.loop_events[1]) CK(cudaEventRecord((cudaEvent_t)o.loop_events[1], s), "event record");
  CK(sp2::launch_finalize(w->buf, dD, n, ld, fmt, s), "finalize launch");
  if (info) return query(w, info);
  return PROGRESS_OK;
}

progress_status_t progress_sp2_dense(const double* dH, int64_t n, int64_t nocc, double tol,
                                     double* dD, void* stream) {
  if (n > 0 && dH == dD) return fail(PROGRESS_EINVAL, "dD must not overlap dH");
  return progress_sp2_dense_ex(dH, n, nocc, tol, dD, nullptr, nullptr, stream);
}

progress_status_t progress_sp2_query(void* stream, progress_info_t* info) {
  if (!info) return fail(PROGRESS_EINVAL, "info is NULL");
  Workspace* w = nullptr;
  progress_status_t st = get_workspace((cudaStream_t)stream, &w);
  if (st != PROGRESS_OK) return st;
  return query(w, info);
}

int32_t progress_sp2_history(void* stream, double* idem, double* margin, int32_t cap) {
  Workspace* w = nullptr;
  if (get_workspace((cudaStream_t)stream, &w) != PROGRESS_OK || cap < 0) return -1;
  if (cudaMemcpyAsync(w->h_state, w->buf.st, sizeof(sp2::State), cudaMemcpyDeviceToHost,
                      w->stream) != cudaSuccess ||
      cudaStreamSynchronize(w->stream) != cudaSuccess) {
    cuda_fail(cudaGetLastError(), "history readback");
    return -1;
  }
  const sp2::State& st = *w->h_state;
  int cnt = st.iter + 1;
  if (cnt > sp2::kMaxHist) cnt = sp2::kMaxHist;
  if (cnt > cap) cnt = cap;
  for (int k = 0; k < cnt; ++k) {
    if (idem) idem[k] = st.idem_hist[k];
    if (margin) margin[k] = k < st.iter ? st.margin_hist[k] : 0.0;
  }
  return cnt;
}

progress_status_t progress_release(void* stream) {
  int dev = 0;
  CK(cudaGetDevice(&dev), "cudaGetDevice");
  CK(cudaStreamSynchronize((cudaStream_t)stream), "cudaStreamSynchronize");
  sp2::batched_release(dev, (cudaStream_t)stream, false);
  sp2::graph_release(dev, (cudaStream_t)stream, false);
  sp2::cheb_release(dev, (cudaStream_t)stream, false);
  Workspace* w = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_ws.find(std::make_pair(dev, (cudaStream_t)stream));
    if (it == g_ws.end()) return PROGRESS_OK;
    w = it->second;
    g_ws.erase(it);
  }
  CK(cudaStreamSynchronize(w->stream), "cudaStreamSynchronize");
  free_workspace(w);
  return PROGRESS_OK;
}

progress_status_t progress_release_all(void) {
  int dev = 0;
  CK(cudaGetDevice(&dev), "cudaGetDevice");
  CK(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
  sp2::batched_release(dev, nullptr, true);
  sp2::graph_release(dev, nullptr, true);
  sp2::cheb_release(dev, nullptr, true);
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto it = g_ws.begin(); it != g_ws.end();) {
    if (it->first.first == dev) {
      free_workspace(it->second);
      it = g_ws.erase(it);
    } else {
      ++it;
    }
  }
  return PROGRESS_OK;
}

}  // extern "C"
