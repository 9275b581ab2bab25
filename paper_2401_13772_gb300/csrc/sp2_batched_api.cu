// C ABI of the batched solver: layout planning on the host (padded orders,
// tall-matrix rows, largest-first order), a cached per-stream workspace and a
// cached CUDA graph holding the queue reset and the one persistent launch.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <numeric>
#include <utility>
#include <vector>

#include "progress_sp2.h"
#include "sp2_batched.h"
#include "sp2_launch.h"
#include "sp2_slices.cuh"

namespace {

using sp2::batched::Config;
using sp2::batched::Instance;
using sp2::batched::InstanceInfo;
using sp2::batched::Params;

// Launch configuration used when neither the caller nor the autotuner chose
// one: for parts of up to 768 orbitals 128 x 64 tiles, clusters of two CTAs
// sharing parts of >= 2 row blocks (among the fastest candidates on 4000
// parts of 64..768); for larger parts 128 x 128 tiles, clusters of two
// sharing from 3 row blocks (1000 parts of 2048: 290 vs 207 solves/s).
constexpr Config kDefaultSmall = {64, 2, 2, 0};
constexpr Config kDefaultLarge = {128, 2, 3, 0};

// Autotuned configurations by batch signature (device, slice format, pitch,
// floor(log2(batch))).
struct TuneKey {
  int dev, fmt, pitch, lgb;
  bool operator<(const TuneKey& o) const {
    if (dev != o.dev) return dev < o.dev;
    if (fmt != o.fmt) return fmt < o.fmt;
    if (pitch != o.pitch) return pitch < o.pitch;
    return lgb < o.lgb;
  }
};
std::mutex g_tmu;
std::map<TuneKey, Config> g_tuned;

int floor_log2(int v) {
  int l = 0;
  while (v > 1) {
    v >>= 1;
    ++l;
  }
  return l;
}

struct BatchWs {
  cudaStream_t cap = nullptr;
  // device buffers
  uint16_t* sl[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
  int nslices = 0;
  size_t slice_elems = 0;
  Instance* inst = nullptr;
  int32_t* order = nullptr;
  int32_t* queue = nullptr;
  InstanceInfo* info = nullptr;
  int cap_batch = 0;
  // cached graph of the last launch
  cudaGraphExec_t exec = nullptr;
  std::vector<Instance> last_inst;
  Params last_prm{};
  Config last_cfg{};
  int last_grid = 0;
  bool have_last = false;
};

std::mutex g_bmu;
std::map<std::pair<int, cudaStream_t>, BatchWs*> g_bws;

progress_status_t bfail(progress_status_t s, const char* what) {
  sp2::set_last_error(what);
  return s;
}

progress_status_t bcuda(cudaError_t e, const char* where) {
  sp2::set_last_error(where);
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? PROGRESS_ENOMEM : PROGRESS_ECUDA;
}

void free_bufs(BatchWs* w) {
  for (int k = 0; k < 2; ++k)
    for (int j = 0; j < 3; ++j) {
      if (w->sl[k][j]) cudaFree(w->sl[k][j]);
      w->sl[k][j] = nullptr;
    }
  w->slice_elems = 0;
  w->nslices = 0;
}

void free_meta(BatchWs* w) {
  if (w->inst) cudaFree(w->inst);
  if (w->order) cudaFree(w->order);
  if (w->queue) cudaFree(w->queue);
  if (w->info) cudaFree(w->info);
  w->inst = nullptr;
  w->order = nullptr;
  w->queue = nullptr;
  w->info = nullptr;
  w->cap_batch = 0;
}

void drop_graph(BatchWs* w) {
  if (w->exec) cudaGraphExecDestroy(w->exec);
  w->exec = nullptr;
  w->have_last = false;
}

bool same_params(const Params& a, const Params& b) { return memcmp(&a, &b, sizeof a) == 0; }
bool same_config(const Config& a, const Config& b) {
  return a.tile_n == b.tile_n && a.cluster == b.cluster && a.share == b.share;
}

progress_status_t batched_impl(int32_t batch, const int32_t* h_n, const int64_t* h_offset,
                               const int32_t* h_nocc, const double* dH, double tol, double* dD,
                               int32_t* d_iters, int32_t* d_status, const progress_opts_t* opts,
                               const progress_batch_ex_t* ex, const Config* force, void* stream);

}  // namespace

extern "C" progress_status_t progress_sp2_batched(int32_t batch, const int32_t* h_n,
                                                  const int64_t* h_offset, const int32_t* h_nocc,
                                                  const double* dH, double tol, double* dD,
                                                  int32_t* d_iters, int32_t* d_status,
                                                  const progress_opts_t* opts, void* stream) {
  return batched_impl(batch, h_n, h_offset, h_nocc, dH, tol, dD, d_iters, d_status, opts, nullptr,
                      nullptr, stream);
}

extern "C" progress_status_t progress_sp2_batched_ex(int32_t batch, const int32_t* h_n,
                                                     const int64_t* h_offset,
                                                     const int32_t* h_nocc, const double* dH,
                                                     double tol, double* dD, int32_t* d_iters,
                                                     int32_t* d_status,
                                                     const progress_opts_t* opts,
                                                     const progress_batch_ex_t* ex, void* stream) {
  return batched_impl(batch, h_n, h_offset, h_nocc, dH, tol, dD, d_iters, d_status, opts, ex,
                      nullptr, stream);
}

namespace {

progress_status_t batched_impl(int32_t batch, const int32_t* h_n, const int64_t* h_offset,
                               const int32_t* h_nocc, const double* dH, double tol, double* dD,
                               int32_t* d_iters, int32_t* d_status, const progress_opts_t* opts,
                               const progress_batch_ex_t* ex, const Config* force, void* stream) {
  progress_opts_t o;
  if (opts) {
    o = *opts;
  } else {
    progress_opts_default(&o);
    o.prec = PROGRESS_FP32_SPLIT;
  }
  if (batch < 0) return bfail(PROGRESS_EINVAL, "batch must be >= 0");
  if (batch == 0) return PROGRESS_OK;
  if (!h_n || !h_offset || !h_nocc || !dH || !dD)
    return bfail(PROGRESS_EINVAL, "NULL pointer argument");
  if (!(tol >= 0.0)) return bfail(PROGRESS_EINVAL, "tol must be >= 0");
  if (o.prec != PROGRESS_FP32_SPLIT && o.prec != PROGRESS_FP32_SPLIT_BF16)
    return bfail(PROGRESS_EUNSUPPORTED,
                 "the batched solver runs PROGRESS_FP32_SPLIT or PROGRESS_FP32_SPLIT_BF16 only");
  const int fmt = o.prec == PROGRESS_FP32_SPLIT_BF16 ? sp2::kBF16x3 : sp2::kFP16x2;
  const int nsl = sp2::fmt_slices(fmt);
  const bool by_mu = o.rule == PROGRESS_RULE_MU;
  if (o.rule != PROGRESS_RULE_NEARER && o.rule != PROGRESS_RULE_PAPER && !by_mu)
    return bfail(PROGRESS_EINVAL, "unknown branch rule");
  if (by_mu && !(ex && ex->d_mu))
    return bfail(PROGRESS_EINVAL, "PROGRESS_RULE_MU needs progress_batch_ex_t.d_mu");
  if (o.maxiter < 0 || o.maxiter > 250) return bfail(PROGRESS_EINVAL, "maxiter must be in [0, 250]");
  std::vector<Instance> inst(batch);
  int pitch = 0;
  int64_t rows = 0;
  for (int i = 0; i < batch; ++i) {
    const int n = h_n[i];
    if (n < 1 || n > 4096) return bfail(PROGRESS_EINVAL, "every n_i must be in [1, 4096]");
    if (!by_mu && (h_nocc[i] < 0 || h_nocc[i] > n))
      return bfail(PROGRESS_EINVAL, "nocc_i must be in [0, n_i]");
    if (h_offset[i] < 0) return bfail(PROGRESS_EINVAL, "offsets must be >= 0");
    Instance& t = inst[i];
    memset(&t, 0, sizeof t);
    t.n = n;
    t.m = (n + 127) / 128 * 128;
    t.nocc = by_mu ? 0 : h_nocc[i];
    t.row0 = rows;
    t.offset = h_offset[i];
    rows += t.m;
    pitch = std::max(pitch, t.m);
  }
  int dev = 0, major = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  if (e != cudaSuccess) return bcuda(e, "device query");
  if (major != 10) return bfail(PROGRESS_EUNSUPPORTED, "the batched solver needs an sm_10x GPU");
  cudaStream_t s = (cudaStream_t)stream;
  // launch configuration: forced (autotuner), explicit (caller), tuned, default
  Config cfg = pitch >= 1024 ? kDefaultLarge : kDefaultSmall;
  if (force) {
    cfg = *force;
  } else if (ex && (ex->tile_n || ex->cluster || ex->share)) {
    cfg.tile_n = ex->tile_n;
    cfg.cluster = ex->cluster;
    cfg.share = ex->share;
  } else {
    std::lock_guard<std::mutex> lk(g_tmu);
    auto it = g_tuned.find(TuneKey{dev, fmt, pitch, floor_log2(batch)});
    if (it != g_tuned.end()) cfg = it->second;
  }
  if (!sp2::batched::config_ok(cfg))
    return bfail(PROGRESS_EINVAL, "batch configuration: tile_n 64 or 128, cluster 1, 2, 4 or 8, share >= 1");
  const int grid = sp2::batched::grid_size(cfg, fmt, batch);
  if (grid < 1) return bcuda(cudaErrorInvalidConfiguration, "batched launch configuration");

  BatchWs* w = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_bmu);
    auto key = std::make_pair(dev, s);
    auto it = g_bws.find(key);
    if (it == g_bws.end()) {
      w = new BatchWs();
      if (cudaStreamCreateWithFlags(&w->cap, cudaStreamNonBlocking) != cudaSuccess) {
        delete w;
        return bcuda(cudaErrorUnknown, "capture stream");
      }
      g_bws[key] = w;
    } else {
      w = it->second;
    }
  }
  // workspace
  const size_t need = (size_t)rows * pitch;
  if (need > w->slice_elems || nsl > w->nslices || batch > w->cap_batch) {
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bcuda(e, "cudaStreamSynchronize");
    drop_graph(w);
  }
  if (need > w->slice_elems || nsl > w->nslices) {
    const size_t alloc = need > w->slice_elems ? need : w->slice_elems;
    const int ns = nsl > w->nslices ? nsl : w->nslices;
    free_bufs(w);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k)
      for (int j = 0; j < ns && e == cudaSuccess; ++j)
        e = cudaMalloc(&w->sl[k][j], alloc * sizeof(uint16_t));
    if (e != cudaSuccess) {
      free_bufs(w);
      return bcuda(e, "batched slice allocation");
    }
    w->slice_elems = alloc;
    w->nslices = ns;
  }
  if (batch > w->cap_batch) {
    free_meta(w);
    e = cudaMalloc(&w->inst, batch * sizeof(Instance));
    if (e == cudaSuccess) e = cudaMalloc(&w->order, batch * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&w->queue, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&w->info, batch * sizeof(InstanceInfo));
    if (e != cudaSuccess) {
      free_meta(w);
      return bcuda(e, "batched metadata allocation");
    }
    w->cap_batch = batch;
  }
  // largest-first order (cost ~ m^3; ties keep the input order)
  std::vector<int32_t> order(batch);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return inst[a].m > inst[b].m; });

  Params prm;
  memset(&prm, 0, sizeof prm);
  prm.inst = w->inst;
  prm.order = w->order;
  prm.queue = w->queue;
  prm.batch = batch;
  prm.rule = o.rule;
  prm.maxiter = o.maxiter;
  prm.pitch = pitch;
  prm.total_rows = rows;
  prm.tol = tol;
  prm.H = dH;
  prm.D = dD;
  prm.fmt = fmt;
  for (int k = 0; k < 2; ++k)
    for (int j = 0; j < 3; ++j) prm.sl[k][j] = w->sl[k][j];
  prm.iters = d_iters;
  prm.status = d_status;
  prm.info = w->info;
  if (ex) {
    prm.bounds_in = ex->d_bounds;
    prm.pred_bits = reinterpret_cast<const unsigned long long*>(ex->d_pred_bits);
    prm.pred_len = ex->d_pred_len;
    prm.judge_delta = ex->judge_delta;
    prm.bits_out = reinterpret_cast<unsigned long long*>(ex->d_bits_out);
    prm.bounds_out = ex->d_bounds_out;
    prm.fallback = ex->d_fallback;
    prm.products = ex->d_products;
    prm.cycles = reinterpret_cast<long long*>(ex->d_cycles);
    prm.mu_in = ex->d_mu;
  }
  prm.share = cfg.share;

  const bool same_layout = w->have_last && w->last_inst.size() == inst.size() &&
                           memcmp(w->last_inst.data(), inst.data(),
                                  inst.size() * sizeof(Instance)) == 0;
  if (!same_layout) {
    // metadata upload (ordered on the stream before the launch)
    e = cudaMemcpyAsync(w->inst, inst.data(), batch * sizeof(Instance), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(w->order, order.data(), batch * sizeof(int32_t), cudaMemcpyHostToDevice,
                          s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host vectors go out of scope
    if (e != cudaSuccess) return bcuda(e, "batched metadata upload");
  }
  if (!(same_layout && w->exec && same_params(prm, w->last_prm) &&
        same_config(cfg, w->last_cfg) && grid == w->last_grid)) {
    drop_graph(w);
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(w->cap, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      cudaMemsetAsync(w->queue, 0, sizeof(int32_t), w->cap);
      if (d_status) cudaMemsetAsync(d_status, 0xFF, batch * sizeof(int32_t), w->cap);
      const cudaError_t le = sp2::batched::launch(prm, cfg, grid, w->cap);
      e = cudaStreamEndCapture(w->cap, &g);
      if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&w->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      drop_graph(w);
      return bcuda(e, "batched graph capture");
    }
    w->last_inst = inst;
    w->last_prm = prm;
    w->last_cfg = cfg;
    w->last_grid = grid;
    w->have_last = true;
  }
  e = cudaGraphLaunch(w->exec, s);
  if (e != cudaSuccess) return bcuda(e, "batched graph launch");
  return PROGRESS_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Autotuner

extern "C" progress_status_t progress_sp2_batched_tune(
    int32_t batch, const int32_t* h_n, const int64_t* h_offset, const int32_t* h_nocc,
    const double* dH, double tol, double* dD, const progress_opts_t* opts, int32_t sample_stride,
    int32_t reps, progress_batch_tune_t* out, void* stream) {
  if (batch < 1) return bfail(PROGRESS_EINVAL, "batch must be >= 1");
  if (!h_n || !h_offset || !h_nocc || !dH || !dD)
    return bfail(PROGRESS_EINVAL, "NULL pointer argument");
  if (sample_stride < 1) return bfail(PROGRESS_EINVAL, "sample_stride must be >= 1");
  if (reps < 1 || reps > 50) return bfail(PROGRESS_EINVAL, "reps must be in [1, 50]");
  progress_opts_t o;
  if (opts) {
    o = *opts;
  } else {
    progress_opts_default(&o);
    o.prec = PROGRESS_FP32_SPLIT;
  }
  if (o.prec != PROGRESS_FP32_SPLIT && o.prec != PROGRESS_FP32_SPLIT_BF16)
    return bfail(PROGRESS_EUNSUPPORTED,
                 "the batched solver runs PROGRESS_FP32_SPLIT or PROGRESS_FP32_SPLIT_BF16 only");
  const int fmt = o.prec == PROGRESS_FP32_SPLIT_BF16 ? sp2::kBF16x3 : sp2::kFP16x2;
  int pitch = 0;
  for (int i = 0; i < batch; ++i) {
    if (h_n[i] < 1 || h_n[i] > 4096) return bfail(PROGRESS_EINVAL, "every n_i must be in [1, 4096]");
    pitch = std::max(pitch, (h_n[i] + 127) / 128 * 128);
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return bcuda(e, "device query");
  // calibration sample: every sample_stride-th instance in decreasing size
  std::vector<int32_t> idx(batch);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return h_n[a] > h_n[b]; });
  std::vector<int32_t> sn, snocc;
  std::vector<int64_t> soff;
  for (int k = 0; k < batch; k += sample_stride) {
    sn.push_back(h_n[idx[k]]);
    snocc.push_back(h_nocc[idx[k]]);
    soff.push_back(h_offset[idx[k]]);
  }
  const int sb = (int)sn.size();
  static const Config cands[] = {{128, 1, 1, 0}, {64, 1, 1, 0},  {128, 2, 2, 0}, {64, 2, 2, 0},
                                 {128, 4, 3, 0}, {64, 4, 3, 0},  {128, 4, 4, 0}, {64, 4, 4, 0},
                                 {128, 8, 4, 0}, {64, 8, 4, 0},  {128, 8, 5, 0}, {64, 8, 5, 0},
                                 {64, 8, 3, 0}};
  const int nc = (int)(sizeof cands / sizeof cands[0]);
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  e = cudaEventCreate(&ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&ev1);
  if (e != cudaSuccess) {
    if (ev0) cudaEventDestroy(ev0);
    return bcuda(e, "tuner events");
  }
  progress_batch_tune_t res;
  memset(&res, 0, sizeof res);
  int best = -1;
  float best_ms = 0.0f;
  progress_status_t st = PROGRESS_OK;
  for (int c = 0; c < nc && st == PROGRESS_OK; ++c) {
    res.cand[c][0] = cands[c].tile_n;
    res.cand[c][1] = cands[c].cluster;
    res.cand[c][2] = cands[c].share;
    res.ms[c] = -1.0f;
    res.ncand = c + 1;
    if (sp2::batched::grid_size(cands[c], fmt, sb) < 1) continue;  // not launchable here
    st = batched_impl(sb, sn.data(), soff.data(), snocc.data(), dH, tol, dD, nullptr, nullptr, &o,
                      nullptr, &cands[c], stream);
    if (st != PROGRESS_OK) break;
    std::vector<float> t;
    for (int r = 0; r < reps && st == PROGRESS_OK; ++r) {
      e = cudaEventRecord(ev0, s);
      if (e == cudaSuccess) {
        st = batched_impl(sb, sn.data(), soff.data(), snocc.data(), dH, tol, dD, nullptr, nullptr,
                          &o, nullptr, &cands[c], stream);
        if (st != PROGRESS_OK) break;
        e = cudaEventRecord(ev1, s);
      }
      if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
      if (e != cudaSuccess) {
        st = bcuda(e, "tuner timing");
        break;
      }
      t.push_back(ms);
    }
    if (st != PROGRESS_OK) break;
    std::sort(t.begin(), t.end());
    res.ms[c] = t[t.size() / 2];
    if (best < 0 || res.ms[c] < best_ms) {
      best = c;
      best_ms = res.ms[c];
    }
  }
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  if (st != PROGRESS_OK) return st;
  if (best < 0) return bfail(PROGRESS_EUNSUPPORTED, "no batched launch configuration fits this GPU");
  res.tile_n = cands[best].tile_n;
  res.cluster = cands[best].cluster;
  res.share = cands[best].share;
  {
    std::lock_guard<std::mutex> lk(g_tmu);
    g_tuned[TuneKey{dev, fmt, pitch, floor_log2(batch)}] = cands[best];
  }
  if (out) *out = res;
  return PROGRESS_OK;
}

namespace sp2 {
void batched_release(int dev, cudaStream_t s, bool all_streams) {
  std::lock_guard<std::mutex> lk(g_bmu);
  for (auto it = g_bws.begin(); it != g_bws.end();) {
    if (it->first.first == dev && (all_streams || it->first.second == s)) {
      BatchWs* w = it->second;
      drop_graph(w);
      free_bufs(w);
      free_meta(w);
      if (w->cap) cudaStreamDestroy(w->cap);
      delete w;
      it = g_bws.erase(it);
    } else {
      ++it;
    }
  }
}
}  // namespace sp2
