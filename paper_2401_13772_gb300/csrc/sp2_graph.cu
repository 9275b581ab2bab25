// Graph-based divide-and-conquer density matrix (§VIII.B): threshold graph
// of an auxiliary matrix, regular-segment core partition, core-halo parts,
// dense submatrices solved in ONE batched SP2 launch at the system's chemical
// potential, core columns mapped back, symmetrized.
//
//   graph_mark_kernel     one warp per row i of the auxiliary matrix G: the
//                         part k whose core holds i marks i and every j with
//                         |G_ij| >= tau in its membership row flags[k][.]
//   (host)                membership rows -> sorted index lists, sizes and
//                         the packed layout of the parts
//   graph_extract_kernel  h_k = H[ch_k, ch_k] into the packed batch
//   batched SP2           PROGRESS_RULE_MU, one launch for all parts
//   graph_scatter_kernel  P[ch_k, core_k] = D_k[:, core positions]; every
//                         column of P belongs to exactly one core, so no two
//                         parts write the same element
//   graph_symmetrize_kernel  P <- (P + P^T) / 2, 32 x 32 tile pairs through
//                         shared memory
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "progress_sp2.h"
#include "sp2_launch.h"
#include "sp2_tc.cuh"

namespace {

__global__ void graph_mark_kernel(const double* __restrict__ G, int64_t n, double tau,
                                  const int32_t* __restrict__ edges, int32_t nparts,
                                  unsigned char* __restrict__ flags) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n;
       i += warps) {
    // the part whose core [edges[k], edges[k + 1]) holds i
    int lo = 0, hi = nparts - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (edges[mid] <= i) lo = mid; else hi = mid - 1;
    }
    unsigned char* row = flags + (size_t)lo * n;
    const double* g = G + (size_t)i * n;
    if (lane == 0) row[i] = 1;
    for (int64_t j = lane; j < n; j += 32)
      if (j != i && fabs(g[j]) >= tau) row[j] = 1;
  }
}

__global__ void graph_extract_kernel(const double* __restrict__ H, int64_t n,
                                     const int32_t* __restrict__ idx,
                                     const int64_t* __restrict__ idx_off,
                                     const int32_t* __restrict__ sizes,
                                     const int64_t* __restrict__ sub_off,
                                     double* __restrict__ Hsub) {
  const int k = blockIdx.y;
  const int64_t s = sizes[k];
  const int32_t* ix = idx + idx_off[k];
  double* out = Hsub + sub_off[k];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < s * s;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e / s, b = e - a * s;
    out[e] = H[(size_t)ix[a] * n + ix[b]];
  }
}

__global__ void graph_scatter_kernel(int64_t n, const int32_t* __restrict__ idx,
                                     const int64_t* __restrict__ idx_off,
                                     const int32_t* __restrict__ sizes,
                                     const int64_t* __restrict__ sub_off,
                                     const int32_t* __restrict__ edges,
                                     const int32_t* __restrict__ core_pos,
                                     const double* __restrict__ Dsub, double* __restrict__ P) {
  const int k = blockIdx.y;
  const int64_t s = sizes[k];
  const int64_t c0 = edges[k], nc = edges[k + 1] - edges[k];
  const int32_t* ix = idx + idx_off[k];
  const double* d = Dsub + sub_off[k];
  const int64_t p0 = core_pos[k];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < s * nc;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e / nc, cj = e - a * nc;  // row of the part, core column
    P[(size_t)ix[a] * n + (c0 + cj)] = d[a * s + p0 + cj];
  }
}

__global__ void graph_symmetrize_kernel(double* __restrict__ P, int64_t n) {
  __shared__ double a[32][33], b[32][33];
  const int64_t T = (n + 31) / 32;
  // upper-triangle tile pairs (I <= J), one per block in a grid-stride loop
  for (int64_t t = blockIdx.x; t < T * (T + 1) / 2; t += gridDim.x) {
    int I, J;
    sp2::tc::tri_tile((int)t, (int)T, I, J);
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
    for (int yy = ty; yy < 32; yy += 8) {
      const int64_t ri = I * 32 + yy, ci = J * 32 + tx;
      a[yy][tx] = (ri < n && ci < n) ? P[(size_t)ri * n + ci] : 0.0;
      const int64_t rj = J * 32 + yy, cj = I * 32 + tx;
      b[yy][tx] = (rj < n && cj < n) ? P[(size_t)rj * n + cj] : 0.0;
    }
    __syncthreads();
    for (int yy = ty; yy < 32; yy += 8) {
      const int64_t ri = I * 32 + yy, ci = J * 32 + tx;
      const double v = 0.5 * (a[yy][tx] + b[tx][yy]);  // (P + P^T) / 2 at (ri, ci)
      if (ri < n && ci < n) P[(size_t)ri * n + ci] = v;
      const int64_t rj = J * 32 + yy, cj = I * 32 + tx;
      if (I != J && rj < n && cj < n) P[(size_t)rj * n + cj] = 0.5 * (b[yy][tx] + a[tx][yy]);
    }
    __syncthreads();
  }
}

struct GraphWs {
  size_t flags_cap = 0, idx_cap = 0, sub_cap = 0, dsub_cap = 0;
  int parts_cap = 0;
  unsigned char* flags = nullptr;
  int32_t* idx = nullptr;
  int64_t* idx_off = nullptr;
  int32_t* sizes = nullptr;
  int64_t* sub_off = nullptr;
  int32_t* edges = nullptr;
  int32_t* core_pos = nullptr;
  int32_t* iters = nullptr;
  int32_t* status = nullptr;
  double* mu = nullptr;
  double* Hsub = nullptr;
  double* Dsub = nullptr;
};

std::mutex g_gmu;
std::map<std::pair<int, cudaStream_t>, GraphWs*> g_gws;

progress_status_t gfail(progress_status_t s, const char* what) {
  sp2::set_last_error(what);
  return s;
}

progress_status_t gcuda(cudaError_t e, const char* where) {
  sp2::set_last_error(where);
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? PROGRESS_ENOMEM : PROGRESS_ECUDA;
}

template <typename T>
cudaError_t grow(T** p, size_t& cap, size_t need) {
  if (need <= cap && *p) return cudaSuccess;
  if (*p) cudaFree(*p);
  *p = nullptr;
  cap = 0;
  cudaError_t e = cudaMalloc(p, need * sizeof(T));
  if (e == cudaSuccess) cap = need;
  return e;
}

}  // namespace

extern "C" progress_status_t progress_sp2_graph(const double* dH, const double* dG, int64_t n,
                                                double tau, int32_t nparts, double mu,
                                                double tol, double* dD,
                                                const progress_opts_t* opts,
                                                progress_graph_info_t* info, void* stream) {
  if (n < 1 || n > 65536) return gfail(PROGRESS_EINVAL, "n must be in [1, 65536]");
  if (nparts < 1 || nparts > n) return gfail(PROGRESS_EINVAL, "nparts must be in [1, n]");
  if (!dH || !dG || !dD) return gfail(PROGRESS_EINVAL, "NULL matrix pointer");
  if (!(tau >= 0.0) || !(tol >= 0.0) || !isfinite(mu))
    return gfail(PROGRESS_EINVAL, "tau and tol must be >= 0 and mu finite");
  if (dD == dH || dD == dG) return gfail(PROGRESS_EINVAL, "dD must not overlap dH or dG");
  progress_opts_t o;
  if (opts) {
    o = *opts;
  } else {
    progress_opts_default(&o);
    o.prec = PROGRESS_FP32_SPLIT;
  }
  o.rule = PROGRESS_RULE_MU;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return gcuda(e, "cudaGetDevice");
  GraphWs* w = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_gmu);
    auto key = std::make_pair(dev, s);
    auto it = g_gws.find(key);
    if (it == g_gws.end()) {
      w = new GraphWs();
      g_gws[key] = w;
    } else {
      w = it->second;
    }
  }
  // core partition: regular segments of the index list
  std::vector<int32_t> edges(nparts + 1);
  for (int k = 0; k <= nparts; ++k) edges[k] = (int32_t)(((int64_t)k * n) / nparts);
  // membership rows of the core-halo parts
  const size_t fl = (size_t)nparts * (size_t)n;
  size_t ecap = w->parts_cap;
  e = cudaStreamSynchronize(s);  // buffers may still be in use by the previous call
  if (e == cudaSuccess) e = grow(&w->flags, w->flags_cap, fl);
  if (e == cudaSuccess && (size_t)nparts + 1 > ecap) {
    size_t c = 0;
    e = grow(&w->edges, c, (size_t)nparts + 1);
    if (e == cudaSuccess) { c = 0; e = grow(&w->sizes, c, (size_t)nparts); }
    if (e == cudaSuccess) { c = 0; e = grow(&w->idx_off, c, (size_t)nparts); }
    if (e == cudaSuccess) { c = 0; e = grow(&w->sub_off, c, (size_t)nparts); }
    if (e == cudaSuccess) { c = 0; e = grow(&w->core_pos, c, (size_t)nparts); }
    if (e == cudaSuccess) { c = 0; e = grow(&w->mu, c, (size_t)nparts); }
    if (e == cudaSuccess) { c = 0; e = grow(&w->iters, c, (size_t)nparts); }
    if (e == cudaSuccess) { c = 0; e = grow(&w->status, c, (size_t)nparts); }
    if (e == cudaSuccess) w->parts_cap = nparts + 1;
  }
  if (e != cudaSuccess) return gcuda(e, "graph workspace allocation");
  e = cudaMemcpyAsync(w->edges, edges.data(), (nparts + 1) * sizeof(int32_t),
                      cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(w->flags, 0, fl, s);
  if (e != cudaSuccess) return gcuda(e, "graph setup");
  graph_mark_kernel<<<152 * 8, 256, 0, s>>>(dG, n, tau, w->edges, nparts, w->flags);
  e = cudaGetLastError();
  if (e != cudaSuccess) return gcuda(e, "graph_mark launch");
  std::vector<unsigned char> flags(fl);
  e = cudaMemcpyAsync(flags.data(), w->flags, fl, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return gcuda(e, "graph membership readback");
  // index lists (sorted), sizes, packed layout
  std::vector<int32_t> idx, sizes(nparts), core_pos(nparts);
  std::vector<int64_t> idx_off(nparts), sub_off(nparts);
  int64_t total = 0, maxs = 0;
  double sum_s = 0.0;
  for (int k = 0; k < nparts; ++k) {
    idx_off[k] = (int64_t)idx.size();
    const unsigned char* row = flags.data() + (size_t)k * n;
    for (int64_t j = 0; j < n; ++j) {
      if (j == edges[k]) core_pos[k] = (int32_t)(idx.size() - idx_off[k]);
      if (row[j]) idx.push_back((int32_t)j);
    }
    sizes[k] = (int32_t)(idx.size() - idx_off[k]);
    if (sizes[k] > 4096) return gfail(PROGRESS_EUNSUPPORTED, "a core-halo part exceeds 4096 nodes");
    sub_off[k] = total;
    total += (int64_t)sizes[k] * sizes[k];
    maxs = std::max<int64_t>(maxs, sizes[k]);
    sum_s += sizes[k];
  }
  e = grow(&w->idx, w->idx_cap, idx.size());
  if (e == cudaSuccess) e = grow(&w->Hsub, w->sub_cap, (size_t)total);
  if (e == cudaSuccess) e = grow(&w->Dsub, w->dsub_cap, (size_t)total);
  if (e != cudaSuccess) return gcuda(e, "graph part allocation");
  std::vector<double> mus(nparts, mu);
  e = cudaMemcpyAsync(w->idx, idx.data(), idx.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w->sizes, sizes.data(), nparts * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w->idx_off, idx_off.data(), nparts * sizeof(int64_t),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w->sub_off, sub_off.data(), nparts * sizeof(int64_t),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w->core_pos, core_pos.data(), nparts * sizeof(int32_t),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w->mu, mus.data(), nparts * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return gcuda(e, "graph layout upload");
  const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(256, (maxs * maxs + 255) / 256));
  graph_extract_kernel<<<dim3(gx, nparts), 256, 0, s>>>(dH, n, w->idx, w->idx_off, w->sizes,
                                                        w->sub_off, w->Hsub);
  e = cudaGetLastError();
  if (e != cudaSuccess) return gcuda(e, "graph_extract launch");
  // every part in one batched SP2 launch at the chemical potential mu
  std::vector<int32_t> zeros(nparts, 0);
  progress_batch_ex_t ex;
  memset(&ex, 0, sizeof ex);
  ex.d_mu = w->mu;
  progress_status_t st =
      progress_sp2_batched_ex(nparts, sizes.data(), sub_off.data(), zeros.data(), w->Hsub, tol,
                              w->Dsub, w->iters, w->status, &o, &ex, stream);
  if (st != PROGRESS_OK) return st;
  // core columns back into P, then (P + P^T) / 2
  e = cudaMemsetAsync(dD, 0, (size_t)n * n * sizeof(double), s);
  if (e != cudaSuccess) return gcuda(e, "graph output clear");
  int64_t maxc = 0;
  for (int k = 0; k < nparts; ++k) maxc = std::max<int64_t>(maxc, edges[k + 1] - edges[k]);
  const unsigned gs = (unsigned)std::max<int64_t>(1, std::min<int64_t>(256, (maxs * maxc + 255) / 256));
  graph_scatter_kernel<<<dim3(gs, nparts), 256, 0, s>>>(n, w->idx, w->idx_off, w->sizes,
                                                        w->sub_off, w->edges, w->core_pos,
                                                        w->Dsub, dD);
  e = cudaGetLastError();
  if (e != cudaSuccess) return gcuda(e, "graph_scatter launch");
  graph_symmetrize_kernel<<<152 * 8, 256, 0, s>>>(dD, n);
  e = cudaGetLastError();
  if (e != cudaSuccess) return gcuda(e, "graph_symmetrize launch");
  if (info) {
    std::vector<int32_t> it(nparts), stt(nparts);
    e = cudaMemcpyAsync(it.data(), w->iters, nparts * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(stt.data(), w->status, nparts * sizeof(int32_t), cudaMemcpyDeviceToHost,
                          s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return gcuda(e, "graph info readback");
    memset(info, 0, sizeof *info);
    info->nparts = nparts;
    info->max_part = (int32_t)maxs;
    info->mean_part = sum_s / nparts;
    info->max_iters = *std::max_element(it.begin(), it.end());
    info->sub_elements = total;
    for (int k = 0; k < nparts; ++k) info->failed_parts += stt[k] != PROGRESS_OK ? 1 : 0;
  }
  return PROGRESS_OK;
}

namespace sp2 {
void graph_release(int dev, cudaStream_t s, bool all_streams) {
  std::lock_guard<std::mutex> lk(g_gmu);
  for (auto it = g_gws.begin(); it != g_gws.end();) {
    if (it->first.first == dev && (all_streams || it->first.second == s)) {
      GraphWs* w = it->second;
      void* ptrs[] = {w->flags, w->idx, w->idx_off, w->sizes, w->sub_off, w->edges,
                      w->core_pos, w->iters, w->status, w->mu, w->Hsub, w->Dsub};
      for (void* p : ptrs)
        if (p) cudaFree(p);
      delete w;
      it = g_gws.erase(it);
    } else {
      ++it;
    }
  }
}
}  // namespace sp2
