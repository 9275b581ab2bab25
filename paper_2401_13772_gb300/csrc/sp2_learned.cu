// Learned-sequence part: input features of H, the perceptron that predicts
// tighter spectral bounds (the eps_1, eps_N of the X0 map, §IV.A) and the SP2
// branch sequence, and its training step -- forward, loss, backward and Adam,
// all in these kernels. Also the energy-like trace Tr(H D) used to turn an
// SP2 projector onto one state into that state's eigenvalue.
//
// The perceptron is tiny (37 -> 128 -> 128 -> 2 + K); its matrix products are
// a few thousand multiply-adds per sample, so plain FP32 SIMT kernels with one
// thread per output element are the right tool; inference reads FP16 weights.
#include <cuda_fp16.h>
#include <math.h>

#include "progress_sp2.h"
#include "sp2_common.cuh"
#include "sp2_learned.h"

namespace sp2 {
namespace learned {

namespace {

constexpr int kThreads = 256;
constexpr float kCOver = 10.0f;  // weight of an over-estimated bound fraction
constexpr int kBounds = 2;

// ---------------------------------------------------------------------------
// features: one CTA per instance

__global__ void __launch_bounds__(kThreads) features_kernel(const int32_t* __restrict__ nn,
                                                            const int64_t* __restrict__ off,
                                                            const double* __restrict__ Hp,
                                                            float* __restrict__ feat) {
  __shared__ double s_lo[kThreads / 32], s_hi[kThreads / 32], s_red[2 * kThreads / 32];
  __shared__ float s_hist[kHistBins];
  __shared__ double s_emin, s_w;
  const int i = blockIdx.x;
  const int n = nn[i];
  const double* H = Hp + off[i];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x < kHistBins) s_hist[threadIdx.x] = 0.0f;
  double lo = INFINITY, hi = -INFINITY, tr = 0.0, fro = 0.0;
  for (int r = warp; r < n; r += kThreads / 32) {
    const double* row = H + (size_t)r * n;
    float sa = 0.0f, sq = 0.0f;  // per-lane partials over <= n/32 entries
    for (int j = lane; j < n; j += 32) {
      const float h = (float)row[j];
      if (j != r) sa += fabsf(h);
      sq += h * h;
    }
    const double rs = warp_sum((double)sa);
    const double q = warp_sum((double)sq);
    const double d = row[r];
    lo = fmin(lo, d - rs);
    hi = fmax(hi, d + rs);
    if (lane == 0) {
      tr += d;
      fro += q;
    }
  }
  lo = warp_min(lo);
  hi = warp_max(hi);
  if (lane == 0) {
    s_lo[warp] = lo;
    s_hi[warp] = hi;
  }
  block_sum2(tr, fro, s_red);
  if (threadIdx.x == 0) {
    for (int w = 1; w < kThreads / 32; ++w) {
      lo = fmin(lo, s_lo[w]);
      hi = fmax(hi, s_hi[w]);
    }
    double w = hi - lo;
    if (!(w > 0.0)) {
      lo -= 1.0;
      hi += 1.0;
      w = 2.0;
    }
    s_emin = lo;
    s_w = w;
    float* f = feat + (size_t)i * kFeatures;
    f[0] = (float)(lo / w);
    f[1] = (float)(hi / w);
    f[2] = (float)(tr / ((double)n * w));
    f[3] = (float)(sqrt(fro) / (sqrt((double)n) * w));
    f[36] = (float)n / 2048.0f;
  }
  __syncthreads();
  const double emin = s_emin, w = s_w;
  for (int r = threadIdx.x; r < n; r += kThreads) {
    int b = (int)floor((H[(size_t)r * n + r] - emin) / w * kHistBins);
    b = b < 0 ? 0 : (b >= kHistBins ? kHistBins - 1 : b);
    atomicAdd(&s_hist[b], 1.0f);  // integer counts: exact in any order
  }
  __syncthreads();
  if (threadIdx.x < kHistBins)
    feat[(size_t)i * kFeatures + 4 + threadIdx.x] = s_hist[threadIdx.x] / (float)n;
}

// Tr(H D) = sum_ij H_ij D_ji = sum_ij H_ij D_ij for symmetric D; one CTA per instance.
__global__ void __launch_bounds__(kThreads) trace_hd_kernel(const int32_t* __restrict__ nn,
                                                            const int64_t* __restrict__ off,
                                                            const double* __restrict__ Hp,
                                                            const double* __restrict__ Dp,
                                                            double* __restrict__ out) {
  __shared__ double s_red[2 * kThreads / 32];
  const int i = blockIdx.x;
  const int64_t nsq = (int64_t)nn[i] * nn[i];
  const double* H = Hp + off[i];
  const double* D = Dp + off[i];
  double acc = 0.0, dummy = 0.0;
  for (int64_t k0 = (int64_t)threadIdx.x * 32; k0 < nsq; k0 += (int64_t)kThreads * 32) {
    float part = 0.0f;  // FP32 over 32 entries, folded into FP64
    const int64_t k1 = k0 + 32 < nsq ? k0 + 32 : nsq;
    for (int64_t k = k0; k < k1; ++k) part += (float)H[k] * (float)D[k];
    acc += (double)part;
  }
  block_sum2(acc, dummy, s_red);
  if (threadIdx.x == 0) out[i] = acc;
}

// ---------------------------------------------------------------------------
// perceptron

struct Layout {
  int in, hid, out;
  __host__ __device__ int w1() const { return 0; }
  __host__ __device__ int b1() const { return hid * in; }
  __host__ __device__ int w2() const { return b1() + hid; }
  __host__ __device__ int b2() const { return w2() + hid * hid; }
  __host__ __device__ int w3() const { return b2() + hid; }
  __host__ __device__ int b3() const { return w3() + out * hid; }
  __host__ __device__ int count() const { return b3() + out; }
};

template <typename WT>
__device__ __forceinline__ float wval(const WT* w, int i) {
  return (float)w[i];
}
template <>
__device__ __forceinline__ float wval<__half>(const __half* w, int i) {
  return __half2float(w[i]);
}

// Z = X W^T + b (W rows = outputs); A = relu(Z) if relu; one thread per (b, j).
template <typename WT>
__global__ void linear_kernel(const float* __restrict__ X, int B, int K, const WT* __restrict__ W,
                              const WT* __restrict__ bias, int J, float* __restrict__ Z,
                              float* __restrict__ A) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= B * J) return;
  const int b = idx / J, j = idx - b * J;
  const float* x = X + (size_t)b * K;
  float s = wval(bias, j);
  for (int k = 0; k < K; ++k) s = fmaf(x[k], wval(W, j * K + k), s);
  Z[idx] = s;
  if (A) A[idx] = s > 0.0f ? s : 0.0f;
}

// Loss and dL/dY (the definition is in the header comment of the API).
__global__ void loss_kernel(const float* __restrict__ Y, const float* __restrict__ T,
                            const float* __restrict__ M, int B, int J, float* __restrict__ G,
                            float* __restrict__ per_sample) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float* y = Y + (size_t)b * J;
  const float* t = T + (size_t)b * J;
  const float* m = M + (size_t)b * J;
  float* g = G + (size_t)b * J;
  float loss = 0.0f, cnt = 0.0f;
  for (int j = kBounds; j < J; ++j) cnt += m[j];
  cnt = cnt > 1.0f ? cnt : 1.0f;
  for (int j = 0; j < kBounds; ++j) {
    const float e = y[j] - t[j];
    const float c = e > 0.0f ? kCOver : 1.0f;
    loss += c * e * e;
    g[j] = 2.0f * c * e / (float)B;
  }
  for (int j = kBounds; j < J; ++j) {
    const float z = y[j];
    const float bce = fmaxf(z, 0.0f) - z * t[j] + log1pf(expf(-fabsf(z)));
    loss += m[j] * bce / cnt;
    const float sig = 1.0f / (1.0f + expf(-z));
    g[j] = m[j] * (sig - t[j]) / cnt / (float)B;
  }
  per_sample[b] = loss / (float)B;
}

// dW[j][k] = sum_b dZ[b][j] A[b][k], db[j] = sum_b dZ[b][j]; one thread per (j, k|bias).
__global__ void grad_w_kernel(const float* __restrict__ dZ, const float* __restrict__ A, int B,
                              int J, int K, float* __restrict__ dW, float* __restrict__ db) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= J * (K + 1)) return;
  const int j = idx / (K + 1), k = idx - j * (K + 1);
  float s = 0.0f;
  if (k < K) {
    for (int b = 0; b < B; ++b) s = fmaf(dZ[(size_t)b * J + j], A[(size_t)b * K + k], s);
    dW[j * K + k] = s;
  } else {
    for (int b = 0; b < B; ++b) s += dZ[(size_t)b * J + j];
    db[j] = s;
  }
}

// dZprev[b][k] = (sum_j dZ[b][j] W[j][k]) * (Zprev[b][k] > 0); one thread per (b, k).
__global__ void grad_x_kernel(const float* __restrict__ dZ, const float* __restrict__ W, int B,
                              int J, int K, const float* __restrict__ Zprev,
                              float* __restrict__ dZprev) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= B * K) return;
  const int b = idx / K, k = idx - b * K;
  float s = 0.0f;
  for (int j = 0; j < J; ++j) s = fmaf(dZ[(size_t)b * J + j], W[j * K + k], s);
  dZprev[idx] = Zprev[idx] > 0.0f ? s : 0.0f;
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, int count, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void to_half_kernel(const float* __restrict__ p, __half* __restrict__ h, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) h[i] = __float2half_rn(p[i]);
}

__global__ void sum_kernel(const float* __restrict__ x, int count, float* __restrict__ out) {
  __shared__ double s_red[2 * kThreads / 32];
  double acc = 0.0, dummy = 0.0;
  for (int i = threadIdx.x; i < count; i += kThreads) acc += (double)x[i];
  block_sum2(acc, dummy, s_red);
  if (threadIdx.x == 0) *out = (float)acc;
}

// ---------------------------------------------------------------------------
// Solve inputs from the predictor's outputs, one thread per instance:
//   bounds: u_min, u_max (outputs 0, 1; fractions of the Gershgorin width w)
//           widened by `margin`, emin' = emin + w max(u_min - margin, 0),
//           emax' = emax - w max(u_max - margin, 0); an empty interval falls
//           back to the Gershgorin enclosure, so the result never leaves it;
//   bits:   branch k is 1 (2X - X^2) iff logit k > 0;
//   len:    the number of leading logits with |logit| >= tau (only that
//           prefix of the sequence is predicted; later branches are left to
//           the trace rule).
// The products and sums are rounded one operation at a time (no FMA), as in a
// plain FP64 evaluation of the formulas.
__global__ void predict_inputs_kernel(int batch, int nout, const float* __restrict__ Y,
                                      const double* __restrict__ gersh, double margin, float tau,
                                      int kmax, double* __restrict__ bounds,
                                      unsigned long long* __restrict__ bits,
                                      int32_t* __restrict__ len) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= batch) return;
  const float* y = Y + (size_t)i * nout;
  const double emin = gersh[2 * i], emax = gersh[2 * i + 1];
  const double w = __dsub_rn(emax, emin);
  const double u0 = fmax(__dsub_rn((double)y[0], margin), 0.0);
  const double u1 = fmax(__dsub_rn((double)y[1], margin), 0.0);
  double lo = __dadd_rn(emin, __dmul_rn(w, u0));
  double hi = __dsub_rn(emax, __dmul_rn(w, u1));
  if (!(hi > lo)) {
    lo = emin;
    hi = emax;
  }
  bounds[2 * i] = lo;
  bounds[2 * i + 1] = hi;
  if (bits) {
    unsigned long long wd[4] = {0ull, 0ull, 0ull, 0ull};
    for (int k = 0; k < kmax; ++k)
      if (y[kBounds + k] > 0.0f) wd[k >> 6] |= 1ull << (k & 63);
    for (int q = 0; q < 4; ++q) bits[4 * i + q] = wd[q];
  }
  if (len) {
    int L = 0;
    while (L < kmax && fabsf(y[kBounds + L]) >= tau) ++L;
    len[i] = L;
  }
}

// Training targets and masks, one thread per instance: the two bound targets
// (ub[i * ld_ub + 0..1]), then the branch bits of a labelled SP2 run, masked
// beyond its product count and for runs that fell back (reject[i] != 0).
__global__ void targets_kernel(int batch, int kmax, const float* __restrict__ ub, int ld_ub,
                               const unsigned long long* __restrict__ bits,
                               const int32_t* __restrict__ iters,
                               const int32_t* __restrict__ reject, float* __restrict__ T,
                               float* __restrict__ M) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= batch) return;
  const int nout = kBounds + kmax;
  float* t = T + (size_t)i * nout;
  float* m = M + (size_t)i * nout;
  t[0] = ub[(size_t)i * ld_ub];
  t[1] = ub[(size_t)i * ld_ub + 1];
  m[0] = 1.0f;
  m[1] = 1.0f;
  const int it = iters ? iters[i] : 0;
  const bool ok = !(reject && reject[i]);
  for (int k = 0; k < kmax; ++k) {
    t[kBounds + k] = bits ? (float)((bits[4 * i + (k >> 6)] >> (k & 63)) & 1ull) : 0.0f;
    m[kBounds + k] = (ok && k < it) ? 1.0f : 0.0f;
  }
}

// Bound targets from the extremal eigenvalues: u_min = max((eps_1 - emin)/w, 0),
// u_max = max((emax - eps_N)/w, 0), w = emax - emin (the Gershgorin enclosure).
__global__ void bound_fractions_kernel(int batch, const double* __restrict__ eps1,
                                       const double* __restrict__ epsN,
                                       const double* __restrict__ gersh,
                                       float* __restrict__ u) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= batch) return;
  const double emin = gersh[2 * i], emax = gersh[2 * i + 1];
  const double w = emax - emin;
  u[2 * i] = (float)fmax((eps1[i] - emin) / w, 0.0);
  u[2 * i + 1] = (float)fmax((emax - epsN[i]) / w, 0.0);
}

// y = -x over `count` doubles (the operator -H whose lowest state is H's highest).
__global__ void negate_kernel(const double* __restrict__ x, int64_t count, double* __restrict__ y) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count;
       q += (int64_t)gridDim.x * blockDim.x)
    y[q] = -x[q];
}

inline int blocks(int64_t work) { return (int)((work + kThreads - 1) / kThreads); }

}  // namespace

cudaError_t predict_inputs(int batch, int nout, const float* d_y, const double* d_gersh,
                           double margin, float tau, double* d_bounds, uint64_t* d_bits,
                           int32_t* d_len, cudaStream_t s) {
  predict_inputs_kernel<<<blocks(batch), kThreads, 0, s>>>(
      batch, nout, d_y, d_gersh, margin, tau, nout - kBounds, d_bounds,
      reinterpret_cast<unsigned long long*>(d_bits), d_len);
  return cudaGetLastError();
}

cudaError_t targets(int batch, int kmax, const float* d_ub, int ld_ub, const uint64_t* d_bits,
                    const int32_t* d_iters, const int32_t* d_reject, float* d_t, float* d_m,
                    cudaStream_t s) {
  targets_kernel<<<blocks(batch), kThreads, 0, s>>>(
      batch, kmax, d_ub, ld_ub, reinterpret_cast<const unsigned long long*>(d_bits), d_iters,
      d_reject, d_t, d_m);
  return cudaGetLastError();
}

cudaError_t bound_fractions(int batch, const double* d_eps1, const double* d_epsN,
                            const double* d_gersh, float* d_u, cudaStream_t s) {
  bound_fractions_kernel<<<blocks(batch), kThreads, 0, s>>>(batch, d_eps1, d_epsN, d_gersh, d_u);
  return cudaGetLastError();
}

cudaError_t negate(const double* d_x, int64_t count, double* d_y, cudaStream_t s) {
  int64_t b = (count + kThreads - 1) / kThreads;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  negate_kernel<<<(int)b, kThreads, 0, s>>>(d_x, count, d_y);
  return cudaGetLastError();
}

int param_count(int in, int hid, int out) { return Layout{in, hid, out}.count(); }

int64_t train_scratch_floats(int in, int hid, int out, int batch) {
  // Z1, A1, Z2, A2, Y, G, dZ2, dZ1, per-sample loss
  return (int64_t)batch * (4 * hid + 2 * out + 2 * hid + 1);
}

cudaError_t features(int batch, const int32_t* d_n, const int64_t* d_off, const double* dH,
                     float* d_feat, cudaStream_t s) {
  features_kernel<<<batch, kThreads, 0, s>>>(d_n, d_off, dH, d_feat);
  return cudaGetLastError();
}

cudaError_t trace_hd(int batch, const int32_t* d_n, const int64_t* d_off, const double* dH,
                     const double* dD, double* d_out, cudaStream_t s) {
  trace_hd_kernel<<<batch, kThreads, 0, s>>>(d_n, d_off, dH, dD, d_out);
  return cudaGetLastError();
}

cudaError_t forward_fp16(int in, int hid, int out, const uint16_t* d_params_h, int batch,
                         const float* d_x, float* d_y, float* d_scratch, cudaStream_t s) {
  const Layout L{in, hid, out};
  const __half* P = reinterpret_cast<const __half*>(d_params_h);
  float* Z1 = d_scratch;
  float* A1 = Z1 + (size_t)batch * hid;
  float* Z2 = A1 + (size_t)batch * hid;
  float* A2 = Z2 + (size_t)batch * hid;
  linear_kernel<__half><<<blocks((int64_t)batch * hid), kThreads, 0, s>>>(
      d_x, batch, in, P + L.w1(), P + L.b1(), hid, Z1, A1);
  linear_kernel<__half><<<blocks((int64_t)batch * hid), kThreads, 0, s>>>(
      A1, batch, hid, P + L.w2(), P + L.b2(), hid, Z2, A2);
  linear_kernel<__half><<<blocks((int64_t)batch * out), kThreads, 0, s>>>(
      A2, batch, hid, P + L.w3(), P + L.b3(), out, d_y, nullptr);
  return cudaGetLastError();
}

cudaError_t train_step(int in, int hid, int out, float* d_params, float* d_grad, float* d_m,
                       float* d_v, int step, float lr, int batch, const float* d_x,
                       const float* d_t, const float* d_mask, float* d_scratch, float* d_loss,
                       cudaStream_t s) {
  const Layout L{in, hid, out};
  float* Z1 = d_scratch;
  float* A1 = Z1 + (size_t)batch * hid;
  float* Z2 = A1 + (size_t)batch * hid;
  float* A2 = Z2 + (size_t)batch * hid;
  float* Y = A2 + (size_t)batch * hid;
  float* G = Y + (size_t)batch * out;
  float* dZ2 = G + (size_t)batch * out;
  float* dZ1 = dZ2 + (size_t)batch * hid;
  float* per = dZ1 + (size_t)batch * hid;
  const float* P = d_params;
  linear_kernel<float><<<blocks((int64_t)batch * hid), kThreads, 0, s>>>(
      d_x, batch, in, P + L.w1(), P + L.b1(), hid, Z1, A1);
  linear_kernel<float><<<blocks((int64_t)batch * hid), kThreads, 0, s>>>(
      A1, batch, hid, P + L.w2(), P + L.b2(), hid, Z2, A2);
  linear_kernel<float><<<blocks((int64_t)batch * out), kThreads, 0, s>>>(
      A2, batch, hid, P + L.w3(), P + L.b3(), out, Y, nullptr);
  loss_kernel<<<blocks(batch), kThreads, 0, s>>>(Y, d_t, d_mask, batch, out, G, per);
  if (d_loss) sum_kernel<<<1, kThreads, 0, s>>>(per, batch, d_loss);
  // layer 3
  grad_w_kernel<<<blocks((int64_t)out * (hid + 1)), kThreads, 0, s>>>(
      G, A2, batch, out, hid, d_grad + L.w3(), d_grad + L.b3());
  grad_x_kernel<<<blocks((int64_t)batch * hid), kThreads, 0, s>>>(G, P + L.w3(), batch, out,
                                                                   hid, Z2, dZ2);
  // layer 2
  grad_w_kernel<<<blocks((int64_t)hid * (hid + 1)), kThreads, 0, s>>>(
      dZ2, A1, batch, hid, hid, d_grad + L.w2(), d_grad + L.b2());
  grad_x_kernel<<<blocks((int64_t)batch * hid), kThreads, 0, s>>>(dZ2, P + L.w2(), batch, hid,
                                                                   hid, Z1, dZ1);
  // layer 1
  grad_w_kernel<<<blocks((int64_t)hid * (in + 1)), kThreads, 0, s>>>(
      dZ1, d_x, batch, hid, in, d_grad + L.w1(), d_grad + L.b1());
  if (lr != 0.0f && d_m && d_v) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    adam_kernel<<<blocks(L.count()), kThreads, 0, s>>>(d_params, d_grad, d_m, d_v, L.count(),
                                                       lr, b1, b2, 1e-8f, c1, c2);
  }
  return cudaGetLastError();
}

cudaError_t to_half(const float* d_params, int count, uint16_t* d_params_h, cudaStream_t s) {
  to_half_kernel<<<blocks(count), kThreads, 0, s>>>(d_params, reinterpret_cast<__half*>(d_params_h),
                                                    count);
  return cudaGetLastError();
}

}  // namespace learned
}  // namespace sp2
