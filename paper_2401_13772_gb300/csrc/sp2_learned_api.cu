// C ABI of the learned-sequence part (features, Tr(HD), perceptron, the
// labels, training targets and solve inputs derived from SP2 runs and from the
// predictor's outputs).
#include <math.h>

#include <algorithm>
#include <vector>

#include "progress_sp2.h"
#include "sp2_launch.h"
#include "sp2_learned.h"

namespace {

progress_status_t lfail(progress_status_t s, const char* what) {
  sp2::set_last_error(what);
  return s;
}

progress_status_t lcuda(cudaError_t e, const char* where) {
  if (e == cudaSuccess) return PROGRESS_OK;
  sp2::set_last_error(where);
  cudaGetLastError();
  return PROGRESS_ECUDA;
}

bool dims_ok(int in, int hid, int out) {
  return in > 0 && hid > 0 && out > 2 && in <= 4096 && hid <= 4096 && out <= 4096;
}

}  // namespace

extern "C" {

progress_status_t progress_features(int32_t batch, const int32_t* d_n, const int64_t* d_offset,
                                    const double* dH, float* d_feat, void* stream) {
  if (batch < 0) return lfail(PROGRESS_EINVAL, "batch must be >= 0");
  if (batch == 0) return PROGRESS_OK;
  if (!d_n || !d_offset || !dH || !d_feat) return lfail(PROGRESS_EINVAL, "NULL pointer argument");
  return lcuda(sp2::learned::features(batch, d_n, d_offset, dH, d_feat, (cudaStream_t)stream),
               "features launch");
}

progress_status_t progress_trace_hd(int32_t batch, const int32_t* d_n, const int64_t* d_offset,
                                    const double* dH, const double* dD, double* d_out,
                                    void* stream) {
  if (batch < 0) return lfail(PROGRESS_EINVAL, "batch must be >= 0");
  if (batch == 0) return PROGRESS_OK;
  if (!d_n || !d_offset || !dH || !dD || !d_out)
    return lfail(PROGRESS_EINVAL, "NULL pointer argument");
  return lcuda(sp2::learned::trace_hd(batch, d_n, d_offset, dH, dD, d_out, (cudaStream_t)stream),
               "trace_hd launch");
}

int32_t progress_mlp_param_count(int32_t in, int32_t hidden, int32_t out) {
  if (!dims_ok(in, hidden, out)) return -1;
  return sp2::learned::param_count(in, hidden, out);
}

int64_t progress_mlp_scratch_floats(int32_t in, int32_t hidden, int32_t out, int32_t batch) {
  if (!dims_ok(in, hidden, out) || batch < 1) return -1;
  return sp2::learned::train_scratch_floats(in, hidden, out, batch);
}

progress_status_t progress_mlp_to_fp16(const float* d_params, int32_t count,
                                       uint16_t* d_params_fp16, void* stream) {
  if (count < 0 || (count > 0 && (!d_params || !d_params_fp16)))
    return lfail(PROGRESS_EINVAL, "bad parameter buffers");
  if (count == 0) return PROGRESS_OK;
  return lcuda(sp2::learned::to_half(d_params, count, d_params_fp16, (cudaStream_t)stream),
               "to_fp16 launch");
}

progress_status_t progress_mlp_forward(int32_t in, int32_t hidden, int32_t out,
                                       const uint16_t* d_params_fp16, int32_t batch,
                                       const float* d_x, float* d_y, float* d_scratch,
                                       void* stream) {
  if (!dims_ok(in, hidden, out)) return lfail(PROGRESS_EINVAL, "bad perceptron dimensions");
  if (batch < 0) return lfail(PROGRESS_EINVAL, "batch must be >= 0");
  if (batch == 0) return PROGRESS_OK;
  if (!d_params_fp16 || !d_x || !d_y || !d_scratch)
    return lfail(PROGRESS_EINVAL, "NULL pointer argument");
  return lcuda(sp2::learned::forward_fp16(in, hidden, out, d_params_fp16, batch, d_x, d_y,
                                          d_scratch, (cudaStream_t)stream),
               "mlp forward launch");
}

progress_status_t progress_mlp_train_step(int32_t in, int32_t hidden, int32_t out,
                                          float* d_params, float* d_grad, float* d_m,
                                          float* d_v, int32_t step, float lr, int32_t batch,
                                          const float* d_x, const float* d_target,
                                          const float* d_mask, float* d_scratch, float* d_loss,
                                          void* stream) {
  if (!dims_ok(in, hidden, out)) return lfail(PROGRESS_EINVAL, "bad perceptron dimensions");
  if (batch < 1) return lfail(PROGRESS_EINVAL, "batch must be >= 1");
  if (lr != 0.0f && (step < 1 || !d_m || !d_v))
    return lfail(PROGRESS_EINVAL, "Adam needs step >= 1 and moment buffers");
  if (!d_params || !d_grad || !d_x || !d_target || !d_mask || !d_scratch)
    return lfail(PROGRESS_EINVAL, "NULL pointer argument");
  return lcuda(sp2::learned::train_step(in, hidden, out, d_params, d_grad, d_m, d_v, step, lr,
                                        batch, d_x, d_target, d_mask, d_scratch, d_loss,
                                        (cudaStream_t)stream),
               "mlp train step launch");
}

progress_status_t progress_learned_inputs(int32_t batch, int32_t nout, const float* d_y,
                                          const double* d_gersh, double margin, float logit_tau,
                                          double* d_bounds, uint64_t* d_bits, int32_t* d_len,
                                          void* stream) {
  if (batch < 0) return lfail(PROGRESS_EINVAL, "batch must be >= 0");
  if (nout < 3 || nout > 2 + 256) return lfail(PROGRESS_EINVAL, "nout must be in [3, 258]");
  if (!(margin >= 0.0) || !isfinite(margin)) return lfail(PROGRESS_EINVAL, "bad margin");
  if (batch == 0) return PROGRESS_OK;
  if (!d_y || !d_gersh || !d_bounds) return lfail(PROGRESS_EINVAL, "NULL pointer argument");
  return lcuda(sp2::learned::predict_inputs(batch, nout, d_y, d_gersh, margin, logit_tau,
                                            d_bounds, d_bits, d_len, (cudaStream_t)stream),
               "learned inputs launch");
}

progress_status_t progress_learned_targets(int32_t batch, int32_t kmax, const float* d_ub,
                                           int32_t ld_ub, const uint64_t* d_bits,
                                           const int32_t* d_iters, const int32_t* d_reject,
                                           float* d_target, float* d_mask, void* stream) {
  if (batch < 0) return lfail(PROGRESS_EINVAL, "batch must be >= 0");
  if (kmax < 1 || kmax > 256) return lfail(PROGRESS_EINVAL, "kmax must be in [1, 256]");
  if (ld_ub < 2) return lfail(PROGRESS_EINVAL, "ld_ub must be >= 2");
  if (batch == 0) return PROGRESS_OK;
  if (!d_ub || !d_target || !d_mask) return lfail(PROGRESS_EINVAL, "NULL pointer argument");
  return lcuda(sp2::learned::targets(batch, kmax, d_ub, ld_ub, d_bits, d_iters, d_reject,
                                     d_target, d_mask, (cudaStream_t)stream),
               "learned targets launch");
}

progress_status_t progress_learned_labels(int32_t batch, const int32_t* h_n,
                                          const int64_t* h_offset, const int32_t* d_n,
                                          const int64_t* d_offset, const double* dH, double tol,
                                          float* d_u, double* d_gersh, double* d_eps,
                                          void* stream) {
  if (batch < 0) return lfail(PROGRESS_EINVAL, "batch must be >= 0");
  if (batch == 0) return PROGRESS_OK;
  if (!h_n || !h_offset || !d_n || !d_offset || !dH || !d_u || !d_gersh)
    return lfail(PROGRESS_EINVAL, "NULL pointer argument");
  int64_t elems = 0;
  for (int i = 0; i < batch; ++i) {
    if (h_n[i] < 1 || h_offset[i] < 0) return lfail(PROGRESS_EINVAL, "bad batch layout");
    elems = std::max(elems, h_offset[i] + (int64_t)h_n[i] * h_n[i]);
  }
  cudaStream_t s = (cudaStream_t)stream;
  double *dD = nullptr, *dNeg = nullptr, *dE = nullptr;
  progress_status_t st = PROGRESS_OK;
  cudaError_t e = cudaMalloc(&dD, (size_t)elems * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&dNeg, (size_t)elems * sizeof(double));
  if (e == cudaSuccess && !d_eps) e = cudaMalloc(&dE, (size_t)2 * batch * sizeof(double));
  if (e != cudaSuccess) st = lcuda(e, "learned labels: work space allocation");
  double* eps = d_eps ? d_eps : dE;
  std::vector<int32_t> ones((size_t)batch, 1);
  progress_opts_t o;
  progress_opts_default(&o);
  o.prec = PROGRESS_FP32_SPLIT_BF16;  // FP32's exponent range: nocc = 1 squares entries small
  progress_batch_ex_t ex{};
  ex.d_bounds_out = d_gersh;
  // eps_1: the projector onto the lowest state of H, then Tr(H D)
  if (st == PROGRESS_OK)
    st = progress_sp2_batched_ex(batch, h_n, h_offset, ones.data(), dH, tol, dD, nullptr,
                                 nullptr, &o, &ex, stream);
  if (st == PROGRESS_OK) st = progress_trace_hd(batch, d_n, d_offset, dH, dD, eps, stream);
  // eps_N: the lowest state of -H is the highest of H
  if (st == PROGRESS_OK)
    st = lcuda(sp2::learned::negate(dH, elems, dNeg, s), "negate launch");
  ex.d_bounds_out = nullptr;
  if (st == PROGRESS_OK)
    st = progress_sp2_batched_ex(batch, h_n, h_offset, ones.data(), dNeg, tol, dD, nullptr,
                                 nullptr, &o, &ex, stream);
  if (st == PROGRESS_OK)
    st = progress_trace_hd(batch, d_n, d_offset, dH, dD, eps + batch, stream);
  if (st == PROGRESS_OK)
    st = lcuda(sp2::learned::bound_fractions(batch, eps, eps + batch, d_gersh, d_u, s),
               "bound fractions launch");
  if (st == PROGRESS_OK) st = lcuda(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  else cudaStreamSynchronize(s);
  if (dD) cudaFree(dD);
  if (dNeg) cudaFree(dNeg);
  if (dE) cudaFree(dE);
  return st;
}

progress_status_t progress_learned_margin(int32_t batch, const float* h_y, int32_t ld_y,
                                          const float* h_t, int32_t ld_t, double quantile,
                                          double floor, double* margin_out) {
  if (batch < 0 || ld_y < 2 || ld_t < 2) return lfail(PROGRESS_EINVAL, "bad sizes");
  if (!(quantile >= 0.0 && quantile <= 1.0)) return lfail(PROGRESS_EINVAL, "quantile in [0, 1]");
  if (!margin_out) return lfail(PROGRESS_EINVAL, "NULL margin_out");
  if (batch == 0) {
    *margin_out = floor;
    return PROGRESS_OK;
  }
  if (!h_y || !h_t) return lfail(PROGRESS_EINVAL, "NULL pointer argument");
  // overshoot of the predicted bound fractions over their targets, the larger
  // of the two per instance; its `quantile` (linear interpolation between
  // order statistics), never below `floor`
  std::vector<double> over((size_t)batch);
  for (int i = 0; i < batch; ++i) {
    const float* y = h_y + (size_t)i * ld_y;
    const float* t = h_t + (size_t)i * ld_t;
    over[i] = std::max(std::max((double)y[0] - (double)t[0], 0.0),
                       std::max((double)y[1] - (double)t[1], 0.0));
  }
  std::sort(over.begin(), over.end());
  const double pos = quantile * (double)(batch - 1);
  const int lo = (int)pos;
  const int hi = lo + 1 < batch ? lo + 1 : lo;
  const double q = over[lo] + (over[hi] - over[lo]) * (pos - (double)lo);
  *margin_out = std::max(floor, q);
  return PROGRESS_OK;
}

}  // extern "C"
