// C ABI of the learned-sequence part (features, Tr(HD), perceptron).
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

}  // extern "C"
