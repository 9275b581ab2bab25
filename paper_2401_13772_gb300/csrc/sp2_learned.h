// Learned-sequence kernels: host-side launchers (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sp2 {
namespace learned {

constexpr int kFeatures = 37;
constexpr int kHistBins = 32;

int param_count(int in, int hid, int out);
int64_t train_scratch_floats(int in, int hid, int out, int batch);
cudaError_t features(int batch, const int32_t* d_n, const int64_t* d_off, const double* dH,
                     float* d_feat, cudaStream_t s);
cudaError_t trace_hd(int batch, const int32_t* d_n, const int64_t* d_off, const double* dH,
                     const double* dD, double* d_out, cudaStream_t s);
cudaError_t forward_fp16(int in, int hid, int out, const uint16_t* d_params_h, int batch,
                         const float* d_x, float* d_y, float* d_scratch, cudaStream_t s);
cudaError_t train_step(int in, int hid, int out, float* d_params, float* d_grad, float* d_m,
                       float* d_v, int step, float lr, int batch, const float* d_x,
                       const float* d_t, const float* d_mask, float* d_scratch, float* d_loss,
                       cudaStream_t s);
cudaError_t to_half(const float* d_params, int count, uint16_t* d_params_h, cudaStream_t s);
cudaError_t predict_inputs(int batch, int nout, const float* d_y, const double* d_gersh,
                           double margin, float tau, double* d_bounds, uint64_t* d_bits,
                           int32_t* d_len, cudaStream_t s);
cudaError_t targets(int batch, int kmax, const float* d_ub, int ld_ub, const uint64_t* d_bits,
                    const int32_t* d_iters, const int32_t* d_reject, float* d_t, float* d_m,
                    cudaStream_t s);
cudaError_t bound_fractions(int batch, const double* d_eps1, const double* d_epsN,
                            const double* d_gersh, float* d_u, cudaStream_t s);
cudaError_t negate(const double* d_x, int64_t count, double* d_y, cudaStream_t s);

}  // namespace learned
}  // namespace sp2
