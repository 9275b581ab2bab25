// Host-side launch wrappers of the SP2 kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sp2 {

struct State;
struct Slices;

// Pointers of one workspace, as the kernels see them.
struct DevBuffers {
  State* st;
  double* x64[2];        // FP64 ping-pong iterates, ld x ld
  uint16_t* sl[2][3];    // slice ping-pong sets, ld x ld each
  uint16_t* dg[5];       // BF16 fixed-point digits of the iterate (digit products):
                         // dg[0] holds digits 0..3 interleaved, ld x 4 ld (row r, column
                         // 64 g + 16 d + i = digit d of element 16 g + i); dg[4] holds
                         // digit 4, ld x ld; dg[1..3] are not used
  uint8_t* tflags[2];    // thresholded SP2: per 128 x 128 tile of slice set k, 1 if it may
                         // hold a non-zero ((ld/128)^2 bytes each)
  double* partials;      // per-CTA partial traces (2 doubles per CTA)
  int max_partials;
};

struct SolveParams {
  int64_t n;
  int ld;
  int64_t nocc;
  int rule;
  int maxiter;
  int prec;
  int fp64_prefix;
  int slice_fmt;
  int df64;  // FP64-accurate products in double-float (FP64 buffers hold hi/lo planes)
  int oz;    // ... computed as exact digit products on the tensor cores (needs df64)
  double tol;
  double emin_override, emax_override;
  float tau;  // thresholded SP2 cutoff (0 = dense)
  unsigned long long wait_ns;  // bound on each pipeline wait of the tensor-core kernels
  int stall_test;              // test of the bounded waits (see progress_opts_t)
  double floor_acc;            // MIXED: round-off floor of the refinement's idempotency
  int split_tile;              // FP16x2 split product: 0 / 1 = 128 x 128 tiles, 2 = 128 x 256
  int prefix_full;             // digit products of the MIXED prefix: 1 = all 15, 0 = 13
};

cudaError_t launch_init(const DevBuffers& b, const SolveParams& p, cudaStream_t s);
// Gershgorin bounds into st->emin/emax (unless overridden) and, if out_min and
// out_max are not null, into *out_min and *out_max.
cudaError_t launch_gershgorin(const double* H, int64_t n, const DevBuffers& b, double* out_min,
                              double* out_max, cudaStream_t s);
cudaError_t launch_x0(const double* H, const DevBuffers& b, const SolveParams& p, cudaStream_t s);
// One FP64 product step (no-op unless the state says the next product is FP64).
cudaError_t launch_square_fp64(const DevBuffers& b, int ld, int slice_fmt,
                               unsigned long long cond_handle, cudaStream_t s);
// One double-float product step on the FP32 pipe (no-op unless the next product
// is FP64-accurate).
cudaError_t launch_square_df64(const DevBuffers& b, int ld, int slice_fmt,
                               unsigned long long cond_handle, cudaStream_t s);
int df64_tile_count(int ld);
// Digits of the iterate, then one FP64-accurate product from exact BF16 digit
// products on the tensor cores (both no-ops unless the next product is
// FP64-accurate); ld <= oz_max_order().
cudaError_t launch_digits(const DevBuffers& b, int ld, cudaStream_t s);
cudaError_t launch_square_oz(const DevBuffers& b, int ld, int slice_fmt,
                             unsigned long long cond_handle, cudaStream_t s);
int oz_max_order();
// One split-precision tcgen05 product step (no-op unless the next product is split).
cudaError_t launch_square_split(const DevBuffers& b, const SolveParams& p,
                                unsigned long long cond_handle, cudaStream_t s);
bool split_tensor_maps_ready(const DevBuffers& b, int ld, int fmt);
// The FP16x2 split product on 128 x 256 tiles (one tcgen05.mma of N = 256 per
// product group); launch_square_split calls it when split_tile is 2.
cudaError_t launch_square_wide(const DevBuffers& b, const SolveParams& p,
                               unsigned long long cond_handle, cudaStream_t s);
// Thresholded SP2: tile flags of X0 into tflags[0] (a tile of H with a
// non-zero, or a diagonal tile) and "unknown content" into tflags[1].
cudaError_t launch_tile_flags(const double* H, int64_t n, int ld, const DevBuffers& b,
                              cudaStream_t s);
cudaError_t launch_finalize(const DevBuffers& b, double* D, int64_t n, int ld, int slice_fmt,
                            cudaStream_t s);

int fp64_tile_count(int ld);

// Record the text that progress_last_error() returns on this thread.
void set_last_error(const char* what);

// Free the batched, graph and Chebyshev work spaces of (dev, stream), or of every stream
// of dev; the caller has synchronized the stream (device).
void batched_release(int dev, cudaStream_t s, bool all_streams);
void graph_release(int dev, cudaStream_t s, bool all_streams);
void cheb_release(int dev, cudaStream_t s, bool all_streams);
int split_tile_count(int ld);

}  // namespace sp2
