// Batched SP2 solver: host/device interface (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sp2 {
namespace batched {

struct Instance {
  int32_t n;       // matrix order
  int32_t m;       // padded order (multiple of 128)
  int32_t nocc;    // occupied states
  int32_t pad;
  int64_t row0;    // first row in the tall slice matrices
  int64_t offset;  // element offset of H and D in the packed input/output
};

struct InstanceInfo {
  double emin, emax, idem;
  int32_t converged, pad;
  unsigned long long bits[4];
};

struct Params {
  const Instance* inst;   // [batch]
  const int32_t* order;   // [batch] instance indices, largest first
  int32_t* queue;         // work counter (zeroed before the launch)
  int32_t batch;
  int32_t rule;
  int32_t maxiter;
  int32_t pitch;          // P = max padded order (row pitch of the slice matrices)
  int64_t total_rows;     // sum of padded orders
  double tol;
  const double* H;        // packed inputs
  double* D;              // packed outputs
  int32_t fmt;            // SliceFmt: kFP16x2 or kBF16x3
  uint16_t* sl[2][3];     // [set][slice] tall slice matrices, total_rows x pitch
  // learned-sequence inputs/outputs (all optional)
  const double* bounds_in;               // [batch][2] emin, emax (NaN = Gershgorin)
  const unsigned long long* pred_bits;   // [batch][4]
  const int32_t* pred_len;               // [batch]
  double judge_delta;
  unsigned long long* bits_out;          // [batch][4]
  double* bounds_out;                    // [batch][2]
  int32_t* fallback;                     // [batch]
  int32_t* products;                     // [batch] products including a rejected attempt
  int32_t* iters;         // [batch] products per instance (may be null)
  int32_t* status;        // [batch] progress_status_t per instance (may be null)
  InstanceInfo* info;     // [batch] optional details
};

cudaError_t launch(const Params& prm, int grid, cudaStream_t s);

}  // namespace batched
}  // namespace sp2
