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

// Launch configuration of the batched kernel (the autotuner's search space).
//   tile_n   width of a product tile (128 x tile_n outputs): 64 or 128
//   cluster  CTAs per thread-block cluster: 1, 2, 4 or 8
//   share    an instance with at least `share` 128-row blocks is solved by
//            the whole cluster (its tiles dealt round-robin to the CTAs);
//            smaller ones by one CTA each
struct Config {
  int32_t tile_n;
  int32_t cluster;
  int32_t share;
  int32_t pad;
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
  int32_t share;          // Config::share
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
  long long* cycles;      // [batch] SM clock cycles the instance took (may be null)
  const double* mu_in;    // [batch] chemical potentials (rule PROGRESS_RULE_MU)
};

// Valid configuration? (tile_n 64/128, cluster 1/2/4/8, share >= 1)
bool config_ok(const Config& c);

// CTAs the launch uses for `cfg` (a multiple of cfg.cluster; 0 on error).
int grid_size(const Config& cfg, int fmt, int batch);

cudaError_t launch(const Params& prm, const Config& cfg, int grid, cudaStream_t s);

}  // namespace batched
}  // namespace sp2
