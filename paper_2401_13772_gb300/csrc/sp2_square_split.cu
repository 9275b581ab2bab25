// Split-precision SP2 product step on tcgen05 tensor cores (placeholder).
#include "sp2_common.cuh"
#include "sp2_launch.h"

namespace sp2 {

int split_tile_count(int ld) {
  const int T = ld / 128;
  return T * (T + 1) / 2;
}

cudaError_t launch_square_split(const DevBuffers& b, const SolveParams& p,
                                unsigned long long cond_handle, cudaStream_t s) {
  (void)b; (void)p; (void)cond_handle; (void)s;
  return cudaErrorNotSupported;
}

}  // namespace sp2
