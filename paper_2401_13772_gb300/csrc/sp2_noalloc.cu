// progress_sp2_dense_noalloc: the FP64 SP2 solve without any device memory
// allocation, for callers that cannot call cudaMalloc -- applications whose
// own memory pool has already reserved the whole device (a cudaMalloc from the
// library would fail or fragment that pool), and time-stepping codes (quantum
// molecular dynamics calls the solver every step) that must not see allocation
// latency or the device-wide synchronization that cudaFree implies.
//
// Its work space -- the two FP64 ping-pong iterates, the per-CTA partial
// traces and the solve state -- lives in one file-scope __device__ array of
// fixed size, so every GPU that loads the library holds those bytes until
// the process exits. The limit is n <= 1024 (ld <= 1024, 16 MiB of iterates).
// In host code the array's name is only a host-side stand-in, not a device
// address: its device address is looked up once per device with
// cudaGetSymbolAddress, on the first call made on that device (with that
// device current). That first call should therefore come before any stream
// capture begins.
//
// Every call on a device shares the array and it keeps the last call's
// contents; the solve clears what must start at zero (the state) itself.
// Calls whose work overlaps on the GPU (two streams at once) race on the
// array: serialize them.
#include <string.h>

#include <mutex>

#include "progress_sp2.h"
#include "sp2_common.cuh"
#include "sp2_launch.h"
#include "sp2_slices.cuh"

namespace {

constexpr int kNoAllocMaxLd = 1024;
constexpr size_t kIterBytes = (size_t)kNoAllocMaxLd * kNoAllocMaxLd * sizeof(double);
constexpr int kNoAllocPartials = 152 * 8;  // >= every launch's CTA count at ld <= 1024
constexpr size_t kPartialBytes = (size_t)kNoAllocPartials * 2 * sizeof(double);
constexpr size_t kStateBytes = (sizeof(sp2::State) + 255) / 256 * 256;
constexpr size_t kScratchBytes = 2 * kIterBytes + kPartialBytes + kStateBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};

progress_status_t noalloc_fail(progress_status_t s, const char* what) {
  sp2::set_last_error(what);  // reported by progress_last_error()
  return s;
}

}  // namespace

extern "C" progress_status_t progress_sp2_dense_noalloc(const double* dH, int64_t n, int64_t nocc,
                                                        double tol, double* dD, void* stream) {
  if (n < 0 || n > kNoAllocMaxLd)
    return noalloc_fail(PROGRESS_EINVAL, "n must be in [0, 1024] for the no-allocation solve");
  if (nocc < 0 || nocc > n) return noalloc_fail(PROGRESS_EINVAL, "nocc must be in [0, n]");
  if (!(tol >= 0.0)) return noalloc_fail(PROGRESS_EINVAL, "tol must be >= 0");
  if (n == 0) return PROGRESS_OK;
  if (!dH || !dD || dH == dD) return noalloc_fail(PROGRESS_EINVAL, "bad matrix pointers");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(PROGRESS_ECUDA, "cudaGetDevice failed");
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return noalloc_fail(PROGRESS_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
      }
      g_noalloc_ptr[dev] = p;
    }
    base = g_noalloc_ptr[dev];
  }
  unsigned char* b = static_cast<unsigned char*>(base);
  sp2::DevBuffers buf;
  memset(&buf, 0, sizeof buf);
  buf.x64[0] = reinterpret_cast<double*>(b);
  buf.x64[1] = reinterpret_cast<double*>(b + kIterBytes);
  buf.partials = reinterpret_cast<double*>(b + 2 * kIterBytes);
  buf.max_partials = kNoAllocPartials;
  buf.st = reinterpret_cast<sp2::State*>(b + 2 * kIterBytes + kPartialBytes);

  sp2::SolveParams p;
  memset(&p, 0, sizeof p);
  p.n = n;
  p.ld = (int)((n + 127) / 128 * 128);
  p.nocc = nocc;
  p.rule = PROGRESS_RULE_NEARER;
  p.maxiter = 100;
  p.prec = PROGRESS_FP64;
  p.slice_fmt = sp2::kFP16x2;
  p.tol = tol;
  p.emin_override = __builtin_nan("");
  p.emax_override = __builtin_nan("");
  cudaStream_t s = (cudaStream_t)stream;
  // Plain launches only (no graph is instantiated): the product kernels exit
  // at once after the device-side stop flag is set.
  if (sp2::launch_init(buf, p, s) != cudaSuccess ||
      sp2::launch_gershgorin(dH, n, buf, nullptr, nullptr, s) != cudaSuccess ||
      sp2::launch_x0(dH, buf, p, s) != cudaSuccess)
    return noalloc_fail(PROGRESS_ECUDA, "kernel launch failed");
  for (int i = 0; i <= p.maxiter; ++i)
    if (sp2::launch_square_fp64(buf, p.ld, p.slice_fmt, 0ull, s) != cudaSuccess)
      return noalloc_fail(PROGRESS_ECUDA, "kernel launch failed");
  if (sp2::launch_finalize(buf, dD, n, p.ld, p.slice_fmt, s) != cudaSuccess)
    return noalloc_fail(PROGRESS_ECUDA, "kernel launch failed");
  return PROGRESS_OK;
}
