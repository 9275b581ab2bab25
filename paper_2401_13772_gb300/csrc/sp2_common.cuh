// Shared device-side state and helpers of the SP2 solver kernels.
//
// The SP2 loop (§IV.A) keeps its whole control state on the device: the
// traces of the current iterate, the branch of the next product, the
// iteration count and the stop flag. Every product kernel's last CTA reduces
// the per-tile partial traces in a fixed order (deterministic), then decides
// the next step, so the host never reads a trace inside the loop.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "progress_sp2.h"

namespace sp2 {

constexpr int kMaxHist = 256;  // branch/idempotency history length (maxiter <= 250)

// Precision of one product.
enum Phase : int { kPhaseFP64 = 0, kPhaseSplit = 1, kPhaseRefine = 2 };

struct State {
  // solve parameters (written by the init kernel)
  int n;
  int ld;
  int nocc;
  int rule;
  int maxiter;
  int prec;
  int fp64_prefix;
  int slice_fmt;  // SliceFmt of the split products
  double tol;
  double emin_override;  // NaN = use Gershgorin
  double emax_override;
  // control state
  double emin, emax;  // bounds used for X0
  double t1, t2;      // Tr X_k and Tr X_k^2 = ||X_k||_F^2 of the current iterate
  double idem;        // |t2 - t1|
  int iter;           // products performed (k)
  int done;           // 1: stop the loop
  int converged;      // 1: idempotency below tol; 2: stopped on the round-off floor of
                      // the FP64-accurate refinement products (MIXED modes)
  int status;         // progress_status_t
  int bit;            // branch of the next product (1: 2X - X^2)
  int phase;          // Phase of the next product
  int phase_iters[3];
  int split_stall;    // consecutive split-phase steps without improvement
  int x_fp64_valid;   // the current iterate X_k is stored in FP64 (buffer k % 2)
  int x_slices_valid; // the current iterate X_k is stored as slices (set k % 2)
  int df64;           // the FP64 buffers hold double-float planes (hi, lo floats)
  unsigned int ticket;  // CTA arrival counter of the running launch
  double best_split_idem;
  // learned-sequence judge: predicted branch bits and the margin beyond which
  // a disagreement with the trace rule aborts the predicted run
  unsigned long long pred_bits[4];
  int pred_len;
  int judge_fail;
  double judge_delta;
  double y_mu;  // PROGRESS_RULE_MU: the chemical potential under the same map as X_k
  unsigned long long kblocks;  // thresholded SP2: 64-wide k-blocks streamed (all products)
  double floor_acc;            // MIXED: idempotency below which the FP64-accurate
                               // refinement has reached its products' round-off floor
  unsigned long long wait_ns;  // bound on each pipeline wait of the tensor-core kernels
  int stall_test;              // 1: CTA 0 of a tensor-core product waits on a barrier that
                               // nothing arrives on (test of the bounded waits)
  int prefix_full;             // MIXED, digit products: 1 = all 15 digit products in the
                               // FP64-accurate prefix too; 0 = 13 there (no x0 x4 pair),
                               // all 15 in the refinement
  unsigned long long bits[4];
  double idem_hist[kMaxHist];
  double margin_hist[kMaxHist];
};

// ---------------------------------------------------------------------------
// reductions

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum of two doubles in a fixed order; result valid in thread 0.
// `scratch` holds 2 * (blockDim.x / 32) doubles.
// Compensated FP32 sum (Kahan): s - c carries the running total. The epilogues
// use it for their partial traces instead of FP64 adds, which are slow on this
// part (a few FP64 operations per clock and SM).
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// v (|v| < 2^7) on the fixed-point grid 2^-40, as an integer: v 2^16 is split
// exactly into its integer part a and the rest, the rest is rounded at 2^-24 of
// the unit (so v at 2^-40), all in FP32 and 32-bit conversions. Sums of these
// integers are exact and do not depend on their order.
__host__ __device__ __forceinline__ long long fixed40(float v) {
  const float x = v * 65536.0f;     // exact
  const float a = rintf(x);         // |a| < 2^23: exact in FP32 and int32
  const float b = rintf((x - a) * 16777216.0f);  // x - a is exact; |b| <= 2^23
  return (long long)(int)a * 16777216LL + (long long)(int)b;
}

__device__ __forceinline__ void block_sum2(double& a, double& b, double* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
  __syncthreads();
  if (lane == 0) {
    scratch[wid] = a;
    scratch[nw + wid] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int w = 0; w < nw; ++w) {
      sa += scratch[w];
      sb += scratch[nw + w];
    }
    a = sa;
    b = sb;
  }
}

// ---------------------------------------------------------------------------
// SP2 control (§IV.A): convergence, divergence and the branch of the next
// product, from the FP64 traces of the current iterate X_k.

__device__ inline void decide(State* st) {
  const int k = st->iter;
  const double t1 = st->t1, t2 = st->t2;
  const double n = (double)st->n;
  const double idem = fabs(t2 - t1);
  st->idem = idem;
  if (k < kMaxHist) st->idem_hist[k] = idem;
  // The mapped spectrum must stay in [0, 1]: then 0 <= Tr X <= n and
  // Tr X^2 <= Tr X. A clear violation means the bounds did not enclose the
  // spectrum (or the input was not finite).
  const bool finite = isfinite(t1) && isfinite(t2);
  const bool escaped = t1 < -1e-6 * n - 1e-3 || t1 > n * (1.0 + 1e-6) + 1e-3 ||
                       t2 > t1 + 1e-3 * (n + 1.0);
  if (!finite || escaped) {
    st->status = PROGRESS_EBOUNDS;
    st->done = 1;
    return;
  }
  int phase = st->phase;
  bool stalled = false;
  bool refine_floor = false;
  if (st->prec == PROGRESS_FP64) {
    phase = kPhaseFP64;
  } else {
    if (st->prec == PROGRESS_FP32_SPLIT) {
      phase = kPhaseSplit;
    } else if (phase == kPhaseFP64 && k >= st->fp64_prefix) {
      // MIXED: the FP64 prefix is over, switch to split products.
      phase = kPhaseSplit;
      st->best_split_idem = idem;
      st->split_stall = 0;
    }
    if (phase == kPhaseSplit && k > 0) {
      // Low precision stops helping once the idempotency error sits on its
      // round-off floor, about n u for split operands (u ~ 2^-22). Above that
      // level the error is not a floor: SP2 can hold it on long plateaus or
      // oscillate (each eigenvalue still inside (0.01, 0.99) adds ~0.01 or
      // more; with few occupied states the error doubles for several steps
      // between drops). So: two steps without a 0.1 % improvement while below
      // 16 n 2^-22.
      const double floor_thr = 16.0 * n * 2.384185791015625e-07;
      if (idem < st->best_split_idem * 0.999) {
        st->best_split_idem = idem;
        st->split_stall = 0;
      } else {
        ++st->split_stall;
        if (st->split_stall >= 2 && idem < floor_thr) stalled = true;
      }
      // MIXED: leave room for the FP64 refinement before maxiter.
      if (st->prec != PROGRESS_FP32_SPLIT && k >= st->maxiter - 10) stalled = true;
    }
    if (stalled && st->prec != PROGRESS_FP32_SPLIT) {  // MIXED: start the refinement
      phase = kPhaseRefine;
      st->best_split_idem = idem;
      st->split_stall = 0;
    } else if (phase == kPhaseRefine) {
      // Refinement converges quadratically down to the round-off floor of
      // its FP64-accurate products, about n times their absolute error u:
      // once the idempotency error is below 2 n u (floor_acc) and the trace
      // is within n u / 2 of Nocc, further products only add noise (measured:
      // the error then wanders up, not down). Two steps that do not halve the
      // error also mean the floor is reached.
      if (idem < st->floor_acc && fabs(t1 - (double)st->nocc) < 0.25 * st->floor_acc)
        refine_floor = true;
      if (idem < st->best_split_idem * 0.5) {
        st->best_split_idem = idem;
        st->split_stall = 0;
      } else if (++st->split_stall >= 2 && idem < 1e-6 * n) {
        refine_floor = true;
      }
    }
  }
  st->phase = phase;
  if (stalled && st->prec == PROGRESS_FP32_SPLIT) {
    // All-split mode: the round-off floor is the answer.
    st->converged = 1;
    st->done = 1;
    return;
  }
  // Convergence is tested in FP64-accurate phases and in the all-split mode.
  if (((phase != kPhaseSplit || st->prec == PROGRESS_FP32_SPLIT) && idem < st->tol) ||
      refine_floor) {
    st->converged = idem < st->tol ? 1 : 2;
    st->done = 1;
    return;
  }
  if (k >= st->maxiter) {
    st->status = PROGRESS_ENOCONV;
    st->done = 1;
    return;
  }
  const double nocc = (double)st->nocc;
  int b;
  double margin;
  if (st->rule == PROGRESS_RULE_MU) {
    // fixed chemical potential: the branch keeps the mapped mu near 1/2
    margin = 0.5 - st->y_mu;
    b = st->y_mu > 0.5 ? 0 : 1;
  } else if (st->rule == PROGRESS_RULE_PAPER) {
    margin = nocc - t1;
    b = (t1 - nocc) <= 0.0 ? 1 : 0;
  } else {
    const double d_square = fabs(t2 - nocc);
    const double d_expand = fabs(2.0 * t1 - t2 - nocc);
    margin = d_square - d_expand;
    b = margin > 1e-12 * fmax(n, 1.0) ? 1 : 0;
  }
  if (k < st->pred_len) {
    // Judge of a predicted branch sequence: the trace rule still runs; a
    // disagreement beyond the margin stops this run (the caller restarts the
    // instance on the plain path), a near-tie follows the prediction.
    const int pb = (int)((st->pred_bits[k >> 6] >> (k & 63)) & 1ull);
    if (pb != b) {
      if (fabs(margin) > st->judge_delta) {
        st->judge_fail = 1;
        st->done = 1;
        if (k < kMaxHist) st->margin_hist[k] = margin;
        return;
      }
      b = pb;
    }
  }
  st->bit = b;
  if (st->rule == PROGRESS_RULE_MU) {  // the mapped mu follows the branch taken
    const double y = st->y_mu;
    st->y_mu = b ? 2.0 * y - y * y : y * y;
  }
  if (k < kMaxHist) {
    st->margin_hist[k] = margin;
    if (b) st->bits[k >> 6] |= 1ull << (k & 63);
  }
}

// Ticket of a CTA that finished its tile; true for the last CTA of the grid.
// Caller must have written its partials before, by thread 0.
__device__ __forceinline__ bool last_cta_arrives(State* st, unsigned int total, int* flag_smem) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int t = atomicAdd(&st->ticket, 1u);
    *flag_smem = (t == total - 1) ? 1 : 0;
  }
  __syncthreads();
  const bool last = *flag_smem != 0;
  if (last) __threadfence();
  return last;
}

// Deterministic sum of `count` pairs (a, b) stored interleaved; valid in thread 0.
__device__ inline void reduce_partials(const double* partials, int count, double& a, double& b,
                                       double* scratch) {
  double sa = 0.0, sb = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    sa += __ldcg(partials + 2 * i);
    sb += __ldcg(partials + 2 * i + 1);
  }
  block_sum2(sa, sb, scratch);
  a = sa;
  b = sb;
}

}  // namespace sp2
