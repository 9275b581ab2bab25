// O(n^2) kernels of the SP2 solver: state init, Gershgorin bounds (§VIII.A),
// the X0 map (§IV.A) and the final copy of the converged iterate into D.
// All are HBM-bound streams over the matrix; rows are read by whole warps
// (coalesced), partial sums are combined in a fixed order.
#include <math.h>

#include "sp2_common.cuh"
#include "sp2_launch.h"
#include "sp2_slices.cuh"

namespace sp2 {

namespace {

constexpr int kEwThreads = 256;
constexpr int kEwMaxBlocks = 152 * 8;

__global__ void init_kernel(State* st, SolveParams p) {
  // zero the whole state, then write the parameters
  const int words = sizeof(State) / sizeof(unsigned int);
  unsigned int* w = reinterpret_cast<unsigned int*>(st);
  for (int i = threadIdx.x; i < words; i += blockDim.x) w[i] = 0u;
  __syncthreads();
  if (threadIdx.x == 0) {
    st->n = (int)p.n;
    st->ld = p.ld;
    st->nocc = (int)p.nocc;
    st->rule = p.rule;
    st->maxiter = p.maxiter;
    st->prec = p.prec;
    st->fp64_prefix = p.fp64_prefix;
    st->slice_fmt = p.slice_fmt;
    st->df64 = p.df64;
    st->tol = p.tol;
    st->emin_override = p.emin_override;
    st->emax_override = p.emax_override;
    st->best_split_idem = INFINITY;
    st->wait_ns = p.wait_ns;
    st->floor_acc = p.floor_acc;
    st->stall_test = p.stall_test;
    st->prefix_full = p.prefix_full;
    st->phase = (p.prec == PROGRESS_FP32_SPLIT) ? kPhaseSplit : kPhaseFP64;
  }
}

// Exact sums of |x| over doubles with integer arithmetic only (GB300 issues
// FP64 adds at a small fraction of its integer rate, and one add per entry
// bounded the plain FP64 row sum at 0.18 of HBM). A 128-bit unsigned
// fixed-point accumulator counts units of 2^(E - 1133), E the largest biased
// exponent added so far: an entry |x| = m 2^(e - 1075) with a 53-bit m is m
// shifted left by e - E + 58 <= 58 bits, below 2^111, so 2^16 entries fit.
// When a larger exponent arrives the accumulator is shifted right to the new
// unit, dropping bits 2^-58 below the new largest entry. The sum is rounded to
// double once at the end: it is more accurate than a sum of FP64 adds.
struct AbsSum {
  unsigned long long lo, hi;  // the 128-bit value
  int E;                      // biased exponent of the unit (0: nothing added yet)
  int special;                // an infinity or NaN was added
};

__device__ __forceinline__ void abs_sum_shift(AbsSum& a, int d) {  // a >>= d, d >= 0
  if (d <= 0) return;
  if (d >= 128) {
    a.lo = 0ull;
    a.hi = 0ull;
  } else if (d >= 64) {
    a.lo = a.hi >> (d - 64);
    a.hi = 0ull;
  } else {
    a.lo = (a.lo >> d) | (a.hi << (64 - d));
    a.hi >>= d;
  }
}

__device__ __forceinline__ void abs_sum_add(AbsSum& a, double x) {
  const unsigned long long u =
      (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
  if (u == 0ull) return;
  int e = (int)(u >> 52);
  if (e == 0x7ff) {
    a.special = 1;
    return;
  }
  unsigned long long m = u & 0xfffffffffffffull;
  if (e == 0) {
    e = 1;  // subnormal: m 2^(1 - 1075)
  } else {
    m |= 1ull << 52;
  }
  if (e > a.E) {
    abs_sum_shift(a, a.E == 0 ? 128 : e - a.E);
    a.E = e;
  }
  const int sh = e - a.E + 58;
  unsigned long long vl, vh = 0ull;
  if (sh >= 0) {
    vl = m << sh;
    if (sh > 0) vh = m >> (64 - sh);
  } else {
    vl = sh > -64 ? (m >> -sh) : 0ull;
  }
  a.lo += vl;
  a.hi += vh + (a.lo < vl ? 1ull : 0ull);
}

__device__ __forceinline__ void abs_sum_merge(AbsSum& a, AbsSum b) {
  if (b.E > a.E) {
    abs_sum_shift(a, a.E == 0 ? 128 : b.E - a.E);
    a.E = b.E;
  } else {
    abs_sum_shift(b, b.E == 0 ? 128 : a.E - b.E);
  }
  a.lo += b.lo;
  a.hi += b.hi + (a.lo < b.lo ? 1ull : 0ull);
  a.special |= b.special;
}

__device__ __forceinline__ AbsSum abs_sum_warp(AbsSum a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    AbsSum b;
    b.lo = __shfl_xor_sync(0xffffffffu, a.lo, o);
    b.hi = __shfl_xor_sync(0xffffffffu, a.hi, o);
    b.E = __shfl_xor_sync(0xffffffffu, a.E, o);
    b.special = __shfl_xor_sync(0xffffffffu, a.special, o);
    abs_sum_merge(a, b);
  }
  return a;
}

__device__ __forceinline__ double abs_sum_value(const AbsSum& a) {
  // an infinite or NaN entry: an infinite radius, so the bounds are not finite
  // and the solve reports EBOUNDS
  if (a.special) return INFINITY;
  if (a.E == 0) return 0.0;
  const double v = __ull2double_rn(a.hi) * 18446744073709551616.0 + __ull2double_rn(a.lo);
  return ldexp(v, a.E - 1133);
}

// One warp per row: R_i = sum_{j != i} |H_ij| (exact fixed-point sums, above);
// per-block min(H_ii - R_i) and max(H_ii + R_i), then the last block combines
// the block results.
__global__ void __launch_bounds__(kEwThreads) gershgorin_kernel(const double* __restrict__ H,
                                                                int64_t n, State* st,
                                                                double* __restrict__ blk,
                                                                double* __restrict__ out_min,
                                                                double* __restrict__ out_max) {
  __shared__ double s_lo[kEwThreads / 32], s_hi[kEwThreads / 32];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t warps = (int64_t)gridDim.x * (kEwThreads / 32);
  double lo = INFINITY, hi = -INFINITY;
  for (int64_t i = (int64_t)blockIdx.x * (kEwThreads / 32) + wid; i < n; i += warps) {
    const double* row = H + i * n;
    AbsSum acc{0ull, 0ull, 0, 0};
    int64_t j = 0;
    if ((n & 1) == 0 && (reinterpret_cast<uintptr_t>(H) & 15u) == 0) {
      // rows start on 16 bytes: pairs of entries, four 16-byte loads in flight
      // per lane (eight entries)
      const double2* row2 = reinterpret_cast<const double2*>(row);
      const int64_t np = n >> 1;
      int64_t q = lane;
      for (; q + 96 < np; q += 128) {
        double2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = __ldcs(row2 + q + 32 * u);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t jj = 2 * (q + 32 * u);
          abs_sum_add(acc, jj == i ? 0.0 : v[u].x);
          abs_sum_add(acc, jj + 1 == i ? 0.0 : v[u].y);
        }
      }
      for (; q < np; q += 32) {
        const double2 v = __ldcs(row2 + q);
        abs_sum_add(acc, 2 * q == i ? 0.0 : v.x);
        abs_sum_add(acc, 2 * q + 1 == i ? 0.0 : v.y);
      }
    } else {
      for (j = lane; j + 96 < n; j += 128) {  // four loads in flight per lane
        const double v0 = __ldcs(row + j), v1 = __ldcs(row + j + 32);
        const double v2 = __ldcs(row + j + 64), v3 = __ldcs(row + j + 96);
        abs_sum_add(acc, j == i ? 0.0 : v0);
        abs_sum_add(acc, j + 32 == i ? 0.0 : v1);
        abs_sum_add(acc, j + 64 == i ? 0.0 : v2);
        abs_sum_add(acc, j + 96 == i ? 0.0 : v3);
      }
      for (; j < n; j += 32) abs_sum_add(acc, j == i ? 0.0 : __ldcs(row + j));
    }
    const double r = abs_sum_value(abs_sum_warp(acc));
    const double d = row[i];
    lo = fmin(lo, d - r);
    hi = fmax(hi, d + r);
  }
  lo = warp_min(lo);
  hi = warp_max(hi);
  if (lane == 0) {
    s_lo[wid] = lo;
    s_hi[wid] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kEwThreads / 32; ++w) {
      lo = fmin(lo, s_lo[w]);
      hi = fmax(hi, s_hi[w]);
    }
    blk[2 * blockIdx.x] = lo;
    blk[2 * blockIdx.x + 1] = hi;
  }
  if (!last_cta_arrives(st, gridDim.x, &s_last)) return;
  if (threadIdx.x == 0) {
    lo = INFINITY;
    hi = -INFINITY;
    for (unsigned b = 0; b < gridDim.x; ++b) {
      lo = fmin(lo, __ldcg(blk + 2 * b));
      hi = fmax(hi, __ldcg(blk + 2 * b + 1));
    }
    double e0 = isnan(st->emin_override) ? lo : st->emin_override;
    double e1 = isnan(st->emax_override) ? hi : st->emax_override;
    // A zero-width enclosure (H = c I, or n = 1) leaves the X0 map undefined;
    // widen it by 1 on each side, which still encloses the spectrum.
    if (!(e1 > e0)) {
      e0 -= 1.0;
      e1 += 1.0;
    }
    st->emin = e0;
    st->emax = e1;
    if (out_min && out_max) {
      *out_min = lo;
      *out_max = hi;
    }
    st->ticket = 0u;
  }
}

// X0 = (emax I - H) / (emax - emin) on the n x n block, zero padding up to
// ld x ld; writes the FP64 iterate and/or its slices; reduces Tr X0 and
// ||X0||_F^2 and decides the first product.
template <int F>
__global__ void __launch_bounds__(kEwThreads) x0_kernel(const double* __restrict__ H, State* st,
                                                        double* __restrict__ X, Slices S,
                                                        int write_fp64, int write_slices,
                                                        double* __restrict__ partials) {
  __shared__ double scratch[2 * kEwThreads / 32];
  __shared__ int s_last;
  const int64_t n = st->n;
  const int ld = st->ld;
  const double emax = st->emax, width = st->emax - st->emin;
  const double inv_w = 1.0 / width;  // one division per thread (FP64 division is slow here)
  const bool df64 = st->df64 != 0;
  float* Xf = reinterpret_cast<float*>(X);
  const size_t plane = (size_t)ld * ld;
  double tr = 0.0, fr = 0.0;
  if (write_fp64) {
    for (int64_t r = blockIdx.x; r < ld; r += gridDim.x) {
      for (int64_t c = threadIdx.x; c < ld; c += kEwThreads) {
        const size_t idx = (size_t)r * ld + c;
        double x = 0.0;
        if (r < n && c < n) {
          const double h = H[r * n + c];
          x = ((r == c) ? (emax - h) : -h) * inv_w;
          if (r == c) tr += x;
          fr += x * x;
        }
        if (df64) {
          const float h = (float)x;
          Xf[idx] = h;
          Xf[plane + idx] = (float)(x - (double)h);
        } else {
          X[idx] = x;
        }
        if (write_slices) store_slices<F>(S, idx, x);
      }
    }
  } else {
    // split products from the start: X0 is only needed as slices (22 / 24
    // significant bits), so it is formed in FP32 (one FP64-to-FP32 conversion
    // per element) and the traces are summed in FP32 along each row segment,
    // then folded into FP64
    const float emax_f = (float)emax, inv_w_f = (float)inv_w;
    for (int64_t r = blockIdx.x; r < ld; r += gridDim.x) {
      float frf = 0.0f;
      for (int64_t c = threadIdx.x; c < ld; c += kEwThreads) {
        const size_t idx = (size_t)r * ld + c;
        float x = 0.0f;
        if (r < n && c < n) {
          const float h = (float)H[r * n + c];
          x = ((r == c) ? (emax_f - h) : -h) * inv_w_f;
          if (r == c) tr += (double)x;
          frf += x * x;
        }
        uint16_t a, b, cc;
        split_value_f<F>(x, a, b, cc);
        S.s[0][idx] = a;
        S.s[1][idx] = b;
        if (fmt_bf16(F)) S.s[2][idx] = cc;
      }
      fr += (double)frf;
    }
  }
  block_sum2(tr, fr, scratch);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = tr;
    partials[2 * blockIdx.x + 1] = fr;
  }
  if (!last_cta_arrives(st, gridDim.x, &s_last)) return;
  double a, b;
  reduce_partials(partials, gridDim.x, a, b, scratch);
  if (threadIdx.x == 0) {
    st->t1 = a;
    st->t2 = b;
    st->iter = 0;
    st->x_fp64_valid = write_fp64;
    st->x_slices_valid = write_slices;
    st->ticket = 0u;
    decide(st);
  }
}

// ---------------------------------------------------------------------------
// X0 as double-float planes (hi, lo floats) without FP64 arithmetic, for the
// solves whose FP64-accurate products keep the iterate as double-float (digit
// and double-float products). GB300 issues FP64 arithmetic and FP64 <-> FP32
// conversions at a small fraction of the FP32 rate, so the plain X0 kernel was
// bound by them (1.2 ms at n = 8192); here each entry of H is cut into two
// floats with integer operations and the map is evaluated in double-float
// arithmetic (about 2^-46 relative accuracy, below the 2^-40 absolute error
// of one digit product).

// x = hi + lo with hi the 24-bit truncation of x and lo the rest rounded to 24
// bits (|x - hi - lo| <= 2^-48 |x|); zero stays zero. Entries outside
// [2^-74, 2^127] in magnitude take an FP64 path.
__device__ __forceinline__ void split_df(double x, float& hi, float& lo) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  if ((u << 1) == 0ull) {
    hi = 0.0f;
    lo = 0.0f;
    return;
  }
  const int e = (int)((u >> 52) & 0x7ffull);
  if (e < 949 || e > 1150) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
    return;
  }
  const unsigned int sign = (unsigned int)(u >> 63) << 31;
  const unsigned long long m = u & 0xfffffffffffffull;
  hi = __uint_as_float(sign | ((unsigned int)(e - 896) << 23) | (unsigned int)(m >> 29));
  const float scale = __uint_as_float((unsigned int)(e - 948) << 23);  // 2^(e - 1075)
  const float l = __uint2float_rn((unsigned int)(m & 0x1fffffffull)) * scale;
  lo = sign ? -l : l;
}

__device__ __forceinline__ void fast_two_sum_f(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}

__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = a + b;
  const float v = s - a;
  e = (a - (s - v)) + (b - v);
}

// (ah + al) (bh + bl) in double-float
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float& rh,
                                       float& rl) {
  const float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  fast_two_sum_f(p, e, rh, rl);
}

// acc += (xh + xl) in double-float
__device__ __forceinline__ void df_acc(float& ch, float& cl, float xh, float xl) {
  float s, t;
  two_sum_f(ch, xh, s, t);
  t += cl + xl;
  fast_two_sum_f(s, t, ch, cl);
}

__global__ void __launch_bounds__(kEwThreads) x0_df_kernel(const double* __restrict__ H,
                                                            State* st, float* __restrict__ Xf,
                                                            double* __restrict__ partials) {
  __shared__ double scratch[2 * kEwThreads / 32];
  __shared__ int s_last;
  const int64_t n = st->n;
  const int ld = st->ld;
  const size_t plane = (size_t)ld * ld;
  // emax and 1 / (emax - emin) as double-float pairs (a handful of FP64
  // operations per thread)
  const double emax = st->emax;
  const double inv_w = 1.0 / (st->emax - st->emin);
  float eh, el, ih, il;
  eh = (float)emax;
  el = (float)(emax - (double)eh);
  ih = (float)inv_w;
  il = (float)(inv_w - (double)ih);
  float trh = 0.0f, trl = 0.0f, frh = 0.0f, frl = 0.0f;
  // X0 entry (r, c) from h (inside the n x n block) as a double-float pair
  auto entry = [&](int64_t r, int64_t c, double h, float& xh, float& xl) {
    float hh, hl;
    split_df(h, hh, hl);
    if (r == c) {  // emax - h
      float s, t;
      two_sum_f(eh, -hh, s, t);
      t += el - hl;
      fast_two_sum_f(s, t, hh, hl);
      df_mul(hh, hl, ih, il, xh, xl);
      df_acc(trh, trl, xh, xl);
    } else {
      df_mul(-hh, -hl, ih, il, xh, xl);
    }
    // x^2 in double-float (xl^2 is below the pair's precision)
    const float p = xh * xh;
    const float e = fmaf(xh, xh, -p) + 2.0f * xh * xl;
    df_acc(frh, frl, p, e);
  };
  // four consecutive entries per thread and step: two 16-byte loads of H (rows
  // start on 16 bytes when n is even) and one 16-byte store per plane
  const bool vec = (n & 1) == 0 && (reinterpret_cast<uintptr_t>(H) & 15u) == 0;
  for (int64_t r = blockIdx.x; r < ld; r += gridDim.x) {
    const double* Hr = H + r * n;
#pragma unroll 2
    for (int64_t c = 4 * threadIdx.x; c < ld; c += 4 * kEwThreads) {
      double h[4];
      bool in[4];
      if (vec && r < n && c + 3 < n) {
        const double2 a = __ldcs(reinterpret_cast<const double2*>(Hr + c));
        const double2 b = __ldcs(reinterpret_cast<const double2*>(Hr + c + 2));
        h[0] = a.x;
        h[1] = a.y;
        h[2] = b.x;
        h[3] = b.y;
#pragma unroll
        for (int e = 0; e < 4; ++e) in[e] = true;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          in[e] = r < n && c + e < n;
          h[e] = in[e] ? Hr[c + e] : 0.0;
        }
      }
      float xh[4], xl[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        xh[e] = 0.0f;
        xl[e] = 0.0f;
        if (in[e]) entry(r, c + e, h[e], xh[e], xl[e]);
      }
      const size_t idx = (size_t)r * ld + c;
      *reinterpret_cast<float4*>(Xf + idx) = make_float4(xh[0], xh[1], xh[2], xh[3]);
      *reinterpret_cast<float4*>(Xf + plane + idx) = make_float4(xl[0], xl[1], xl[2], xl[3]);
    }
  }
  double tr = (double)trh + (double)trl, fr = (double)frh + (double)frl;
  block_sum2(tr, fr, scratch);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = tr;
    partials[2 * blockIdx.x + 1] = fr;
  }
  if (!last_cta_arrives(st, gridDim.x, &s_last)) return;
  double a, b;
  reduce_partials(partials, gridDim.x, a, b, scratch);
  if (threadIdx.x == 0) {
    st->t1 = a;
    st->t2 = b;
    st->iter = 0;
    st->x_fp64_valid = 1;
    st->x_slices_valid = 0;
    st->ticket = 0u;
    decide(st);
  }
}

// D (n x n, leading dim n) <- the current iterate, from FP64 if it is stored
// that way, else from its slices.
template <int F>
__global__ void __launch_bounds__(kEwThreads) finalize_kernel(const State* __restrict__ st,
                                                              DevBuffers b, double* __restrict__ D,
                                                              int64_t n) {
  const int ld = st->ld;
  const int k = st->iter & 1;
  const bool from64 = st->x_fp64_valid != 0;
  const double* X = b.x64[k];
  const float* Xf = reinterpret_cast<const float*>(b.x64[k]);
  const size_t plane = (size_t)ld * ld;
  const bool df64 = st->df64 != 0;
  const uint16_t* s0 = b.sl[k][0];
  const uint16_t* s1 = b.sl[k][1];
  const uint16_t* s2 = b.sl[k][2];
  for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
    for (int64_t c = threadIdx.x; c < n; c += kEwThreads) {
      const size_t src = (size_t)r * ld + c;
      double v;
      if (from64) {
        v = df64 ? (double)Xf[src] + (double)Xf[plane + src] : X[src];
      } else if (!fmt_bf16(F)) {
        // joined in FP32 (FP64 arithmetic is scarce here): within 2^-24 of the
        // value, below the 2^-22 resolution of the two FP16 slices themselves
        v = (double)join_value<F>(s0[src], s1[src], (uint16_t)0);
      } else {
        v = join_value_d<F>(s0[src], s1[src], s2[src]);
      }
      D[r * n + c] = v;
    }
  }
}

int ew_blocks(int64_t rows) {
  int64_t b = rows;
  if (b > kEwMaxBlocks) b = kEwMaxBlocks;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

cudaError_t launch_init(const DevBuffers& b, const SolveParams& p, cudaStream_t s) {
  init_kernel<<<1, 256, 0, s>>>(b.st, p);
  return cudaGetLastError();
}

cudaError_t launch_gershgorin(const double* H, int64_t n, const DevBuffers& b, double* out_min,
                              double* out_max, cudaStream_t s) {
  int64_t blocks = (n + kEwThreads / 32 - 1) / (kEwThreads / 32);
  if (blocks > kEwMaxBlocks) blocks = kEwMaxBlocks;
  if (blocks > b.max_partials) blocks = b.max_partials;
  gershgorin_kernel<<<(int)blocks, kEwThreads, 0, s>>>(H, n, b.st, b.partials, out_min, out_max);
  return cudaGetLastError();
}

cudaError_t launch_x0(const double* H, const DevBuffers& b, const SolveParams& p, cudaStream_t s) {
  const bool split_first =
      p.prec == PROGRESS_FP32_SPLIT || (p.prec != PROGRESS_FP64 && p.fp64_prefix == 0);
  const int write_fp64 = split_first ? 0 : 1;
  const int write_slices = split_first ? 1 : 0;
  int blocks = ew_blocks(p.ld);
  if (blocks > b.max_partials) blocks = b.max_partials;
  if (write_fp64 && p.df64) {  // double-float planes, no FP64 arithmetic per entry
    x0_df_kernel<<<blocks, kEwThreads, 0, s>>>(H, b.st, reinterpret_cast<float*>(b.x64[0]),
                                               b.partials);
    return cudaGetLastError();
  }
  Slices S;
  for (int i = 0; i < 3; ++i) S.s[i] = b.sl[0][i];
  switch (p.slice_fmt) {
#define SP2_X0(F)                                                                         \
  case F:                                                                                 \
    x0_kernel<F><<<blocks, kEwThreads, 0, s>>>(H, b.st, b.x64[0], S, write_fp64, write_slices, \
                                               b.partials);                              \
    break;
    SP2_X0(kFP16x2)
    SP2_X0(kBF16x3)
    SP2_X0(kFP16x2F)
    SP2_X0(kBF16x3F)
#undef SP2_X0
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// One CTA per 128 x 128 tile (I, J): flag 1 if X0 may be non-zero there (a
// diagonal tile inside the matrix, or a non-zero of H), and "unknown content"
// for the other slice set, whose buffers have not been written yet.
__global__ void __launch_bounds__(kEwThreads)
    tile_flags_kernel(const double* __restrict__ H, int64_t n, int T, uint8_t* __restrict__ f0,
                      uint8_t* __restrict__ f1) {
  const int I = blockIdx.x / T, J = blockIdx.x - (blockIdx.x / T) * T;
  const int64_t r0 = (int64_t)I * 128, c0 = (int64_t)J * 128;
  int any = (I == J && r0 < n) ? 1 : 0;
  if (!any) {
    for (int e = threadIdx.x; e < 128 * 128; e += kEwThreads) {
      const int64_t r = r0 + (e >> 7), c = c0 + (e & 127);
      if (r < n && c < n && H[r * n + c] != 0.0) any = 1;
    }
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    f0[blockIdx.x] = (uint8_t)(any ? 1 : 0);
    f1[blockIdx.x] = 1;
  }
}

cudaError_t launch_tile_flags(const double* H, int64_t n, int ld, const DevBuffers& b,
                              cudaStream_t s) {
  const int T = ld / 128;
  tile_flags_kernel<<<T * T, kEwThreads, 0, s>>>(H, n, T, b.tflags[0], b.tflags[1]);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const DevBuffers& b, double* D, int64_t n, int ld, int slice_fmt,
                            cudaStream_t s) {
  (void)ld;
  const int blocks = ew_blocks(n);
  switch (slice_fmt) {
#define SP2_FIN(F)                                                    \
  case F:                                                             \
    finalize_kernel<F><<<blocks, kEwThreads, 0, s>>>(b.st, b, D, n); \
    break;
    SP2_FIN(kFP16x2)
    SP2_FIN(kBF16x3)
    SP2_FIN(kFP16x2F)
    SP2_FIN(kBF16x3F)
#undef SP2_FIN
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace sp2
