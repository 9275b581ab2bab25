// Operand slices of the split-precision products.
//
// Floating-point splits (the defaults, kFP16x2 / kBF16x3): x = hi + lo / 2048
// with hi = rn_fp16(x), or x = hi + mid + lo with bf16 slices, every entry
// keeping 22 / 24 significant bits relative to its own magnitude.
//
// Fixed-point splits (kFP16x2F / kBF16x3F, an option) for |x| <= 1, one global
// scale (no per-row exponents):
//
//   FP16x2F: hi = rint(x 2^11)              integer, |hi| <= 2^11 (exact in fp16)
//            lo = rn_fp16((x 2^11 - hi) 2^11)   |lo| <= 2^10, 11 significant bits
//            x ~ 2^-11 hi + 2^-22 lo        (absolute error <= 2^-23)
//   BF16x3F: hi  = rint(x 2^8)              integer, |hi| <= 2^8 (exact in bf16)
//            mid = rint((x 2^8 - hi) 2^8)   integer, |mid| <= 2^7 (exact in bf16)
//            lo  = rn_bf16(((x 2^8 - hi) 2^8 - mid) 2^8)
//            x ~ 2^-8 hi + 2^-16 mid + 2^-24 lo  (absolute error <= 2^-26)
//
// The idea of fixed point: in S_ij = sum_k x_ik x_jk the leading group
// sum_k hi_ik hi_jk is a sum of integer products bounded (Cauchy-Schwarz and
// row norms <= 1) by 2^22 (FP16x2F) or 2^16 (BF16x3F), which an exact FP32
// accumulator would sum without error. Measured on GB300 the fixed-point FP16
// products were nevertheless LESS accurate than the floating ones (a diagonal
// bias of -1.1e-5 per square of a matrix whose diagonal entries are near +-1,
// against -5.7e-7 floating with 64-k chunks), so floating splits are the
// default and the leading group is summed in short chunks instead.
//
// Each slice is an ld x ld row-major matrix; for a symmetric matrix a row panel
// is the K-major operand of both sides of the product.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace sp2 {

// kFP16x2 / kBF16x3: floating-point splits; kFP16x2F / kBF16x3F: the
// fixed-point variants described above.
enum SliceFmt : int { kFP16x2 = 0, kBF16x3 = 1, kFP16x2F = 2, kBF16x3F = 3 };

__host__ __device__ constexpr bool fmt_bf16(int f) { return f == kBF16x3 || f == kBF16x3F; }
__host__ __device__ constexpr int fmt_slices(int f) { return fmt_bf16(f) ? 3 : 2; }

struct Slices {
  uint16_t* s[3];  // hi, lo (FP16x2) or hi, mid, lo (BF16x3); row-major, leading dim ld
};

__device__ __forceinline__ uint16_t h_bits(__half h) { return __half_as_ushort(h); }
__device__ __forceinline__ uint16_t b_bits(__nv_bfloat16 b) { return __bfloat16_as_ushort(b); }
__device__ __forceinline__ float h_val(uint16_t u) { return __half2float(__ushort_as_half(u)); }
__device__ __forceinline__ float b_val(uint16_t u) {
  return __bfloat162float(__ushort_as_bfloat16(u));
}

// Split x (|x| <= 1) into the slices of format F (16-bit patterns).
template <int F>
__device__ __forceinline__ void split_value_f(float x, uint16_t& a, uint16_t& b, uint16_t& c) {
  if (F == kFP16x2) {
    const __half h = __float2half_rn(x);
    a = h_bits(h);
    b = h_bits(__float2half_rn((x - __half2float(h)) * 2048.0f));
    c = 0;
  } else if (F == kBF16x3) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(h);
    const __nv_bfloat16 m = __float2bfloat16_rn(r1);
    a = b_bits(h);
    b = b_bits(m);
    c = b_bits(__float2bfloat16_rn(r1 - __bfloat162float(m)));
  } else if (F == kFP16x2F) {
    const float y = x * 2048.0f;  // exact scaling
    const float h = rintf(y);
    a = h_bits(__float2half_rn(h));                  // integer, exact
    b = h_bits(__float2half_rn((y - h) * 2048.0f));  // y - h is exact
    c = 0;
  } else {
    const float y = x * 256.0f;
    const float h = rintf(y);
    const float r1 = (y - h) * 256.0f;
    const float m = rintf(r1);
    a = b_bits(__float2bfloat16_rn(h));
    b = b_bits(__float2bfloat16_rn(m));
    c = b_bits(__float2bfloat16_rn((r1 - m) * 256.0f));
  }
}

// The same split from an FP64 value. FP64 arithmetic is scarce on this part,
// so each slice is rounded through FP32 (a double rounding of the leading slice
// is harmless: the next slice takes the exact FP64 remainder) and only the
// remainders are formed in FP64 (exact subtractions).
template <int F>
__device__ __forceinline__ void split_value(double x, uint16_t& a, uint16_t& b, uint16_t& c) {
  if (F == kFP16x2) {
    const __half h = __float2half_rn((float)x);
    a = h_bits(h);
    b = h_bits(__float2half_rn((float)((x - (double)__half2float(h)) * 2048.0)));
    c = 0;
  } else if (F == kBF16x3) {
    const __nv_bfloat16 h = __float2bfloat16_rn((float)x);
    const double r1 = x - (double)__bfloat162float(h);
    const __nv_bfloat16 m = __float2bfloat16_rn((float)r1);
    a = b_bits(h);
    b = b_bits(m);
    c = b_bits(__float2bfloat16_rn((float)(r1 - (double)__bfloat162float(m))));
  } else if (F == kFP16x2F) {
    const double y = x * 2048.0;
    const double h = rint(y);
    a = h_bits(__float2half_rn((float)h));                      // integer, exact
    b = h_bits(__float2half_rn((float)((y - h) * 2048.0)));
    c = 0;
  } else {
    const double y = x * 256.0;
    const double h = rint(y);
    const double r1 = (y - h) * 256.0;
    const double m = rint(r1);
    a = b_bits(__float2bfloat16_rn((float)h));
    b = b_bits(__float2bfloat16_rn((float)m));
    c = b_bits(__float2bfloat16_rn((float)((r1 - m) * 256.0)));
  }
}

// Value represented by the slices (FP32).
template <int F>
__device__ __forceinline__ float join_value(uint16_t a, uint16_t b, uint16_t c) {
  if (F == kFP16x2) {
    return h_val(a) + h_val(b) * (1.0f / 2048.0f);
  } else if (F == kBF16x3) {
    return b_val(a) + (b_val(b) + b_val(c));
  } else if (F == kFP16x2F) {
    return h_val(a) * (1.0f / 2048.0f) + h_val(b) * (1.0f / 4194304.0f);
  } else {
    return b_val(a) * (1.0f / 256.0f) +
           (b_val(b) * (1.0f / 65536.0f) + b_val(c) * (1.0f / 16777216.0f));
  }
}

template <int F>
__device__ __forceinline__ double join_value_d(uint16_t a, uint16_t b, uint16_t c) {
  if (F == kFP16x2) {
    return (double)h_val(a) + (double)h_val(b) * (1.0 / 2048.0);
  } else if (F == kBF16x3) {
    return (double)b_val(a) + (double)b_val(b) + (double)b_val(c);
  } else if (F == kFP16x2F) {
    return (double)h_val(a) * (1.0 / 2048.0) + (double)h_val(b) * (1.0 / 4194304.0);
  } else {
    return (double)b_val(a) * (1.0 / 256.0) + (double)b_val(b) * (1.0 / 65536.0) +
           (double)b_val(c) * (1.0 / 16777216.0);
  }
}

// Weights of the accumulator groups: S = w0 acc0 + w1 acc1 + w2 acc2.
//   *x2: acc0 = sum hi hi, acc1 = sum (hi lo + lo hi)
//   *x3: acc0 = sum hi hi, acc1 = sum (hi mid + mid hi),
//        acc2 = sum (hi lo + lo hi + mid mid)
template <int F>
struct SliceWeights;
template <>
struct SliceWeights<kFP16x2> {
  static constexpr float w0 = 1.0f;
  static constexpr float w1 = 1.0f / 2048.0f;
  static constexpr float w2 = 0.0f;
  static constexpr int groups = 2;
};
template <>
struct SliceWeights<kBF16x3> {
  static constexpr float w0 = 1.0f, w1 = 1.0f, w2 = 1.0f;
  static constexpr int groups = 3;
};
template <>
struct SliceWeights<kFP16x2F> {
  static constexpr float w0 = 1.0f / 4194304.0f;        // 2^-22
  static constexpr float w1 = 1.0f / 8589934592.0f;     // 2^-33
  static constexpr float w2 = 0.0f;
  static constexpr int groups = 2;
};
template <>
struct SliceWeights<kBF16x3F> {
  static constexpr float w0 = 1.0f / 65536.0f;          // 2^-16
  static constexpr float w1 = 1.0f / 16777216.0f;       // 2^-24
  static constexpr float w2 = 1.0f / 4294967296.0f;     // 2^-32
  static constexpr int groups = 3;
};

template <int F>
__device__ __forceinline__ void store_slices(const Slices& S, size_t idx, double x) {
  uint16_t a, b, c;
  split_value<F>(x, a, b, c);
  S.s[0][idx] = a;
  S.s[1][idx] = b;
  if (fmt_bf16(F)) S.s[2][idx] = c;
}

}  // namespace sp2
