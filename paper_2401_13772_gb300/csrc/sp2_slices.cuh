// Operand slices of the split-precision products.
//
// A split product represents each entry x of the iterate by 16-bit slices so
// that X*X runs on the fp16/bf16 tensor cores with FP32 accumulation:
//   FP16x2: hi = rn_fp16(x), lo = rn_fp16((x - hi) * 2^11)          (22 bits)
//   BF16x3: hi = rn_bf16(x), mid = rn_bf16(x - hi), lo = rn_bf16(x - hi - mid)
// (24 bits). Each slice is an ld x ld row-major matrix; for the symmetric X a
// row panel is the K-major operand of both sides of the product.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace sp2 {

enum SliceFmt : int { kFP16x2 = 0, kBF16x3 = 1 };

constexpr float kLoScale = 2048.0f;          // 2^11, FP16x2 lo scaling
constexpr float kLoUnscale = 1.0f / 2048.0f;

struct Slices {
  uint16_t* s[3];  // hi, lo (FP16x2) or hi, mid, lo (BF16x3); row-major, leading dim ld
};

__device__ __forceinline__ uint16_t h_bits(__half h) { return __half_as_ushort(h); }
__device__ __forceinline__ uint16_t b_bits(__nv_bfloat16 b) { return __bfloat16_as_ushort(b); }

// Split a double into the slices of format F (packed as 16-bit patterns).
template <int F>
__device__ __forceinline__ void split_value(double x, uint16_t& a, uint16_t& b, uint16_t& c) {
  if (F == kFP16x2) {
    __half h = __double2half(x);
    double r = (x - (double)__half2float(h)) * (double)kLoScale;
    a = h_bits(h);
    b = h_bits(__double2half(r));
    c = 0;
  } else {
    __nv_bfloat16 h = __double2bfloat16(x);
    double r1 = x - (double)__bfloat162float(h);
    __nv_bfloat16 m = __double2bfloat16(r1);
    double r2 = r1 - (double)__bfloat162float(m);
    a = b_bits(h);
    b = b_bits(m);
    c = b_bits(__double2bfloat16(r2));
  }
}

template <int F>
__device__ __forceinline__ void split_value_f(float x, uint16_t& a, uint16_t& b, uint16_t& c) {
  if (F == kFP16x2) {
    __half h = __float2half_rn(x);
    a = h_bits(h);
    b = h_bits(__float2half_rn((x - __half2float(h)) * kLoScale));
    c = 0;
  } else {
    __nv_bfloat16 h = __float2bfloat16_rn(x);
    float r1 = x - __bfloat162float(h);
    __nv_bfloat16 m = __float2bfloat16_rn(r1);
    float r2 = r1 - __bfloat162float(m);
    a = b_bits(h);
    b = b_bits(m);
    c = b_bits(__float2bfloat16_rn(r2));
  }
}

// Value represented by the slices.
template <int F>
__device__ __forceinline__ float join_value(uint16_t a, uint16_t b, uint16_t c) {
  if (F == kFP16x2) {
    return __half2float(__ushort_as_half(a)) + __half2float(__ushort_as_half(b)) * kLoUnscale;
  } else {
    return __bfloat162float(__ushort_as_bfloat16(a)) +
           (__bfloat162float(__ushort_as_bfloat16(b)) + __bfloat162float(__ushort_as_bfloat16(c)));
  }
}

template <int F>
__device__ __forceinline__ double join_value_d(uint16_t a, uint16_t b, uint16_t c) {
  if (F == kFP16x2) {
    return (double)__half2float(__ushort_as_half(a)) +
           (double)__half2float(__ushort_as_half(b)) * (double)kLoUnscale;
  } else {
    return (double)__bfloat162float(__ushort_as_bfloat16(a)) +
           (double)__bfloat162float(__ushort_as_bfloat16(b)) +
           (double)__bfloat162float(__ushort_as_bfloat16(c));
  }
}

template <int F>
__device__ __forceinline__ void store_slices(const Slices& S, size_t idx, double x) {
  uint16_t a, b, c;
  split_value<F>(x, a, b, c);
  S.s[0][idx] = a;
  S.s[1][idx] = b;
  if (F == kBF16x3) S.s[2][idx] = c;
}

}  // namespace sp2
