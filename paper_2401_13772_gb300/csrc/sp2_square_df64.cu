// Double-float SP2 product step: FP64-class X' = X*X or 2X - X*X on the FP32
// pipe (§IV.A).
//
// Every number is an unevaluated pair of floats x = hi + lo (|lo| <= ulp(hi)/2,
// about 48 significant bits; Dekker 1971, "A floating-point technique for
// extending the available precision"). The product of two pairs uses the
// exact product error of an FMA (p = a_hi b_hi, e = fma(a_hi, b_hi, -p)) and
// the sum uses Knuth's two-sum; the dot product is compensated (the errors
// of all terms collect in a second float, renormalized once at the end), so a
// multiply-add costs twelve FP32 instructions. On this part the FP32 pipe
// issues several times more of those per second than the FP64 pipe issues
// DFMAs, which makes double-float the faster way to FP64-class products
// (relative error ~2^-45 per product, far below what the SP2 prefix and
// refinement phases need).
//
// Layout: an iterate in double-float form occupies the FP64 ping-pong buffer
// of the workspace as two float planes, hi then lo, each ld x ld row-major.
// Tiles: 128 x 128 upper-triangle output tiles (I <= J), 256 threads, 8 x 8
// outputs per thread (rows ty*4 + {0..3, 64..67}, columns tx*4 + {0..3, 64..67}
// so that shared-memory vector loads are conflict-free). Because X is
// symmetric, the A operand X[I-rows, k] equals X[k, I-cols]: both operand
// tiles are plain row segments of X, copied with 16-byte cp.async and used
// k-major without any transpose.
#include "sp2_common.cuh"
#include "sp2_launch.h"
#include "sp2_slices.cuh"

namespace sp2 {

namespace {

constexpr int BT = 128;       // tile edge
constexpr int BKD = 16;       // k depth per stage
constexpr int THREADS = 256;  // 16 x 16
constexpr int STAGES = 2;

struct DfSmem {
  float Ah[STAGES][BKD][BT];
  float Al[STAGES][BKD][BT];
  float Bh[STAGES][BKD][BT];
  float Bl[STAGES][BKD][BT];
  double scratch[2 * THREADS / 32];
  int last;
};

__device__ __forceinline__ void cp16(void* s, const void* g) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(s);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(g));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// c += a * b in double-float, renormalized every step (used where few terms
// are summed)
__device__ __forceinline__ void df_fma(float& ch, float& cl, float ah, float al, float bh,
                                       float bl) {
  const float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  // two-sum of (ch, p)
  const float s = ch + p;
  const float v = s - ch;
  const float t = (ch - (s - v)) + (p - v);
  const float lo = t + cl + e;
  // renormalize
  ch = s + lo;
  cl = lo - (ch - s);
}

// One term of a compensated dot product (Ogita, Rump & Oishi 2005, "Dot2"):
// the exact product error (FMA) and the exact addition error (two-sum) go to
// a separate float c; s + c is renormalized once, after the last term.
// Twelve FP32 instructions per multiply-add of double-float operands.
__device__ __forceinline__ void dot2_step(float& s, float& c, float ah, float al, float bh,
                                          float bl) {
  const float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  const float s1 = s + p;
  const float v = s1 - s;
  const float q = (s - (s1 - v)) + (p - v);
  c += q + e;
  s = s1;
}

// (ah, al) * k for an exact power-of-two k is exact; 2a - s in double-float:
__device__ __forceinline__ void df_sub(float ah, float al, float bh, float bl, float& rh,
                                       float& rl) {
  const float s = ah - bh;
  const float v = s - ah;
  const float t = (ah - (s - v)) + (-bh - v);
  const float lo = t + al - bl;
  rh = s + lo;
  rl = lo - (rh - s);
}

__device__ __forceinline__ void tri_tile_df(int t, int T, int& I, int& J) {
  const double b = 2.0 * T + 1.0;
  int i = (int)floor((b - sqrt(b * b - 8.0 * (double)t)) * 0.5);
  if (i < 0) i = 0;
  while (i > 0 && i * T - i * (i - 1) / 2 > t) --i;
  while ((i + 1) * T - (i + 1) * i / 2 <= t) ++i;
  I = i;
  J = i + (t - (i * T - i * (i - 1) / 2));
}

__device__ __forceinline__ void load_stage(DfSmem& sm, int s, const float* __restrict__ Xh,
                                           const float* __restrict__ Xl, int ld, int col_a,
                                           int col_b, int k0, bool same) {
  // each operand: BKD rows x 128 floats per plane = 512 chunks of 16 B; 2 per thread
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int c = threadIdx.x + q * THREADS;
    const int kr = c >> 5, col = (c & 31) * 4;
    const size_t ga = (size_t)(k0 + kr) * ld + col_a + col;
    cp16(&sm.Ah[s][kr][col], Xh + ga);
    cp16(&sm.Al[s][kr][col], Xl + ga);
    if (!same) {
      const size_t gb = (size_t)(k0 + kr) * ld + col_b + col;
      cp16(&sm.Bh[s][kr][col], Xh + gb);
      cp16(&sm.Bl[s][kr][col], Xl + gb);
    }
  }
}

template <int F>
__global__ void __launch_bounds__(THREADS, 1) square_df64_kernel(DevBuffers buf,
                                                                 unsigned long long cond) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DfSmem& sm = *reinterpret_cast<DfSmem*>(smem_raw);
  State* st = buf.st;
  const int done = __ldcg(&st->done);
  const int phase = __ldcg(&st->phase);
  if (done) {
    if (cond && blockIdx.x == 0 && threadIdx.x == 0)
      cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0u);
    return;
  }
  if (phase == kPhaseSplit) return;  // the split kernel owns this step
  const int k_iter = __ldcg(&st->iter);
  const int bit = __ldcg(&st->bit);
  const int ld = st->ld;
  const int prec = st->prec;
  const bool want_slices =
      (prec == PROGRESS_MIXED_FP16 || prec == PROGRESS_MIXED_BF16) && phase == kPhaseFP64 &&
      (k_iter + 1 >= st->fp64_prefix);
  const size_t plane = (size_t)ld * ld;
  const float* __restrict__ Xh = reinterpret_cast<const float*>(buf.x64[k_iter & 1]);
  const float* __restrict__ Xl = Xh + plane;
  float* __restrict__ Yh = reinterpret_cast<float*>(buf.x64[(k_iter + 1) & 1]);
  float* __restrict__ Yl = Yh + plane;
  Slices S;
  for (int i = 0; i < 3; ++i) S.s[i] = buf.sl[(k_iter + 1) & 1][i];

  const int T = ld / BT;
  int I, J;
  tri_tile_df(blockIdx.x, T, I, J);
  const int row_a = I * BT, row_b = J * BT;
  const bool same = (I == J);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;

  float ch[8][8], cl[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) ch[i][j] = cl[i][j] = 0.0f;

  const int KT = ld / BKD;
  load_stage(sm, 0, Xh, Xl, ld, row_a, row_b, 0, same);
  cp_commit();
  for (int kt = 0; kt < KT; ++kt) {
    const int s = kt & 1;
    if (kt + 1 < KT) load_stage(sm, s ^ 1, Xh, Xl, ld, row_a, row_b, (kt + 1) * BKD, same);
    cp_commit();
    cp_wait<1>();
    __syncthreads();
    const float(*Ah)[BT] = sm.Ah[s];
    const float(*Al)[BT] = sm.Al[s];
    const float(*Bh)[BT] = same ? sm.Ah[s] : sm.Bh[s];
    const float(*Bl)[BT] = same ? sm.Al[s] : sm.Bl[s];
#pragma unroll 1
    for (int k = 0; k < BKD; ++k) {
      float ah[8], al[8], bh[8], bl[8];
      *reinterpret_cast<float4*>(&ah[0]) = *reinterpret_cast<const float4*>(&Ah[k][ty * 4]);
      *reinterpret_cast<float4*>(&ah[4]) = *reinterpret_cast<const float4*>(&Ah[k][ty * 4 + 64]);
      *reinterpret_cast<float4*>(&al[0]) = *reinterpret_cast<const float4*>(&Al[k][ty * 4]);
      *reinterpret_cast<float4*>(&al[4]) = *reinterpret_cast<const float4*>(&Al[k][ty * 4 + 64]);
      *reinterpret_cast<float4*>(&bh[0]) = *reinterpret_cast<const float4*>(&Bh[k][tx * 4]);
      *reinterpret_cast<float4*>(&bh[4]) = *reinterpret_cast<const float4*>(&Bh[k][tx * 4 + 64]);
      *reinterpret_cast<float4*>(&bl[0]) = *reinterpret_cast<const float4*>(&Bl[k][tx * 4]);
      *reinterpret_cast<float4*>(&bl[4]) = *reinterpret_cast<const float4*>(&Bl[k][tx * 4 + 64]);
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) dot2_step(ch[i][j], cl[i][j], ah[i], al[i], bh[j], bl[j]);
    }
    __syncthreads();
  }
  cp_wait<0>();

  // epilogue: branch, mirror store, slices, partial traces (double-float sums
  // per thread, folded into FP64 once)
  float trh = 0.0f, trl = 0.0f, frh = 0.0f, frl = 0.0f;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = row_a + ty * 4 + (i & 3) + (i >> 2) * 64;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = row_b + tx * 4 + (j & 3) + (j >> 2) * 64;
      if (r > c) continue;  // covered by the mirror of the tile above the diagonal
      // renormalize the compensated sum into a double-float pair
      float xh = ch[i][j] + cl[i][j];
      float xl = cl[i][j] - (xh - ch[i][j]);
      if (bit) {
        const size_t g = (size_t)r * ld + c;
        df_sub(2.0f * Xh[g], 2.0f * Xl[g], xh, xl, xh, xl);
      }
      const size_t d = (size_t)r * ld + c;
      Yh[d] = xh;
      Yl[d] = xl;
      if (r != c) {
        const size_t m = (size_t)c * ld + r;
        Yh[m] = xh;
        Yl[m] = xl;
      }
      if (want_slices) {
        const float x = xh + xl;
        uint16_t a, b2, c2;
        split_value_f<F>(x, a, b2, c2);
        S.s[0][d] = a;
        S.s[1][d] = b2;
        if (fmt_bf16(F)) S.s[2][d] = c2;
        if (r != c) {
          const size_t m = (size_t)c * ld + r;
          S.s[0][m] = a;
          S.s[1][m] = b2;
          if (fmt_bf16(F)) S.s[2][m] = c2;
        }
      }
      const float w = (r == c) ? 1.0f : 2.0f;
      if (r == c) df_fma(trh, trl, xh, xl, 1.0f, 0.0f);
      df_fma(frh, frl, w * xh, w * xl, xh, xl);
    }
  }
  double tr = (double)trh + (double)trl, fr = (double)frh + (double)frl;
  block_sum2(tr, fr, sm.scratch);
  if (threadIdx.x == 0) {
    buf.partials[2 * blockIdx.x] = tr;
    buf.partials[2 * blockIdx.x + 1] = fr;
  }
  if (!last_cta_arrives(st, gridDim.x, &sm.last)) return;
  double a, b;
  reduce_partials(buf.partials, gridDim.x, a, b, sm.scratch);
  if (threadIdx.x == 0) {
    st->t1 = a;
    st->t2 = b;
    st->iter = k_iter + 1;
    st->phase_iters[phase] += 1;
    st->x_fp64_valid = 1;
    st->x_slices_valid = want_slices ? 1 : 0;
    st->ticket = 0u;
    decide(st);
    if (st->done && cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0u);
  }
}

}  // namespace

int df64_tile_count(int ld) {
  const int T = ld / BT;
  return T * (T + 1) / 2;
}

cudaError_t launch_square_df64(const DevBuffers& b, int ld, int slice_fmt,
                               unsigned long long cond_handle, cudaStream_t s) {
  const int tiles = df64_tile_count(ld);
  if (tiles > b.max_partials || ld % BT) return cudaErrorInvalidValue;
  const int smem = (int)sizeof(DfSmem);
  switch (slice_fmt) {
#define SP2_SQDF(F)                                                                        \
  case F:                                                                                  \
    cudaFuncSetAttribute(square_df64_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                         smem);                                                            \
    square_df64_kernel<F><<<tiles, THREADS, smem, s>>>(b, cond_handle);                    \
    break;
    SP2_SQDF(kFP16x2)
    SP2_SQDF(kBF16x3)
    SP2_SQDF(kFP16x2F)
    SP2_SQDF(kBF16x3F)
#undef SP2_SQDF
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace sp2
