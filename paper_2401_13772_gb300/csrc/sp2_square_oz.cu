// FP64-accurate SP2 product step (§IV.A) on the tcgen05 tensor cores, by
// exact products of fixed-point digits (the Ozaki scheme: Ozaki, Ogita,
// Oishi & Rump, "Error-free transformations of matrix multiplication by
// using fast routines of matrix multiplication and its applications",
// Numer. Algorithms 59 (2012) 95-118).
//
// Digits. The iterate X has its spectrum in [0, 1], so |x_ij| <= 1 and every
// row of X has 2-norm <= 1. X (double-float planes hi + lo) is rounded to 52
// fractional bits and cut into five balanced digits
//     x = x0 + x1 + x2 + x3 + x4,  x_s = a_s 2^-(8 + 9 s),  |a_s| <= 256,
// each exactly a BF16 number (8 significant bits); the rest is below 2^-45.
//
// Products. S = X X^T (X symmetric) is approximated by the 15 digit products
// x_s x_t^T with s + t <= 4 (the dropped ones are below ~2^-40), collected by
// weight in four tensor-memory accumulators:
//     G0 = x0 x0^T                       multiples of 2^-16
//     G1 = x0 x1^T + x1 x0^T             multiples of 2^-25
//     G2 = x0 x2^T + x1 x1^T + x2 x0^T   multiples of 2^-34
//     T  = the nine products with s + t = 3 or 4
// With |a0| <= 256 |x| + 1/2 and Cauchy-Schwarz over a row pair,
//     sum_k |a0_ik a0_jk| <= (256 + sqrt(K)/2)^2,
//     sum_k |a0_ik a1_jk| + |a1_ik a0_jk| <= 2 (256 + sqrt(K)/2) 256 sqrt(K),
// so for K <= 8192 every partial sum of G0 and G1 is an integer below 2^24
// units: the tensor core's FP32 accumulation is exact for them over the whole
// K. G2 stays below 2^24 units over 128 consecutive k (x1 x1^T contributes
// up to 256^2 per k); after every such chunk the drain warps move it into
// int32 registers (exact). T (terms below 2^-27) is accumulated in FP32 over
// the same 128-k chunks and the chunk sums are added in shared memory with
// round-to-nearest: the tensor core's FP32 accumulation truncates, and T's
// diagonal entries carry the always-positive x2 x2 term, so one accumulation
// over the whole K shaved about 1e-11 off every diagonal entry (a trace bias
// of -8e-8 at n = 8192); short chains remove that bias. S = G0 + G1 + 2^-34
// g2 + T is then summed in double-float (Knuth's two-sum), X' = S or 2X - S,
// and X' is written back as double-float planes.
//
// Short form (the products of the prefix before the split phase, unless the
// caller asks for all 15): without x0 x4^T + x4 x0^T, 13 products, and digit
// 4 is not loaded. Digit 4 is at most 2^-36 per entry, so by Cauchy-Schwarz
// over a row pair (row norms of x0 <= 1 + ...) the dropped pair is at most
// 2 sqrt(K) 2^-36 per entry (2.6e-9 at K = 8192), of random sign, ~1e-11 in
// practice. The other products with digits 3 and 4 cannot go: the digits are
// fixed-point, so for the typical entry (~0.01) digit 1 carries most of the
// value (rms ~1e-3) and x1 x3^T alone is ~1e-9 per entry, as large as the
// relative 2^-22 of the split products that follow.
//
// Roles (one CTA per 128 x 128 upper-triangle tile, 384 threads):
//   warp 0 lane 0 : TMA producer; per stage (16 k) and operand one 128 x 64
//                   box of the interleaved plane (digits 0..3 of the 16 k in
//                   one 128 B row, 128 B swizzle) and one 128 x 16 box of
//                   digit 4 (32 B rows, 32 B swizzle); four stages
//   warp 1 lane 0 : MMA issuer (kind::f16 with BF16 operands, M = N = 128,
//                   K = 16); per stage it issues the G2 and T products first,
//                   so that at the end of a chunk the drain can read them
//                   while the tensor core works on G0 and G1
//   warps 4..11   : drain (G2 and T chunks, 64 columns each) and epilogue
// The digit planes come from digits_kernel, run right before each product.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "sp2_common.cuh"
#include "sp2_launch.h"
#include "sp2_slices.cuh"
#include "sp2_tc.cuh"

namespace sp2 {

namespace {

using namespace tc;

constexpr int BM = 128;
constexpr int BK = 16;                       // 16-bit elements = 32 B rows
constexpr int BOX_BYTES = BM * BK * 2;       // 4 KB: one digit of a 128 x 16 operand
constexpr int IBOX_BYTES = 4 * BOX_BYTES;    // 16 KB: digits 0..3 interleaved
constexpr int ND = 5;                        // digits
constexpr int STAGES = 4;
constexpr int STAGE_BYTES = 2 * ND * BOX_BYTES;  // 40 KB
constexpr int CHUNK_KB = 128 / BK;           // k-blocks per G2 chunk (128 k)
constexpr int THREADS = 384;
constexpr int EPI_WARP0 = 4;
constexpr int NEPI = 8;
constexpr int TMEM_COLS = 512;               // G0 | G1 | G2 | T
// running T sums of the drain threads after the ring: [warp][column][lane]
constexpr int TSUM_BYTES = NEPI * 64 * 32 * 4;
constexpr int SMEM = STAGES * STAGE_BYTES + TSUM_BYTES + 1024;
constexpr int kMaxOrder = 8192;              // G1 exactness bound
// epilogue use of the (then idle) operand ring: staging of the (r, c) stores,
// then the G2 sums of every epilogue thread
constexpr int STAGING_BYTES = NEPI * 2 * 32 * 17 * 4;
constexpr int G2S_OFFSET = 36864;
static_assert(STAGING_BYTES <= G2S_OFFSET, "staging overlaps the G2 sums");
static_assert(G2S_OFFSET + NEPI * 64 * 32 * 4 <= STAGES * STAGE_BYTES, "ring too small");

struct OzMaps {
  CUtensorMap p0;  // digits 0..3 interleaved (ld x 4 ld), 64 x 128 boxes, 128 B swizzle
  CUtensorMap p4;  // digit 4 (ld x ld), 16 x 128 boxes, 32 B swizzle
};

// Shared-memory matrix descriptor: K-major operand, 32 B swizzle (8-row atoms
// of 256 B), sm_100-family version bit.
__device__ __forceinline__ uint64_t smem_desc_sw32(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(256 >> 4) << 32;   // stride byte offset: 8 rows x 32 B
  d |= (uint64_t)1 << 46;            // descriptor version
  d |= (uint64_t)6 << 61;            // SWIZZLE_32B
  return d;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

// Knuth's two-sum: s + e = a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float v = s - a;
  e = (a - (s - v)) + (b - v);
}

// c += a * b in double-float (few terms; renormalized each step)
__device__ __forceinline__ void dfz_fma(float& ch, float& cl, float ah, float al, float bh,
                                        float bl) {
  const float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  float s, t;
  two_sum(ch, p, s, t);
  const float lo = t + cl + e;
  ch = s + lo;
  cl = lo - (ch - s);
}

// (ah + al) - (bh + bl) in double-float
__device__ __forceinline__ void dfz_sub(float ah, float al, float bh, float bl, float& rh,
                                        float& rl) {
  float s, t;
  two_sum(ah, -bh, s, t);
  const float lo = t + al - bl;
  rh = s + lo;
  rl = lo - (rh - s);
}

// ---------------------------------------------------------------------------
// Digits of X_k (double-float planes) for the next FP64-accurate product.

__global__ void __launch_bounds__(256) digits_kernel(DevBuffers buf, int ld) {
  const State* st = buf.st;
  if (__ldcg(&st->done) || __ldcg(&st->phase) == kPhaseSplit) return;
  const int k = __ldcg(&st->iter);
  const size_t plane = (size_t)ld * ld;
  const float* __restrict__ Xh =
      reinterpret_cast<const float*>((k & 1) ? buf.x64[1] : buf.x64[0]);
  const float* __restrict__ Xl = Xh + plane;
  const size_t n4 = plane / 4;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4;
       q += (size_t)gridDim.x * blockDim.x) {
    const float4 h = __ldcs(reinterpret_cast<const float4*>(Xh) + q);
    const float4 l = __ldcs(reinterpret_cast<const float4*>(Xl) + q);
    uint32_t w[ND][2];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      // x = hi + lo; the remainder is carried as an unevaluated pair (rh, rl)
      // renormalized by two-sum before each digit, so that every step is
      // exact: a = rint(rh) is an integer of at most 9 bits and rh - a is
      // exact (|rh - a| <= 1/2, Sterbenz), scalings are by powers of two.
      float rh = (e == 0 ? h.x : (e == 1 ? h.y : (e == 2 ? h.z : h.w))) * 256.0f;
      float rl = (e == 0 ? l.x : (e == 1 ? l.y : (e == 2 ? l.z : l.w))) * 256.0f;
#pragma unroll
      for (int s = 0; s < ND; ++s) {
        if (s > 0) {
          rh *= 512.0f;
          rl *= 512.0f;
        }
        float t;
        two_sum(rh, rl, rh, t);
        rl = t;
        float a = rintf(rh);
        if (s == 0) a = fminf(fmaxf(a, -256.0f), 256.0f);  // |x| <= 1 in a valid run
        rh -= a;
        // a 2^-(8 + 9 s) is exact in BF16: |a| <= 256
        const uint32_t bits = __bfloat16_as_ushort(
            __float2bfloat16_rn(a * __int_as_float((127 - 8 - 9 * s) << 23)));
        if (e & 1)
          w[s][e >> 1] |= bits << 16;
        else
          w[s][e >> 1] = bits;
      }
    }
    // element (r, k) = 4 q .. 4 q + 3 of the plane: digits 0..3 go to the
    // interleaved plane at row r, column 64 (k / 16) + 16 d + k % 16
    const size_t e0 = 4 * q;
    const size_t r = e0 / (size_t)ld, k = e0 % (size_t)ld;
    uint16_t* rowp = buf.dg[0] + r * (size_t)(4 * ld) + (k >> 4) * 64 + (k & 15);
#pragma unroll
    for (int s = 0; s < ND - 1; ++s)
      *reinterpret_cast<uint2*>(rowp + 16 * s) = make_uint2(w[s][0], w[s][1]);
    reinterpret_cast<uint2*>(buf.dg[4])[q] = make_uint2(w[ND - 1][0], w[ND - 1][1]);
  }
}

// ---------------------------------------------------------------------------
// The product step.

template <int F>
__global__ void __launch_bounds__(THREADS, 1)
    square_oz_kernel(const __grid_constant__ OzMaps maps, DevBuffers buf,
                     unsigned long long cond) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint32_t s_tmem;
  __shared__ int s_err;
  __shared__ int s_consumed;
  __shared__ int s_last;
  __shared__ double s_scratch[2 * THREADS / 32];
  __shared__ __align__(8) uint64_t s_bars[2 * STAGES + 4];

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
  const uint64_t wlim = __ldcg(&st->wait_ns);  // bound on the pipeline waits
  const bool stall = __ldcg(&st->stall_test) != 0 && blockIdx.x == 0;
  const bool want_slices =
      (prec == PROGRESS_MIXED_FP16 || prec == PROGRESS_MIXED_BF16) && phase == kPhaseFP64 &&
      (k_iter + 1 >= st->fp64_prefix);
  const size_t plane = (size_t)ld * ld;
  // prefix products (before the split phase) may take 13 of the 15 digit
  // products: no x0 x4^T + x4 x0^T, digit 4 not loaded (see the header)
  const bool low = phase == kPhaseFP64 && __ldcg(&st->prefix_full) == 0;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int T = ld / BM;
  int I, J;
  band_tile<8>(blockIdx.x, T, I, J);
  const int row_a = I * BM, row_b = J * BM;
  const bool same = (I == J);

  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t bars = smem_u32(&s_bars[0]);
  auto full_bar = [&](int s) { return bars + 8u * s; };
  auto empty_bar = [&](int s) { return bars + 8u * (STAGES + s); };
  const uint32_t g2full = bars + 8u * (2 * STAGES);
  const uint32_t g2empty = bars + 8u * (2 * STAGES + 1);
  const uint32_t accum_bar = bars + 8u * (2 * STAGES + 2);
  const uint32_t stall_bar = bars + 8u * (2 * STAGES + 3);  // nothing arrives on it

  if (threadIdx.x == 0) {
    s_err = 0;
    s_consumed = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    mbar_init(g2full, 1);
    mbar_init(g2empty, NEPI);
    mbar_init(accum_bar, 1);
    mbar_init(stall_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(&s_tmem), TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  volatile int* err = &s_err;

  const int KB = ld / BK;
  const int NC = (KB + CHUNK_KB - 1) / CHUNK_KB;
  const int nd_loaded = low ? ND - 1 : ND;  // digit 4 is not loaded for the short form
  const uint32_t stage_bytes = (uint32_t)((same ? 1 : 2) * nd_loaded * BOX_BYTES);
  int issued = 0;
  if (warp == 0) {
    if (lane == 0) {
      for (int kb = 0; kb < KB; ++kb, ++issued) {
        const int s = kb % STAGES;
        const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
        if (!mbar_wait(empty_bar(s), ph ^ 1u, err, true, wlim)) break;
        mbar_expect_tx(full_bar(s), stage_bytes);
        // stage: A interleaved | B interleaved | A digit 4 | B digit 4
        const uint32_t sa = base + s * STAGE_BYTES;
        tma_load_2d(sa, &maps.p0, kb * 64, row_a, full_bar(s));
        if (!low) tma_load_2d(sa + 2 * IBOX_BYTES, &maps.p4, kb * BK, row_a, full_bar(s));
        if (!same) {
          tma_load_2d(sa + IBOX_BYTES, &maps.p0, kb * 64, row_b, full_bar(s));
          if (!low)
            tma_load_2d(sa + 2 * IBOX_BYTES + BOX_BYTES, &maps.p4, kb * BK, row_b, full_bar(s));
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f16(1, BM, BM);  // BF16 x BF16 -> FP32
      const uint32_t g0 = tmem, g1 = tmem + 128, g2 = tmem + 256, tt = tmem + 384;
      // operand descriptors of stage s: digit d < 4 of the interleaved box is
      // the 32 B slice at 32 d of every 128 B swizzled row (its descriptor
      // starts 32 d bytes in); digit 4 has its own box
      auto descs = [&](int s, uint64_t* a, uint64_t* b) {
        const uint32_t sa = base + s * STAGE_BYTES;
        const uint64_t a0 = smem_desc_sw128(sa), b0 = smem_desc_sw128(sa + IBOX_BYTES);
#pragma unroll
        for (int d = 0; d < ND - 1; ++d) {
          a[d] = a0 + (uint64_t)((d * 32) >> 4);
          b[d] = same ? a[d] : b0 + (uint64_t)((d * 32) >> 4);
        }
        a[ND - 1] = smem_desc_sw32(sa + 2 * IBOX_BYTES);
        b[ND - 1] = same ? a[ND - 1] : smem_desc_sw32(sa + 2 * IBOX_BYTES + BOX_BYTES);
      };
      // G0 and G1: whole-K accumulators (exact); the first block overwrites
      auto issue_rest = [&](int kb, const uint64_t* a, const uint64_t* b) {
        const uint32_t first = kb == 0 ? 0u : 1u;
        mma_f16(g0, a[0], b[0], idesc, first);
        mma_f16(g1, a[0], b[1], idesc, first);
        mma_f16(g1, a[1], b[0], idesc, 1u);
      };
      // G2 and T: accumulated per 128-k chunk (the chunk's first block
      // overwrites); the chunk's last block commits them to the drain
      auto issue_chunked = [&](int kb, const uint64_t* a, const uint64_t* b) {
        const uint32_t c_acc = (kb % CHUNK_KB) == 0 ? 0u : 1u;
        mma_f16(g2, a[0], b[2], idesc, c_acc);
        mma_f16(g2, a[1], b[1], idesc, 1u);
        mma_f16(g2, a[2], b[0], idesc, 1u);
        // T: small terms first (the short form drops the x0 x4 pair)
        if (!low) {
          mma_f16(tt, a[0], b[4], idesc, c_acc);
          mma_f16(tt, a[4], b[0], idesc, 1u);
        }
        mma_f16(tt, a[1], b[3], idesc, low ? c_acc : 1u);
        mma_f16(tt, a[3], b[1], idesc, 1u);
        mma_f16(tt, a[2], b[2], idesc, 1u);
        mma_f16(tt, a[0], b[3], idesc, 1u);
        mma_f16(tt, a[3], b[0], idesc, 1u);
        mma_f16(tt, a[1], b[2], idesc, 1u);
        mma_f16(tt, a[2], b[1], idesc, 1u);
        if ((kb % CHUNK_KB) == CHUNK_KB - 1 || kb == KB - 1) mma_commit(g2full);
      };
      auto wait_full = [&](int kb) {
        return mbar_wait(full_bar(kb % STAGES), (uint32_t)(kb / STAGES) & 1u, err, true, wlim);
      };
      bool ok = true;
      for (int kb = 0; kb < KB && ok;) {
        const int c = kb / CHUNK_KB;
        uint64_t a[ND], b[ND];
        if (c > 0 && (kb % CHUNK_KB) == 0) {
          // chunk boundary: G2 and T may be reused only after the drain has
          // read the previous chunk. Issue G0 and G1 of up to STAGES - 1
          // blocks first (the tensor core works while the drain reads), then
          // wait, then their G2 and T products.
          int L = STAGES - 1;
          if (L > KB - kb) L = KB - kb;
          if (L > CHUNK_KB) L = CHUNK_KB;
          for (int l = 0; l < L; ++l) {
            if (!wait_full(kb + l)) {
              ok = false;
              break;
            }
            tc_fence_after();
            descs((kb + l) % STAGES, a, b);
            issue_rest(kb + l, a, b);
          }
          if (!ok) break;
          if (!mbar_wait(g2empty, (uint32_t)(c - 1) & 1u, err, true, wlim)) {
            ok = false;
            break;
          }
          tc_fence_after();
          for (int l = 0; l < L; ++l) {
            descs((kb + l) % STAGES, a, b);
            issue_chunked(kb + l, a, b);
            mma_commit(empty_bar((kb + l) % STAGES));  // frees the stage once read
            s_consumed = kb + l + 1;
          }
          kb += L;
          continue;
        }
        // test of the bounded waits: after the first k-block's products, wait
        // on a barrier that nothing arrives on; it runs out after wlim
        if (stall && kb == 1 && !mbar_wait(stall_bar, 0u, err, true, wlim)) {
          ok = false;
          break;
        }
        if (!wait_full(kb)) {
          ok = false;
          break;
        }
        tc_fence_after();
        descs(kb % STAGES, a, b);
        // G2 and T first, so that a chunk's last commit is followed by that
        // block's G0 and G1 products as well
        issue_chunked(kb, a, b);
        issue_rest(kb, a, b);
        mma_commit(empty_bar(kb % STAGES));
        s_consumed = kb + 1;
        ++kb;
      }
      mma_commit(accum_bar);  // every MMA issued so far is complete -> epilogue
    }
    __syncwarp();
  }

  // ---- drain + epilogue warps: TMEM lanes of quarter (warp & 3), 64 columns
  const bool epi = warp >= EPI_WARP0;
  const int quarter = warp & 3;
  const int half = epi ? (warp - EPI_WARP0) >> 2 : 0;
  const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
  int g2acc[64];
#pragma unroll
  for (int j = 0; j < 64; ++j) g2acc[j] = 0;
  // this thread's running T sums: [warp][column][lane] after the ring
  float* tsum = reinterpret_cast<float*>(smem_raw + (base - smem_u32(smem_raw)) +
                                         STAGES * STAGE_BYTES) +
                (epi ? (warp - EPI_WARP0) * (64 * 32) : 0) + lane;
  if (epi) {
#pragma unroll
    for (int j = 0; j < 64; ++j) tsum[j * 32] = 0.0f;
    for (int c = 0; c < NC; ++c) {
      if (!mbar_wait(g2full, (uint32_t)c & 1u, err, true, wlim)) break;
      tc_fence_after();
      uint32_t v[64];
#pragma unroll
      for (int q = 0; q < 4; ++q) tmem_ld16(lane_addr + 256 + half * 64 + q * 16, v + q * 16);
      tmem_ld_wait();
#pragma unroll
      for (int j = 0; j < 64; ++j)  // exact: an integer number of 2^-34 below 2^24
        g2acc[j] += __float2int_rn(__uint_as_float(v[j]) * 17179869184.0f);
#pragma unroll
      for (int q = 0; q < 4; ++q) tmem_ld16(lane_addr + 384 + half * 64 + q * 16, v + q * 16);
      tmem_ld_wait();
      // the chunk is in registers: free G2 and T for the next chunk's products
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(g2empty);
#pragma unroll
      for (int j = 0; j < 64; ++j) tsum[j * 32] += __uint_as_float(v[j]);  // round to nearest
    }
  }
  const bool ok = mbar_wait(accum_bar, 0u, err, false);
  tc_fence_after();

  double tr = 0.0, fr = 0.0;
  if (epi && ok && *err == 0) {
    const int row = quarter * 32 + lane;
    const int r = row_a + row;
    const bool odd = (k_iter & 1) != 0;
    const float* __restrict__ Xh = reinterpret_cast<const float*>(odd ? buf.x64[1] : buf.x64[0]);
    const float* __restrict__ Xl = Xh + plane;
    float* __restrict__ Yh = reinterpret_cast<float*>(odd ? buf.x64[0] : buf.x64[1]);
    float* __restrict__ Yl = Yh + plane;
    uint16_t* out[3] = {odd ? buf.sl[0][0] : buf.sl[1][0], odd ? buf.sl[0][1] : buf.sl[1][1],
                        odd ? buf.sl[0][2] : buf.sl[1][2]};
    // staging of the (r, c) stores (the operand ring is free now): per warp
    // 32 rows x 16 columns of hi and of lo, row stride 17 floats
    float* stg = reinterpret_cast<float*>(smem_raw + (base - smem_u32(smem_raw))) +
                 (warp - EPI_WARP0) * (2 * 32 * 17);
    // the G2 sums move to shared memory (behind the staging area), freeing
    // their registers for the epilogue: [warp][column][lane]
    int* g2s = reinterpret_cast<int*>(smem_raw + (base - smem_u32(smem_raw)) + G2S_OFFSET) +
               (warp - EPI_WARP0) * (64 * 32);
#pragma unroll
    for (int j = 0; j < 64; ++j) g2s[j * 32 + lane] = g2acc[j];
    __syncwarp();
    float trh = 0.0f, trl = 0.0f, frh = 0.0f, frl = 0.0f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int col = half * 64 + q * 16;  // column in the tile
      const int c0 = row_b + col;
      // X at the mirror (for 2X - S) does not depend on the products: load
      // it before the tensor-memory reads (X symmetric: coalesced)
      float xmh[16], xml[16];
      if (bit) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const size_t m = (size_t)(c0 + j) * ld + r;
          xmh[j] = Xh[m];
          xml[j] = Xl[m];
        }
      }
      uint32_t u0[16], u1[16];
      tmem_ld16(lane_addr + col, u0);
      tmem_ld16(lane_addr + 128 + col, u1);
      tmem_ld_wait();
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int c = c0 + j;
        // S = G0 + G1 + 2^-34 g2 + T in double-float
        const int gi = g2s[(q * 16 + j) * 32 + lane];
        const float g2h = (float)gi;
        const float g2l = (float)(gi - (int)g2h);  // exact remainder
        float s, e, e2;
        two_sum(__uint_as_float(u0[j]), __uint_as_float(u1[j]), s, e);
        two_sum(s, g2h * 5.820766091346741e-11f, s, e2);  // 2^-34
        e += e2;
        two_sum(s, tsum[(q * 16 + j) * 32], s, e2);
        e += e2 + g2l * 5.820766091346741e-11f;
        float yh = s + e;
        float yl = e - (yh - s);
        if (bit) dfz_sub(2.0f * xmh[j], 2.0f * xml[j], yh, yl, yh, yl);
        stg[lane * 17 + j] = yh;
        stg[32 * 17 + lane * 17 + j] = yl;
        if (r <= c) {
          const float w = (r == c) ? 1.0f : 2.0f;
          if (r == c) dfz_fma(trh, trl, yh, yl, 1.0f, 0.0f);
          dfz_fma(frh, frl, w * yh, w * yl, yh, yl);
          if (r != c) {
            const size_t m = (size_t)c * ld + r;
            Yh[m] = yh;
            Yl[m] = yl;
          }
          if (want_slices) {
            uint16_t a2, b2, c2;
            split_value_f<F>(yh + yl, a2, b2, c2);
            const size_t d = (size_t)r * ld + c;
            out[0][d] = a2;
            out[1][d] = b2;
            if (fmt_bf16(F)) out[2][d] = c2;
            if (r != c) {
              const size_t m = (size_t)c * ld + r;
              out[0][m] = a2;
              out[1][m] = b2;
              if (fmt_bf16(F)) out[2][m] = c2;
            }
          }
        }
      }
      // (r, c) rows back out of the staging area, two rows per store
      __syncwarp();
      const int rb = row_a + quarter * 32;
      const int cc = c0 + (lane & 15);
#pragma unroll 4
      for (int it = 0; it < 16; ++it) {
        const int i = 2 * it + (lane >> 4);
        if (rb + i <= cc) {
          const size_t d = (size_t)(rb + i) * ld + cc;
          Yh[d] = stg[i * 17 + (lane & 15)];
          Yl[d] = stg[32 * 17 + i * 17 + (lane & 15)];
        }
      }
      __syncwarp();
    }
    tr = (double)trh + (double)trl;
    fr = (double)frh + (double)frl;
  }
  tc_fence_before();
  __syncthreads();
  if (*err) {
    // failure path: let TMA copies still in flight land before the CTA exits
    if (threadIdx.x == 0) {
      for (int kb = s_consumed; kb < issued; ++kb)
        mbar_wait(full_bar(kb % STAGES), (uint32_t)(kb / STAGES) & 1u, err, false,
                  kWaitLimitNs / 10);
    }
    __syncthreads();
  }
  if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
  if (*err && threadIdx.x == 0) {
    st->status = PROGRESS_ETIMEOUT;
    st->done = 1;
  }

  block_sum2(tr, fr, s_scratch);
  if (threadIdx.x == 0) {
    buf.partials[2 * blockIdx.x] = tr;
    buf.partials[2 * blockIdx.x + 1] = fr;
  }
  if (!last_cta_arrives(st, gridDim.x, &s_last)) return;
  double ta, tb;
  reduce_partials(buf.partials, gridDim.x, ta, tb, s_scratch);
  if (threadIdx.x == 0) {
    st->ticket = 0u;
    if (st->status == PROGRESS_ETIMEOUT) {
      st->done = 1;
    } else {
      st->t1 = ta;
      st->t2 = tb;
      st->iter = k_iter + 1;
      st->phase_iters[phase] += 1;
      st->x_fp64_valid = 1;
      st->x_slices_valid = want_slices ? 1 : 0;
      decide(st);
    }
    if (st->done && cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0u);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 oz_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

bool encode_oz_maps(const DevBuffers& b, int ld, OzMaps* maps) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = oz_encoder();
  if (!enc) return false;
  memset(maps, 0, sizeof *maps);
  if (!b.dg[0] || !b.dg[4]) return false;
  cuuint32_t estr[2] = {1, 1};
  {  // digits 0..3 interleaved: ld rows of 4 ld elements, boxes of 64 x 128
    cuuint64_t dims[2] = {(cuuint64_t)(4 * ld), (cuuint64_t)ld};
    cuuint64_t strides[1] = {(cuuint64_t)(4 * ld) * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)BM};
    if (enc(&maps->p0, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)b.dg[0], dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  {  // digit 4: ld x ld, boxes of 16 x 128
    cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)ld};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)BM};
    if (enc(&maps->p4, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)b.dg[4], dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

}  // namespace

int oz_max_order() { return kMaxOrder; }

cudaError_t launch_digits(const DevBuffers& b, int ld, cudaStream_t s) {
  if (ld % BM || ld > kMaxOrder) return cudaErrorInvalidValue;
  if (!b.dg[0] || !b.dg[4]) return cudaErrorInvalidValue;
  const size_t n4 = (size_t)ld * ld / 4;
  int blocks = (int)((n4 + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  digits_kernel<<<blocks, 256, 0, s>>>(b, ld);
  return cudaGetLastError();
}

cudaError_t launch_square_oz(const DevBuffers& b, int ld, int slice_fmt,
                             unsigned long long cond_handle, cudaStream_t s) {
  if (ld % BM || ld > kMaxOrder) return cudaErrorInvalidValue;
  const int T = ld / BM;
  const int tiles = T * (T + 1) / 2;
  if (tiles > b.max_partials) return cudaErrorInvalidValue;
  OzMaps maps;
  if (!encode_oz_maps(b, ld, &maps)) return cudaErrorInvalidValue;
  switch (slice_fmt) {
#define SP2_SQOZ(F)                                                                          \
  case F:                                                                                    \
    cudaFuncSetAttribute(square_oz_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                         SMEM);                                                              \
    square_oz_kernel<F><<<tiles, THREADS, SMEM, s>>>(maps, b, cond_handle);                  \
    break;
    SP2_SQOZ(kFP16x2)
    SP2_SQOZ(kBF16x3)
    SP2_SQOZ(kFP16x2F)
    SP2_SQOZ(kBF16x3F)
#undef SP2_SQOZ
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace sp2
