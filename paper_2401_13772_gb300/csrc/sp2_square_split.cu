// Split-precision SP2 product step on the sm_103a tcgen05 tensor cores.
//
// One CTA computes one 128 x 128 upper-triangle tile (I <= J) of S = X*X for
// the symmetric iterate X. X is held as 16-bit fixed-point operand slices
// (FP16x2: hi, lo; BF16x3: hi, mid, lo -- see sp2_slices.cuh), each an ld x ld
// row-major matrix, so both operands of tile (I, J) are K-major row panels of
// the same slices.
//
//   warp 0, one lane : TMA producer -- 128 x 64 slice boxes (128 B rows,
//                      128 B swizzle) of the I and J row panels into a
//                      STAGES-deep shared-memory ring (mbarrier complete_tx)
//   warp 1, one lane : MMA issuer -- tcgen05.mma kind::f16, M = N = 128,
//                      K = 16, FP32 accumulators in tensor memory, one per
//                      weight group of the slices: acc0 += hi*hi^T,
//                      acc1 += hi*lo^T + lo*hi^T (x2) or hi*mid^T + mid*hi^T
//                      (x3), acc2 += hi*lo^T + lo*hi^T + mid*mid^T (x3).
//                      The leading group acc0 rotates through three (x2) or
//                      two (x3) chunk buffers of CHUNK k-blocks (K = 256), so
//                      the MMA runs ahead of the drain: the tensor core's
//                      FP32 accumulation truncates, and over a whole K = n
//                      chain of same-sign products (the diagonal of X*X) that
//                      truncation becomes a measurable bias; short chains
//                      summed with round-to-nearest adds remove it.
//   warps 4..11      : drain -- two warps per 32-lane quarter of tensor
//                      memory, each thread owns one lane (a tile row) and 64
//                      of the tile's columns; it adds every finished acc0
//                      chunk into 64 FP32 registers and frees the buffer
//                      (mbarrier), then
//                      runs the epilogue: S = w0 sum0 + w1 acc1 (+ w2 acc2)
//                      in FP32 (no FP64 arithmetic: it is slow on this part),
//                      the SP2 branch of §IV.A chosen on the device (X' = S or
//                      2X - S), the new slices of X' at (r, c) (staged
//                      through the then idle operand ring so that the stores
//                      run along rows) and at the mirror (c, r), FP64 X' when
//                      the precision schedule may
//                      leave the split phase next, and the partial traces
//                      Tr X', ||X'||_F^2 (FP32 over 32 columns, folded into
//                      FP64 per chunk).
//
// Thresholded SP2 (Listing 1's cutoff tau) has its own persistent kernel below,
// square_split_sparse_kernel: the epilogue drops |x| < tau from the product and
// from 2X - X^2 and records, per 128 x 128 tile, whether the new iterate holds a
// non-zero there (tflags, one byte per tile and slice set); a tile (I, J) then
// streams only the k-blocks whose tiles (I, k) and (J, k) of X may be non-zero,
// and a result tile that stays zero where zeros already are is skipped.
//
// Every mbarrier wait is bounded; a wait that runs out records
// PROGRESS_ETIMEOUT in the solve state, stops the loop and the CTA still frees
// its tensor memory before it exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdio.h>

#include "sp2_common.cuh"
#include "sp2_launch.h"
#include "sp2_slices.cuh"
#include "sp2_tc.cuh"

namespace sp2 {

namespace {

constexpr int BM = 128;
constexpr int BN = 128;
constexpr int BK = 64;                         // 16-bit elements = 128 B rows
constexpr int TILE_BYTES = BM * BK * 2;        // one 128 x 64 slice box (16 KB)
constexpr int THREADS = 384;       // warp 0 TMA, warp 1 MMA, warps 4..11 drain + epilogue
constexpr int DRAIN_WARPS = 8;     // two per 32-lane quarter of tensor memory
constexpr int DRAIN_WARP0 = 4;
constexpr int DCOLS = BN / 2;      // columns per drain thread
constexpr int CHUNK = 4;           // k-blocks per leading-group accumulation chunk
constexpr int TMEM_COLS = 512;     // acc0 chunk buffers | acc1 | (acc2), 128 columns each


template <int F>
struct Cfg {
  static constexpr int NS = fmt_slices(F);                          // slices
  static constexpr int STAGE_BYTES = 2 * NS * TILE_BYTES;            // A and B boxes
  static constexpr int STAGES = fmt_bf16(F) ? 2 : 3;
  // leading-group chunk buffers in tensor memory: three for FP16x2 (acc1 in
  // the fourth 128 columns), two for BF16x3 (acc1, acc2 in the others)
  static constexpr int NBUF = fmt_bf16(F) ? 2 : 3;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 256;    // + align + barriers
};

struct TensorMaps {
  CUtensorMap m[2][3];  // [ping-pong set][slice]
};

using namespace tc;

__device__ __forceinline__ void mbar_arrive_cta(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

template <int F>
__global__ void __launch_bounds__(THREADS, 1)
    square_split_kernel(const __grid_constant__ TensorMaps maps, DevBuffers buf,
                        unsigned long long cond) {
  using C = Cfg<F>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint32_t s_tmem;
  __shared__ int s_err;
  __shared__ int s_consumed;
  __shared__ int s_last;
  __shared__ double s_scratch[2 * THREADS / 32];

  State* st = buf.st;
  const int done = __ldcg(&st->done);
  const int phase = __ldcg(&st->phase);
  if (done) {
    if (cond && blockIdx.x == 0 && threadIdx.x == 0)
      cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0u);
    return;
  }
  if (phase != kPhaseSplit) return;  // the FP64 kernel owns this step
  const int k_iter = __ldcg(&st->iter);
  const int bit = __ldcg(&st->bit);
  const int ld = st->ld;
  const uint64_t wlim = __ldcg(&st->wait_ns);  // bound on the pipeline waits
  const bool stall = __ldcg(&st->stall_test) != 0 && blockIdx.x == 0;
  // FP64 X' is needed if the schedule may switch to FP64 refinement after
  // this product (MIXED: the split phase has stalled once already).
  const bool want_fp64 = (st->prec == PROGRESS_MIXED_FP16 || st->prec == PROGRESS_MIXED_BF16) &&
                         __ldcg(&st->split_stall) >= 1;
  const int src = k_iter & 1, dst = (k_iter + 1) & 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int T = ld / BM;
  int I, J;
  band_tile<8>(blockIdx.x, T, I, J);  // tiles running together share few operand panels
  const int row_a = I * BM, row_b = J * BN;

  // shared memory: stage ring (1024-aligned), then barriers
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t bars = base + C::STAGES * C::STAGE_BYTES;
  auto full_bar = [&](int s) { return bars + 8u * s; };
  auto empty_bar = [&](int s) { return bars + 8u * (C::STAGES + s); };
  const uint32_t accum_bar = bars + 8u * (2 * C::STAGES);

  const uint32_t chunk_full = bars + 8u * (2 * C::STAGES + 1);              // [NBUF]
  const uint32_t chunk_empty = bars + 8u * (2 * C::STAGES + 1 + C::NBUF);   // [NBUF]
  const uint32_t stall_bar = bars + 8u * (2 * C::STAGES + 1 + 2 * C::NBUF); // never arrived

  if (threadIdx.x == 0) {
    s_err = 0;
    s_consumed = 0;
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    mbar_init(accum_bar, 1);
    for (int b = 0; b < C::NBUF; ++b) {
      mbar_init(chunk_full + 8u * b, 1);
      mbar_init(chunk_empty + 8u * b, DRAIN_WARPS);
    }
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
  const int NC = (KB + CHUNK - 1) / CHUNK;  // leading-group chunks
  int issued = 0;  // k-blocks whose loads were issued (producer thread)
  if (warp == 0) {
    if (lane == 0) {
      // TMA producer
      for (int kb = 0; kb < KB; ++kb, ++issued) {
        const int s = kb % C::STAGES;
        const uint32_t ph = (uint32_t)(kb / C::STAGES) & 1u;
        if (!mbar_wait(empty_bar(s), ph ^ 1u, err, true, wlim)) break;
        mbar_expect_tx(full_bar(s), C::STAGE_BYTES);
        const uint32_t sa = base + s * C::STAGE_BYTES;
#pragma unroll
        for (int j = 0; j < C::NS; ++j) {
          tma_load_2d(sa + j * TILE_BYTES, &maps.m[src][j], kb * BK, row_a, full_bar(s));
          tma_load_2d(sa + (C::NS + j) * TILE_BYTES, &maps.m[src][j], kb * BK, row_b,
                      full_bar(s));
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer. The leading group goes to one of two chunk accumulators
      // (CHUNK k-blocks each) that the drain warps empty in turn; the
      // correction groups accumulate over the whole K.
      constexpr uint32_t idesc = idesc_f16(fmt_bf16(F) ? 1 : 0, BM, BN);
      const uint32_t acc1 = tmem + 128u * C::NBUF, acc2 = acc1 + 128u;
      bool ok = true;
      for (int kb = 0; kb < KB && ok; ++kb) {
        const int c = kb / CHUNK, cb = c % C::NBUF;
        const bool chunk_first = (kb % CHUNK) == 0;
        const bool chunk_last = (kb % CHUNK) == CHUNK - 1 || kb == KB - 1;
        const uint32_t acc0 = tmem + 128u * cb;
        if (chunk_first) {
          if (!mbar_wait(chunk_empty + 8u * cb, ((uint32_t)(c / C::NBUF) & 1u) ^ 1u, err, true,
                         wlim)) {
            ok = false;
            break;
          }
          tc_fence_after();
        }
        const int s = kb % C::STAGES;
        const uint32_t ph = (uint32_t)(kb / C::STAGES) & 1u;
        // test of the bounded waits: after the first k-block's products, wait
        // on a barrier that nothing arrives on; it runs out after wlim
        if (stall && kb == 1 && !mbar_wait(stall_bar, 0u, err, true, wlim)) {
          ok = false;
          break;
        }
        if (!mbar_wait(full_bar(s), ph, err, true, wlim)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t sa = base + s * C::STAGE_BYTES;
        uint64_t a[3], b[3];
#pragma unroll
        for (int j = 0; j < C::NS; ++j) {
          a[j] = smem_desc_sw128(sa + j * TILE_BYTES);
          b[j] = smem_desc_sw128(sa + (C::NS + j) * TILE_BYTES);
        }
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint64_t adv = (uint64_t)(kk * 32) >> 4;  // 32 B per K = 16 step
          const uint32_t first = (kb == 0 && kk == 0) ? 0u : 1u;
          const uint32_t chunk_acc = (chunk_first && kk == 0) ? 0u : 1u;
          mma_f16(acc0, a[0] + adv, b[0] + adv, idesc, chunk_acc);
          mma_f16(acc1, a[0] + adv, b[1] + adv, idesc, first);
          mma_f16(acc1, a[1] + adv, b[0] + adv, idesc, 1u);
          if (fmt_bf16(F)) {
            mma_f16(acc2, a[0] + adv, b[2] + adv, idesc, first);
            mma_f16(acc2, a[2] + adv, b[0] + adv, idesc, 1u);
            mma_f16(acc2, a[1] + adv, b[1] + adv, idesc, 1u);
          }
        }
        mma_commit(empty_bar(s));  // frees the stage once these MMAs have read it
        if (chunk_last) mma_commit(chunk_full + 8u * cb);
        s_consumed = kb + 1;
      }
      mma_commit(accum_bar);  // all MMAs issued so far are complete -> epilogue
    }
    __syncwarp();
  }

  // ---- drain warps: thread owns TMEM lane = tile row and DCOLS columns, sums
  // the leading-group chunks with round-to-nearest FP32 adds, then runs the
  // epilogue.
  const bool drain = warp >= DRAIN_WARP0;
  const int quarter = warp & 3;
  const int half = drain ? (warp - DRAIN_WARP0) >> 2 : 0;
  const int row = quarter * 32 + lane;
  const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
  float sum0[DCOLS];
#pragma unroll
  for (int j = 0; j < DCOLS; ++j) sum0[j] = 0.0f;
  if (drain) {
    for (int c = 0; c < NC; ++c) {
      const int cb = c % C::NBUF;
      if (!mbar_wait(chunk_full + 8u * cb, (uint32_t)(c / C::NBUF) & 1u, err, true, wlim)) break;
      tc_fence_after();
      float v[DCOLS];
#pragma unroll
      for (int q = 0; q < DCOLS / 32; ++q) tmem_ld32(lane_addr + 128u * cb + half * DCOLS + q * 32, v + q * 32);
      tmem_ld_wait();
      // the values are in registers: free the buffer before adding them
      tc_fence_before();
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(chunk_empty + 8u * cb)
                     : "memory");
#pragma unroll
      for (int j = 0; j < DCOLS; ++j) sum0[j] += v[j];
    }
  }
  // (the MMA thread always commits accum_bar, so this wait does not abort
  // early: no MMA may still be writing tensor memory past it)
  const bool ok = mbar_wait(accum_bar, 0u, err, false);
  tc_fence_after();
  double tr = 0.0, fr = 0.0;
  if (drain && ok && *err == 0) {
    using W = SliceWeights<F>;
    const int r = row_a + row;
    // (selects, not a runtime index into the parameter arrays)
    const bool odd = src != 0;
    const uint16_t* xs0 = odd ? buf.sl[1][0] : buf.sl[0][0];
    const uint16_t* xs1 = odd ? buf.sl[1][1] : buf.sl[0][1];
    const uint16_t* xs2 = odd ? buf.sl[1][2] : buf.sl[0][2];
    uint16_t* const out0 = odd ? buf.sl[0][0] : buf.sl[1][0];
    uint16_t* const out1 = odd ? buf.sl[0][1] : buf.sl[1][1];
    uint16_t* const out2 = odd ? buf.sl[0][2] : buf.sl[1][2];
    double* out64 = odd ? buf.x64[0] : buf.x64[1];
    // FP64-accurate phases read the next iterate from the FP64 buffer: as
    // doubles, or as double-float planes (hi = x, lo = 0)
    const bool df = st->df64 != 0;
    float* out_hi = reinterpret_cast<float*>(out64);
    float* out_lo = out_hi + (size_t)ld * ld;
    // staging of the (r, c) slice stores in the idle operand ring: per warp
    // 32 rows x 32 columns of packed (slice0 | slice1 << 16) words (row
    // stride 33) and, for BF16x3, of slice-2 half words (row stride 34)
    uint32_t* stA = reinterpret_cast<uint32_t*>(smem_raw + (base - smem_u32(smem_raw))) +
                    (warp - DRAIN_WARP0) * (32 * 33);
    uint16_t* stB = reinterpret_cast<uint16_t*>(smem_raw + (base - smem_u32(smem_raw)) +
                                                DRAIN_WARPS * 32 * 33 * 4) +
                    (warp - DRAIN_WARP0) * (32 * 34);
    const int rb = row_a + quarter * 32;
#pragma unroll
    for (int ch = 0; ch < DCOLS / 32; ++ch) {
      const int col = half * DCOLS + ch * 32;  // column in the tile
      const int c0 = row_b + col;
      float trf = 0.0f, frf = 0.0f;  // chunk partials (FP32), folded into FP64 below
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int cs = c0 + hh * 16;
        // the mirror values of X for 2X - X^2 do not depend on the products:
        // load them before waiting on tensor memory (packed slice0 | slice1)
        uint32_t m01[16], m2[16];
        if (bit) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const size_t m = (size_t)(cs + j) * ld + r;  // X is symmetric: coalesced
            m01[j] = (uint32_t)xs0[m] | ((uint32_t)xs1[m] << 16);
            m2[j] = fmt_bf16(F) ? (uint32_t)xs2[m] : 0u;
          }
        }
        uint32_t u1[16], u2[16];
        tmem_ld16(lane_addr + 128u * C::NBUF + col + hh * 16, u1);
        if (fmt_bf16(F)) tmem_ld16(lane_addr + 128u * (C::NBUF + 1) + col + hh * 16, u2);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int jj = hh * 16 + j;  // column within the 32-column chunk
          const int c = cs + j;
          float x = sum0[ch * 32 + jj] * W::w0 + __uint_as_float(u1[j]) * W::w1;
          if (fmt_bf16(F)) x += __uint_as_float(u2[j]) * W::w2;
          if (bit)
            x = 2.0f * join_value<F>((uint16_t)(m01[j] & 0xffffu), (uint16_t)(m01[j] >> 16),
                                     (uint16_t)m2[j]) -
                x;
          uint16_t a, b2, c2;
          split_value_f<F>(x, a, b2, c2);
          stA[lane * 33 + jj] = (uint32_t)a | ((uint32_t)b2 << 16);
          if (fmt_bf16(F)) stB[lane * 34 + jj] = c2;
          if (r <= c) {
            if (r == c) {
              trf += x;
              frf += x * x;
            } else {
              frf += 2.0f * x * x;
              // mirror (c, r): consecutive threads write consecutive r
              const size_t m = (size_t)c * ld + r;
              out0[m] = a;
              out1[m] = b2;
              if (fmt_bf16(F)) out2[m] = c2;
              if (want_fp64) {
                if (df) {
                  out_hi[m] = x;
                  out_lo[m] = 0.0f;
                } else {
                  out64[m] = (double)x;
                }
              }
            }
            if (want_fp64) {  // (r, c), a few products per solve: direct stores
              const size_t d = (size_t)r * ld + c;
              if (df) {
                out_hi[d] = x;
                out_lo[d] = 0.0f;
              } else {
                out64[d] = (double)x;
              }
            }
          }
        }
      }
      tr += (double)trf;
      fr += (double)frf;
      // (r, c) slices: 32 rows of 32 columns back out, one row per store
      __syncwarp();
      const int cc = c0 + lane;
#pragma unroll 4
      for (int i = 0; i < 32; ++i) {
        if (rb + i <= cc) {
          const uint32_t v = stA[i * 33 + lane];
          const size_t d = (size_t)(rb + i) * ld + cc;
          out0[d] = (uint16_t)(v & 0xffffu);
          out1[d] = (uint16_t)(v >> 16);
          if (fmt_bf16(F)) out2[d] = stB[i * 34 + lane];
        }
      }
      __syncwarp();
    }
  }
  tc_fence_before();
  __syncthreads();
  if (*err) {
    // failure path: let TMA copies still in flight land before the CTA exits
    if (threadIdx.x == 0) {
      for (int kb = s_consumed; kb < issued; ++kb)
        mbar_wait(full_bar(kb % C::STAGES), (uint32_t)(kb / C::STAGES) & 1u, err, false,
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
  double a, b;
  reduce_partials(buf.partials, gridDim.x, a, b, s_scratch);
  if (threadIdx.x == 0) {
    st->ticket = 0u;
    if (st->status == PROGRESS_ETIMEOUT) {
      st->done = 1;
    } else {
      st->t1 = a;
      st->t2 = b;
      st->iter = k_iter + 1;
      st->phase_iters[kPhaseSplit] += 1;
      st->x_fp64_valid = want_fp64 ? 1 : 0;
      st->x_slices_valid = 1;
      decide(st);
    }
    if (st->done && cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0u);
  }
}

// Persistent variant for the two-slice formats (FP16x2, FP16x2F): one CTA per
// SM walks the upper tiles t = blockIdx.x, blockIdx.x + gridDim.x, ... with
// barriers and tensor memory kept across tiles, so that the epilogue of one
// tile overlaps the products of the next. Tensor memory: two leading-group
// chunk buffers (columns 0..255) and two correction accumulators acc1
// (256..383 for even, 384..511 for odd tiles of the CTA). At the end of a tile
// the drain warps fold their FP32 chunk sums into the tile's acc1 buffer
// (S = w0 sum0 + w1 acc1, written back with tcgen05.st), which frees their
// registers for the next tile; the rest of that tile's epilogue (branch
// update, slices at (r, c) and at the mirror, traces) then runs in four
// 16-column pieces, each taken whenever the next tile's chunk has not arrived
// yet. A tile's acc1 buffer is handed back to the MMA issuer (acc_empty) after
// its last piece; the MMA issuer needs it again two tiles later.
constexpr int P_STAGES = 3;
constexpr int P_STG_WORDS = 32 * 17;  // per drain warp: 32 rows x 16 columns, stride 17
constexpr int P_SMEM = 1024 + P_STAGES * 2 * 2 * TILE_BYTES + DRAIN_WARPS * P_STG_WORDS * 4 + 256;

template <int F>
__global__ void __launch_bounds__(THREADS, 1)
    square_split_persist_kernel(const __grid_constant__ TensorMaps maps, DevBuffers buf,
                                unsigned long long cond) {
  static_assert(!fmt_bf16(F), "the persistent product holds two slices");
  constexpr int NS = 2;
  constexpr int STAGE_BYTES = 2 * NS * TILE_BYTES;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint32_t s_tmem;
  __shared__ int s_err;
  __shared__ int s_consumed;
  __shared__ int s_last;
  __shared__ double s_scratch[2 * THREADS / 32];

  State* st = buf.st;
  const int done = __ldcg(&st->done);
  const int phase = __ldcg(&st->phase);
  if (done) {
    if (cond && blockIdx.x == 0 && threadIdx.x == 0)
      cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0u);
    return;
  }
  if (phase != kPhaseSplit) return;  // the FP64-accurate kernel owns this step
  const int k_iter = __ldcg(&st->iter);
  const int bit = __ldcg(&st->bit);
  const int ld = st->ld;
  const uint64_t wlim = __ldcg(&st->wait_ns);  // bound on the pipeline waits
  const bool stall = __ldcg(&st->stall_test) != 0 && blockIdx.x == 0;
  const bool want_fp64 = (st->prec == PROGRESS_MIXED_FP16 || st->prec == PROGRESS_MIXED_BF16) &&
                         __ldcg(&st->split_stall) >= 1;
  const int src = k_iter & 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int T = ld / BM;
  const int tiles = T * (T + 1) / 2;
  const int my_tiles = (tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const int KB = ld / BK;
  const int NC = (KB + CHUNK - 1) / CHUNK;

  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t stg_base = base + P_STAGES * STAGE_BYTES;
  const uint32_t bars = stg_base + DRAIN_WARPS * P_STG_WORDS * 4;
  auto full_bar = [&](int s) { return bars + 8u * s; };
  auto empty_bar = [&](int s) { return bars + 8u * (P_STAGES + s); };
  auto chunk_full = [&](int b) { return bars + 8u * (2 * P_STAGES + b); };
  auto chunk_empty = [&](int b) { return bars + 8u * (2 * P_STAGES + 2 + b); };
  auto acc_full = [&](int b) { return bars + 8u * (2 * P_STAGES + 4 + b); };
  auto acc_empty = [&](int b) { return bars + 8u * (2 * P_STAGES + 6 + b); };
  const uint32_t mma_done = bars + 8u * (2 * P_STAGES + 8);
  const uint32_t stall_bar = bars + 8u * (2 * P_STAGES + 9);  // nothing arrives on it

  if (threadIdx.x == 0) {
    s_err = 0;
    s_consumed = 0;
    for (int q = 0; q < P_STAGES; ++q) {
      mbar_init(full_bar(q), 1);
      mbar_init(empty_bar(q), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(chunk_full(b), 1);
      mbar_init(chunk_empty(b), DRAIN_WARPS);
      mbar_init(acc_full(b), 1);
      mbar_init(acc_empty(b), DRAIN_WARPS);
    }
    mbar_init(mma_done, 1);
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

  int issued = 0;  // producer: k-blocks whose loads were issued (all tiles)
  if (warp == 0) {
    if (lane == 0) {
      int gk = 0;
      bool ok = true;
      for (int j = 0; j < my_tiles && ok; ++j) {
        int I, J;
        band_tile<8>((int)blockIdx.x + j * (int)gridDim.x, T, I, J);
        const int row_a = I * BM, row_b = J * BN;
        for (int kb = 0; kb < KB; ++kb, ++gk) {
          const int q = gk % P_STAGES;
          const uint32_t ph = (uint32_t)(gk / P_STAGES) & 1u;
          if (!mbar_wait(empty_bar(q), ph ^ 1u, err, true, wlim)) {
            ok = false;
            break;
          }
          mbar_expect_tx(full_bar(q), STAGE_BYTES);
          const uint32_t sa = base + q * STAGE_BYTES;
#pragma unroll
          for (int js = 0; js < NS; ++js) {
            tma_load_2d(sa + js * TILE_BYTES, &maps.m[src][js], kb * BK, row_a, full_bar(q));
            tma_load_2d(sa + (NS + js) * TILE_BYTES, &maps.m[src][js], kb * BK, row_b,
                        full_bar(q));
          }
        }
      }
      issued = gk;
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f16(0, BM, BN);
      int gk = 0, gc = 0;
      bool ok = true;
      for (int j = 0; j < my_tiles && ok; ++j) {
        const int ab = j & 1;
        const uint32_t acc1 = tmem + 256u + 128u * ab;
        if (j >= 2) {  // the epilogue of tile j - 2 has read this acc1 buffer
          if (!mbar_wait(acc_empty(ab), (uint32_t)((j - 2) >> 1) & 1u, err, true, wlim)) {
            ok = false;
            break;
          }
          tc_fence_after();
        }
        for (int kb = 0; kb < KB; ++kb, ++gk) {
          const bool chunk_first = (kb % CHUNK) == 0;
          const bool chunk_last = (kb % CHUNK) == CHUNK - 1 || kb == KB - 1;
          const int cb = gc & 1;
          const uint32_t acc0 = tmem + 128u * cb;
          if (chunk_first) {
            if (!mbar_wait(chunk_empty(cb), ((uint32_t)(gc >> 1) & 1u) ^ 1u, err, true, wlim)) {
              ok = false;
              break;
            }
            tc_fence_after();
          }
          // test of the bounded waits: after the first k-block's products, wait
          // on a barrier that nothing arrives on; it runs out after wlim
          if (stall && j == 0 && kb == 1 && !mbar_wait(stall_bar, 0u, err, true, wlim)) {
            ok = false;
            break;
          }
          const int q = gk % P_STAGES;
          const uint32_t ph = (uint32_t)(gk / P_STAGES) & 1u;
          if (!mbar_wait(full_bar(q), ph, err, true, wlim)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = base + q * STAGE_BYTES;
          const uint64_t a0 = smem_desc_sw128(sa), a1 = smem_desc_sw128(sa + TILE_BYTES);
          const uint64_t b0 = smem_desc_sw128(sa + 2 * TILE_BYTES);
          const uint64_t b1 = smem_desc_sw128(sa + 3 * TILE_BYTES);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t adv = (uint64_t)(kk * 32) >> 4;  // 32 B per K = 16 step
            const uint32_t first = (kb == 0 && kk == 0) ? 0u : 1u;
            const uint32_t chunk_acc = (chunk_first && kk == 0) ? 0u : 1u;
            mma_f16(acc0, a0 + adv, b0 + adv, idesc, chunk_acc);
            mma_f16(acc1, a0 + adv, b1 + adv, idesc, first);
            mma_f16(acc1, a1 + adv, b0 + adv, idesc, 1u);
          }
          mma_commit(empty_bar(q));  // frees the stage once these MMAs have read it
          if (chunk_last) {
            mma_commit(chunk_full(cb));
            ++gc;
          }
          s_consumed = gk + 1;
        }
        if (ok) mma_commit(acc_full(ab));  // the tile's acc1 (and last chunk) complete
      }
      mma_commit(mma_done);  // every MMA issued so far is complete
    }
    __syncwarp();
  }

  // ---- drain + epilogue warps: thread owns TMEM lane = tile row and 64
  // columns; sums the leading-group chunks with round-to-nearest FP32 adds,
  // folds them into acc1 at the end of a tile and runs the tile's epilogue in
  // pieces while the next tile's products proceed.
  double tr = 0.0, fr = 0.0;
  if (warp >= DRAIN_WARP0) {
    using W = SliceWeights<F>;
    const int dw = warp - DRAIN_WARP0;
    const int quarter = warp & 3;
    const int half = dw >> 2;
    const int row = quarter * 32 + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
    const bool odd = src != 0;
    const uint16_t* xs0 = odd ? buf.sl[1][0] : buf.sl[0][0];
    const uint16_t* xs1 = odd ? buf.sl[1][1] : buf.sl[0][1];
    uint16_t* const out0 = odd ? buf.sl[0][0] : buf.sl[1][0];
    uint16_t* const out1 = odd ? buf.sl[0][1] : buf.sl[1][1];
    double* out64 = odd ? buf.x64[0] : buf.x64[1];
    const bool df = st->df64 != 0;
    float* out_hi = reinterpret_cast<float*>(out64);
    float* out_lo = out_hi + (size_t)ld * ld;
    uint32_t* stg = reinterpret_cast<uint32_t*>(smem_raw + (stg_base - smem_u32(smem_raw))) +
                    dw * P_STG_WORDS;
    float sum0[DCOLS];
#pragma unroll
    for (int i = 0; i < DCOLS; ++i) sum0[i] = 0.0f;
    // the tile whose epilogue is pending (-1: none) and its next piece
    int p_j = -1, p_piece = 0, p_ra = 0, p_rb = 0;

    // one 16-column piece of the pending epilogue
    auto do_piece = [&]() {
      const int r = p_ra + row;
      const int col = half * DCOLS + p_piece * 16;  // column in the tile
      const int c0 = p_rb + col;
      uint32_t m01[16];
      if (bit) {  // X at the mirror (X symmetric: consecutive lanes read consecutive r)
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const size_t m = (size_t)(c0 + i) * ld + r;
          m01[i] = (uint32_t)xs0[m] | ((uint32_t)xs1[m] << 16);
        }
      }
      uint32_t u[16];
      tmem_ld16(lane_addr + 256u + 128u * (uint32_t)(p_j & 1) + (uint32_t)col, u);
      tmem_ld_wait();
      float trf = 0.0f, frf = 0.0f;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int c = c0 + i;
        float x = __uint_as_float(u[i]);
        if (bit)
          x = 2.0f * join_value<F>((uint16_t)(m01[i] & 0xffffu), (uint16_t)(m01[i] >> 16),
                                   (uint16_t)0) -
              x;
        uint16_t a, b2, c2;
        split_value_f<F>(x, a, b2, c2);
        stg[lane * 17 + i] = (uint32_t)a | ((uint32_t)b2 << 16);
        if (r <= c) {
          if (r == c) {
            trf += x;
            frf += x * x;
          } else {
            frf += 2.0f * x * x;
            const size_t m = (size_t)c * ld + r;  // mirror (c, r)
            out0[m] = a;
            out1[m] = b2;
            if (want_fp64) {
              if (df) {
                out_hi[m] = x;
                out_lo[m] = 0.0f;
              } else {
                out64[m] = (double)x;
              }
            }
          }
          if (want_fp64) {
            const size_t d = (size_t)r * ld + c;
            if (df) {
              out_hi[d] = x;
              out_lo[d] = 0.0f;
            } else {
              out64[d] = (double)x;
            }
          }
        }
      }
      tr += (double)trf;
      fr += (double)frf;
      // (r, c) slices: 32 rows of 16 columns, two rows per store instruction
      __syncwarp();
      const int rbase = p_ra + quarter * 32;
      const int cc = c0 + (lane & 15);
#pragma unroll 4
      for (int it = 0; it < 16; ++it) {
        const int i = 2 * it + (lane >> 4);
        if (rbase + i <= cc) {
          const uint32_t v = stg[i * 17 + (lane & 15)];
          const size_t d = (size_t)(rbase + i) * ld + cc;
          out0[d] = (uint16_t)(v & 0xffffu);
          out1[d] = (uint16_t)(v >> 16);
        }
      }
      __syncwarp();
      if (++p_piece == DCOLS / 16) {  // the tile's acc1 buffer is free again
        tc_fence_before();
        if (lane == 0) mbar_arrive_cta(acc_empty(p_j & 1));
        p_j = -1;
      }
    };

    int gc = 0;
    bool ok = true;
    for (int j = 0; j < my_tiles && ok; ++j) {
      for (int c = 0; c < NC; ++c, ++gc) {
        const int cb = gc & 1;
        const uint32_t par = (uint32_t)(gc >> 1) & 1u;
        // pieces of the pending epilogue while this chunk is not ready yet
        while (p_j >= 0 && __shfl_sync(0xffffffffu, (int)mbar_test_wait(chunk_full(cb), par), 0) == 0)
          do_piece();
        if (!mbar_wait(chunk_full(cb), par, err, true, wlim)) {
          ok = false;
          break;
        }
        tc_fence_after();
        // 32 columns at a time (register budget), the buffer freed after the last
#pragma unroll
        for (int q = 0; q < DCOLS / 32; ++q) {
          float v[32];
          tmem_ld32(lane_addr + 128u * cb + half * DCOLS + q * 32, v);
          tmem_ld_wait();
          if (q == DCOLS / 32 - 1) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cta(chunk_empty(cb));
          }
#pragma unroll
          for (int i = 0; i < 32; ++i) sum0[q * 32 + i] += v[i];
        }
      }
      if (!ok) break;
      while (p_j >= 0) do_piece();
      if (!mbar_wait(acc_full(j & 1), (uint32_t)(j >> 1) & 1u, err, true, wlim)) {
        ok = false;
        break;
      }
      tc_fence_after();
      // S = w0 sum0 + w1 acc1, written back over acc1 (this thread's row and columns)
      const uint32_t a1 = lane_addr + 256u + 128u * (uint32_t)(j & 1) + half * DCOLS;
#pragma unroll
      for (int q = 0; q < DCOLS / 16; ++q) {
        uint32_t u[16];
        tmem_ld16(a1 + q * 16, u);
        tmem_ld_wait();
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          u[i] = __float_as_uint(sum0[q * 16 + i] * W::w0 + __uint_as_float(u[i]) * W::w1);
          sum0[q * 16 + i] = 0.0f;
        }
        tmem_st16(a1 + q * 16, u);
      }
      tmem_st_wait();
      int I, J;
      band_tile<8>((int)blockIdx.x + j * (int)gridDim.x, T, I, J);
      p_j = j;
      p_piece = 0;
      p_ra = I * BM;
      p_rb = J * BN;
    }
    if (ok)
      while (p_j >= 0) do_piece();
  }

  // every MMA is complete before tensor memory is released (the MMA thread
  // always commits mma_done; this wait does not abort early)
  mbar_wait(mma_done, 0u, err, false);
  tc_fence_after();
  tc_fence_before();
  __syncthreads();
  if (*err) {
    // failure path: let TMA copies still in flight land before the CTA exits
    if (threadIdx.x == 0) {
      for (int g = s_consumed; g < issued; ++g)
        mbar_wait(full_bar(g % P_STAGES), (uint32_t)(g / P_STAGES) & 1u, err, false,
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
  double a, b;
  reduce_partials(buf.partials, gridDim.x, a, b, s_scratch);
  if (threadIdx.x == 0) {
    st->ticket = 0u;
    if (st->status == PROGRESS_ETIMEOUT) {
      st->done = 1;
    } else {
      st->t1 = a;
      st->t2 = b;
      st->iter = k_iter + 1;
      st->phase_iters[kPhaseSplit] += 1;
      st->x_fp64_valid = want_fp64 ? 1 : 0;
      st->x_slices_valid = 1;
      decide(st);
    }
    if (st->done && cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0u);
  }
}

// Thresholded SP2 product (Listing 1's cutoff tau), persistent: one CTA per SM
// walks the upper tiles t = blockIdx.x, blockIdx.x + gridDim.x, ... First every
// warp checks one tile at a time (all warps at once): a tile needs work unless
// no k-tile pair (I, k), (J, k) of X is flagged non-zero, the result is zero
// (X^2, or X zero there) and the destination set already holds zeros there.
// The tiles that need work then run the pipeline of square_split_kernel one
// after the other with tensor memory and mbarriers kept across tiles (the
// stage, chunk and accumulator phases continue from tile to tile), streaming
// only the flagged k-blocks. The epilogue prunes |x| < tau from the product and
// from 2X - X^2 and writes the tile's new flag.
constexpr int SP_MAX_TILES = 1024;  // tiles per CTA (the host sizes the grid)

template <int F>
__global__ void __launch_bounds__(THREADS, 1)
    square_split_sparse_kernel(const __grid_constant__ TensorMaps maps, DevBuffers buf,
                               unsigned long long cond, float tau) {
  using C = Cfg<F>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint32_t s_tmem;
  __shared__ int s_err;
  __shared__ int s_consumed;  // global k-block index consumed by the MMA thread
  __shared__ int s_last;
  __shared__ double s_scratch[2 * THREADS / 32];
  __shared__ uint16_t s_klist[1024];
  __shared__ int s_wcnt[THREADS / 32];
  __shared__ uint8_t s_work[SP_MAX_TILES];

  State* st = buf.st;
  const int done = __ldcg(&st->done);
  const int phase = __ldcg(&st->phase);
  if (done) {
    if (cond && blockIdx.x == 0 && threadIdx.x == 0)
      cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0u);
    return;
  }
  if (phase != kPhaseSplit) return;
  const int k_iter = __ldcg(&st->iter);
  const int bit = __ldcg(&st->bit);
  const int ld = st->ld;
  const int src = k_iter & 1, dst = (k_iter + 1) & 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int T = ld / BM;
  const int tiles = T * (T + 1) / 2;
  const int my_tiles = (tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const uint8_t* fl = buf.tflags[src];
  uint8_t* fd = buf.tflags[dst];

  // pass 1: which of this CTA's tiles need work (one warp per tile)
  for (int j = warp; j < my_tiles; j += THREADS / 32) {
    int I, J;
    tri_tile((int)blockIdx.x + j * (int)gridDim.x, T, I, J);
    bool any = false;
    for (int b0 = 0; b0 < T && !any; b0 += 32) {
      const int q = b0 + lane;
      any = __any_sync(0xffffffffu, q < T && fl[(size_t)I * T + q] != 0 &&
                                        fl[(size_t)J * T + q] != 0);
    }
    if (lane == 0) {
      const bool zero_result = !any && (bit == 0 || fl[(size_t)I * T + J] == 0);
      s_work[j] = (zero_result && fd[(size_t)I * T + J] == 0) ? 0 : 1;
    }
  }
  __syncthreads();
  int nwork = 0;
  for (int j = 0; j < my_tiles; ++j) nwork += s_work[j];

  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t bars = base + C::STAGES * C::STAGE_BYTES;
  auto full_bar = [&](int s) { return bars + 8u * s; };
  auto empty_bar = [&](int s) { return bars + 8u * (C::STAGES + s); };
  const uint32_t accum_bar = bars + 8u * (2 * C::STAGES);
  const uint32_t chunk_full = bars + 8u * (2 * C::STAGES + 1);
  const uint32_t chunk_empty = bars + 8u * (2 * C::STAGES + 1 + C::NBUF);

  double tr = 0.0, fr = 0.0;
  if (nwork > 0) {
    if (threadIdx.x == 0) {
      s_err = 0;
      s_consumed = 0;
      for (int s = 0; s < C::STAGES; ++s) {
        mbar_init(full_bar(s), 1);
        mbar_init(empty_bar(s), 1);
      }
      mbar_init(accum_bar, 1);
      for (int b = 0; b < C::NBUF; ++b) {
        mbar_init(chunk_full + 8u * b, 1);
        mbar_init(chunk_empty + 8u * b, DRAIN_WARPS);
      }
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    if (warp == 0) tmem_alloc(smem_u32(&s_tmem), TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    volatile int* err = &s_err;
    const bool drain = warp >= DRAIN_WARP0;
    const int quarter = warp & 3;
    const int half = drain ? (warp - DRAIN_WARP0) >> 2 : 0;
    const int row = quarter * 32 + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
    const bool odd = src != 0;
    const uint16_t* xs0 = odd ? buf.sl[1][0] : buf.sl[0][0];
    const uint16_t* xs1 = odd ? buf.sl[1][1] : buf.sl[0][1];
    const uint16_t* xs2 = odd ? buf.sl[1][2] : buf.sl[0][2];
    uint16_t* const out0 = odd ? buf.sl[0][0] : buf.sl[1][0];
    uint16_t* const out1 = odd ? buf.sl[0][1] : buf.sl[1][1];
    uint16_t* const out2 = odd ? buf.sl[0][2] : buf.sl[1][2];
    int g = 0;        // k-blocks of the earlier tiles (stage ring position)
    int gc = 0;       // leading-group chunks of the earlier tiles
    int ntile = 0;    // tiles done (accumulator barrier phase)
    int issued = 0;   // producer: global k-blocks whose loads were issued
    for (int j = 0; j < my_tiles; ++j) {
      if (!s_work[j]) continue;
      int I, J;
      tri_tile((int)blockIdx.x + j * (int)gridDim.x, T, I, J);
      const int row_a = I * BM, row_b = J * BN;
      // this tile's flagged k-blocks, in order (every thread counts the same)
      int total = 0;
      for (int b0 = 0; b0 < T; b0 += THREADS) {
        const int t = b0 + (int)threadIdx.x;
        const bool act = t < T && fl[(size_t)I * T + t] != 0 && fl[(size_t)J * T + t] != 0;
        const unsigned bal = __ballot_sync(0xffffffffu, act);
        if (lane == 0) s_wcnt[warp] = __popc(bal);
        __syncthreads();
        int before = total, sum = 0;
        for (int w2 = 0; w2 < THREADS / 32; ++w2) {
          if (w2 < warp) before += s_wcnt[w2];
          sum += s_wcnt[w2];
        }
        before += __popc(bal & ((1u << lane) - 1u));
        if (act) {
          s_klist[2 * before] = (uint16_t)(2 * t);
          s_klist[2 * before + 1] = (uint16_t)(2 * t + 1);
        }
        total += sum;
        __syncthreads();
      }
      const int nkb = 2 * total;
      const int NC = (nkb + CHUNK - 1) / CHUNK;
      if (threadIdx.x == 0 && nkb > 0) atomicAdd(&st->kblocks, (unsigned long long)nkb);
      if (warp == 0) {
        if (lane == 0) {
          for (int q = 0; q < nkb; ++q) {
            const int gq = g + q;
            const int s = gq % C::STAGES;
            const uint32_t ph = (uint32_t)(gq / C::STAGES) & 1u;
            if (!mbar_wait(empty_bar(s), ph ^ 1u, err)) break;
            mbar_expect_tx(full_bar(s), C::STAGE_BYTES);
            const uint32_t sa = base + s * C::STAGE_BYTES;
            const int kb = (int)s_klist[q];
#pragma unroll
            for (int jj = 0; jj < C::NS; ++jj) {
              tma_load_2d(sa + jj * TILE_BYTES, &maps.m[src][jj], kb * BK, row_a, full_bar(s));
              tma_load_2d(sa + (C::NS + jj) * TILE_BYTES, &maps.m[src][jj], kb * BK, row_b,
                          full_bar(s));
            }
            issued = gq + 1;
          }
        }
        __syncwarp();
      } else if (warp == 1) {
        if (lane == 0) {
          constexpr uint32_t idesc = idesc_f16(fmt_bf16(F) ? 1 : 0, BM, BN);
          const uint32_t acc1 = tmem + 128u * C::NBUF, acc2 = acc1 + 128u;
          bool ok = true;
          for (int q = 0; q < nkb && ok; ++q) {
            const int c = gc + q / CHUNK, cb = c % C::NBUF;
            const bool chunk_first = (q % CHUNK) == 0;
            const bool chunk_last = (q % CHUNK) == CHUNK - 1 || q == nkb - 1;
            const uint32_t acc0 = tmem + 128u * cb;
            if (chunk_first) {
              if (!mbar_wait(chunk_empty + 8u * cb, ((uint32_t)(c / C::NBUF) & 1u) ^ 1u, err)) {
                ok = false;
                break;
              }
              tc_fence_after();
            }
            const int gq = g + q;
            const int s = gq % C::STAGES;
            const uint32_t ph = (uint32_t)(gq / C::STAGES) & 1u;
            if (!mbar_wait(full_bar(s), ph, err)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = base + s * C::STAGE_BYTES;
            uint64_t a[3], b[3];
#pragma unroll
            for (int jj = 0; jj < C::NS; ++jj) {
              a[jj] = smem_desc_sw128(sa + jj * TILE_BYTES);
              b[jj] = smem_desc_sw128(sa + (C::NS + jj) * TILE_BYTES);
            }
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              const uint64_t adv = (uint64_t)(kk * 32) >> 4;
              const uint32_t first = (q == 0 && kk == 0) ? 0u : 1u;
              const uint32_t chunk_acc = (chunk_first && kk == 0) ? 0u : 1u;
              mma_f16(acc0, a[0] + adv, b[0] + adv, idesc, chunk_acc);
              mma_f16(acc1, a[0] + adv, b[1] + adv, idesc, first);
              mma_f16(acc1, a[1] + adv, b[0] + adv, idesc, 1u);
              if (fmt_bf16(F)) {
                mma_f16(acc2, a[0] + adv, b[2] + adv, idesc, first);
                mma_f16(acc2, a[2] + adv, b[0] + adv, idesc, 1u);
                mma_f16(acc2, a[1] + adv, b[1] + adv, idesc, 1u);
              }
            }
            mma_commit(empty_bar(s));
            if (chunk_last) mma_commit(chunk_full + 8u * cb);
            s_consumed = gq + 1;
          }
          if (nkb > 0)
            mma_commit(accum_bar);
          else
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(accum_bar) : "memory");
        }
        __syncwarp();
      }
      float sum0[DCOLS];
#pragma unroll
      for (int jj = 0; jj < DCOLS; ++jj) sum0[jj] = 0.0f;
      if (drain) {
        for (int c = 0; c < NC; ++c) {
          const int gcc = gc + c, cb = gcc % C::NBUF;
          if (!mbar_wait(chunk_full + 8u * cb, (uint32_t)(gcc / C::NBUF) & 1u, err)) break;
          tc_fence_after();
          float v[DCOLS];
#pragma unroll
          for (int q = 0; q < DCOLS / 32; ++q)
            tmem_ld32(lane_addr + 128u * cb + half * DCOLS + q * 32, v + q * 32);
          tmem_ld_wait();
          tc_fence_before();
          __syncwarp();
          if (lane == 0)
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(chunk_empty + 8u * cb)
                         : "memory");
#pragma unroll
          for (int jj = 0; jj < DCOLS; ++jj) sum0[jj] += v[jj];
        }
      }
      const bool ok = mbar_wait(accum_bar, (uint32_t)ntile & 1u, err, false);
      tc_fence_after();
      int nz = 0;
      if (drain && ok && *err == 0) {
        using W = SliceWeights<F>;
        const int r = row_a + row;
        uint32_t* stA = reinterpret_cast<uint32_t*>(smem_raw + (base - smem_u32(smem_raw))) +
                        (warp - DRAIN_WARP0) * (32 * 33);
        uint16_t* stB = reinterpret_cast<uint16_t*>(smem_raw + (base - smem_u32(smem_raw)) +
                                                    DRAIN_WARPS * 32 * 33 * 4) +
                        (warp - DRAIN_WARP0) * (32 * 34);
        const int rb = row_a + quarter * 32;
#pragma unroll
        for (int ch = 0; ch < DCOLS / 32; ++ch) {
          const int col = half * DCOLS + ch * 32;
          const int c0 = row_b + col;
          float trf = 0.0f, frf = 0.0f;
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            const int cs = c0 + hh * 16;
            uint32_t m01[16], m2[16];
            if (bit) {
#pragma unroll
              for (int jj = 0; jj < 16; ++jj) {
                const size_t m = (size_t)(cs + jj) * ld + r;
                m01[jj] = (uint32_t)xs0[m] | ((uint32_t)xs1[m] << 16);
                m2[jj] = fmt_bf16(F) ? (uint32_t)xs2[m] : 0u;
              }
            }
            uint32_t u1[16], u2[16];
            if (nkb > 0) {
              tmem_ld16(lane_addr + 128u * C::NBUF + col + hh * 16, u1);
              if (fmt_bf16(F)) tmem_ld16(lane_addr + 128u * (C::NBUF + 1) + col + hh * 16, u2);
              tmem_ld_wait();
            } else {
#pragma unroll
              for (int jj = 0; jj < 16; ++jj) u1[jj] = u2[jj] = 0u;
            }
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) {
              const int jc = hh * 16 + jj;
              const int c = cs + jj;
              float x = sum0[ch * 32 + jc] * W::w0 + __uint_as_float(u1[jj]) * W::w1;
              if (fmt_bf16(F)) x += __uint_as_float(u2[jj]) * W::w2;
              if (fabsf(x) < tau) x = 0.0f;  // prune the product
              if (bit) {
                x = 2.0f * join_value<F>((uint16_t)(m01[jj] & 0xffffu),
                                         (uint16_t)(m01[jj] >> 16), (uint16_t)m2[jj]) -
                    x;
                if (fabsf(x) < tau) x = 0.0f;  // prune the update
              }
              if (x != 0.0f) nz = 1;
              uint16_t a, b2, c2;
              split_value_f<F>(x, a, b2, c2);
              stA[lane * 33 + jc] = (uint32_t)a | ((uint32_t)b2 << 16);
              if (fmt_bf16(F)) stB[lane * 34 + jc] = c2;
              if (r <= c) {
                if (r == c) {
                  trf += x;
                  frf += x * x;
                } else {
                  frf += 2.0f * x * x;
                  const size_t m = (size_t)c * ld + r;
                  out0[m] = a;
                  out1[m] = b2;
                  if (fmt_bf16(F)) out2[m] = c2;
                }
              }
            }
          }
          tr += (double)trf;
          fr += (double)frf;
          __syncwarp();
          const int cc = c0 + lane;
#pragma unroll 4
          for (int i = 0; i < 32; ++i) {
            if (rb + i <= cc) {
              const uint32_t v = stA[i * 33 + lane];
              const size_t d = (size_t)(rb + i) * ld + cc;
              out0[d] = (uint16_t)(v & 0xffffu);
              out1[d] = (uint16_t)(v >> 16);
              if (fmt_bf16(F)) out2[d] = stB[i * 34 + lane];
            }
          }
          __syncwarp();
        }
        // the staging area is the operand ring: order these generic-proxy
        // writes before the next tile's TMA writes into it
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      }
      tc_fence_before();
      const int any = __syncthreads_or(nz);
      tc_fence_after();
      if (threadIdx.x == 0) {
        fd[(size_t)I * T + J] = (uint8_t)(any ? 1 : 0);
        fd[(size_t)J * T + I] = (uint8_t)(any ? 1 : 0);
      }
      g += nkb;
      gc += NC;
      ++ntile;
      if (*err) break;  // (uniform: read after the barrier above)
    }
    __syncthreads();
    if (*err) {
      // failure path: let TMA copies still in flight land before the CTA exits
      if (threadIdx.x == 0) {
        for (int gq = s_consumed; gq < issued; ++gq)
          mbar_wait(full_bar(gq % C::STAGES), (uint32_t)(gq / C::STAGES) & 1u, err, false,
                    kWaitLimitNs / 10);
      }
      __syncthreads();
    }
    if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
    if (*err && threadIdx.x == 0) {
      st->status = PROGRESS_ETIMEOUT;
      st->done = 1;
    }
  }

  block_sum2(tr, fr, s_scratch);
  if (threadIdx.x == 0) {
    buf.partials[2 * blockIdx.x] = tr;
    buf.partials[2 * blockIdx.x + 1] = fr;
  }
  if (!last_cta_arrives(st, gridDim.x, &s_last)) return;
  double a, b;
  reduce_partials(buf.partials, gridDim.x, a, b, s_scratch);
  if (threadIdx.x == 0) {
    st->ticket = 0u;
    if (st->status == PROGRESS_ETIMEOUT) {
      st->done = 1;
    } else {
      st->t1 = a;
      st->t2 = b;
      st->iter = k_iter + 1;
      st->phase_iters[kPhaseSplit] += 1;
      st->x_fp64_valid = 0;
      st->x_slices_valid = 1;
      decide(st);
    }
    if (st->done && cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0u);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encoder() {
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

bool encode_maps(const DevBuffers& b, int ld, int fmt, TensorMaps* maps) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = get_encoder();
  if (!enc) return false;
  const int ns = fmt_slices(fmt);
  memset(maps, 0, sizeof *maps);
  for (int k = 0; k < 2; ++k) {
    for (int j = 0; j < ns; ++j) {
      if (!b.sl[k][j]) return false;
      cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)ld};
      cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
      cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)BM};
      cuuint32_t estr[2] = {1, 1};
      CUresult r = enc(&maps->m[k][j],
                       fmt_bf16(fmt) ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                     : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                       2, (void*)b.sl[k][j], dims, strides, box, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return false;
    }
  }
  return true;
}

}  // namespace

int split_tile_count(int ld) {
  const int T = ld / BM;
  return T * (T + 1) / 2;
}

bool split_tensor_maps_ready(const DevBuffers& b, int ld, int fmt) {
  TensorMaps m;
  return encode_maps(b, ld, fmt, &m);
}

cudaError_t launch_square_split(const DevBuffers& b, const SolveParams& p,
                                unsigned long long cond_handle, cudaStream_t s) {
  const int ld = p.ld;
  if (ld % BM) return cudaErrorInvalidValue;
  const int tiles = split_tile_count(ld);
  if (tiles > b.max_partials) return cudaErrorInvalidValue;
  TensorMaps maps;
  if (!encode_maps(b, ld, p.slice_fmt, &maps)) return cudaErrorInvalidValue;
  if (p.tau > 0.0f) {
    if (p.slice_fmt != kFP16x2 && p.slice_fmt != kBF16x3) return cudaErrorInvalidValue;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // one CTA per SM, at most SP_MAX_TILES tiles each, never more CTAs than tiles
    int grid = nsm < tiles ? nsm : tiles;
    if ((tiles + grid - 1) / grid > SP_MAX_TILES) grid = (tiles + SP_MAX_TILES - 1) / SP_MAX_TILES;
    switch (p.slice_fmt) {
#define SP2_SQP(F)                                                                          \
  case F: {                                                                                 \
    const int smem = Cfg<F>::SMEM;                                                          \
    cudaFuncSetAttribute(square_split_sparse_kernel<F>,                                     \
                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);                \
    square_split_sparse_kernel<F><<<grid, THREADS, smem, s>>>(maps, b, cond_handle, p.tau); \
    break;                                                                                  \
  }
      SP2_SQP(kFP16x2)
      SP2_SQP(kBF16x3)
#undef SP2_SQP
      default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  if (!fmt_bf16(p.slice_fmt) && p.split_tile == 2) return launch_square_wide(b, p, cond_handle, s);
  if (!fmt_bf16(p.slice_fmt)) {
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int grid = nsm < tiles ? nsm : tiles;  // one CTA per SM, never more than tiles
    switch (p.slice_fmt) {
#define SP2_SQPER(F)                                                                       \
  case F:                                                                                  \
    cudaFuncSetAttribute(square_split_persist_kernel<F>,                                   \
                         cudaFuncAttributeMaxDynamicSharedMemorySize, P_SMEM);            \
    square_split_persist_kernel<F><<<grid, THREADS, P_SMEM, s>>>(maps, b, cond_handle);    \
    break;
      SP2_SQPER(kFP16x2)
      SP2_SQPER(kFP16x2F)
#undef SP2_SQPER
      default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  switch (p.slice_fmt) {
#define SP2_SQS(F)                                                                     \
  case F: {                                                                            \
    const int smem = Cfg<F>::SMEM;                                                     \
    cudaFuncSetAttribute(square_split_kernel<F>,                                       \
                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);           \
    square_split_kernel<F><<<tiles, THREADS, smem, s>>>(maps, b, cond_handle);         \
    break;                                                                             \
  }
    SP2_SQS(kFP16x2)
    SP2_SQS(kBF16x3)
    SP2_SQS(kFP16x2F)
    SP2_SQS(kBF16x3F)
#undef SP2_SQS
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace sp2
