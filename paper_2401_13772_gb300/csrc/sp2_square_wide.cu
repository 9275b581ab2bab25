// Split-precision SP2 product step (FP16x2 slices) on 128 x 256 tiles.
//
// The same product as square_split_persist_kernel -- S = X*X from the FP16
// hi/lo slices of the symmetric iterate, acc0 = sum hi*hi^T summed in 256-k
// chunks with round-to-nearest FP32 adds, acc1 = sum (hi*lo^T + lo*hi^T) over
// the whole K, S = w0 sum0 + w1 acc1, the SP2 branch (§IV.A) chosen on the
// device, new slices at (r, c) and at the mirror (c, r), partial traces -- with
// one tcgen05.mma of N = 256 where that kernel issues two of N = 128. The wider
// product reads its 128-row A slice from shared memory once per 256 columns
// instead of once per 128: per k-step of 16 the three products read 36 KB
// and the TMA writes 24 KB for 426 tensor-core clocks (141 B/clk), against
// 24 KB + 16 KB for 213 clocks (188 B/clk) with 128 x 128 tiles, above the
// 128 B/clk that shared memory delivers. Every MMA of an element is the same
// in both kernels, in the same order, so the results agree bit for bit.
//
//   warp 0, one lane : TMA producer -- per k-block of 64: A hi, A lo (128 x 64,
//                      128 B rows, 128 B swizzle) and B hi, B lo (256 x 64) into
//                      a 2-deep ring of 96 KB stages (64 B rows halve the bytes per
//                      TMA row request: measured, the operand stream alone then
//                      ran at 8.8 TB/s instead of 24)
//   warp 1, one lane : MMA issuer -- per k-block two groups of products: H
//                      (acc0 += hi hi^T, two MMAs) and C (acc1 += hi lo^T +
//                      lo hi^T, four MMAs). acc0 (tensor memory columns 0..255)
//                      is one chunk buffer and acc1 (256..511) one accumulator,
//                      so H waits for the drain of the previous chunk and C for
//                      the previous tile's epilogue; the issuer runs either
//                      group one k-block ahead of the other meanwhile.
//                      A stage is freed once both of its groups are issued.
//   warps 3..18      : drain -- four warps per 32-lane quarter of tensor memory,
//                      each thread owns one tile row and 64 columns: adds every
//                      finished chunk into 64 FP32 registers, writes S over acc1
//                      at the end of a tile and runs the epilogue from there in
//                      8-column pieces; acc1 is handed back after the last one.
//                      The partial traces go to shared memory once per tile, so
//                      that no FP64 value stays in registers next to the 64 sums.
//
// The persistent grid walks the tiles in the band order of wide_tile (one CTA
// per SM). Every mbarrier wait is bounded; a wait that runs out records
// PROGRESS_ETIMEOUT in the solve state, stops the loop, and the CTA lets its
// copies in flight land and frees its tensor memory before it exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <string.h>

#include "sp2_common.cuh"
#include "sp2_launch.h"
#include "sp2_slices.cuh"
#include "sp2_tc.cuh"

namespace sp2 {
namespace {

using namespace tc;

constexpr int BM = 128;                          // tile rows
constexpr int BN = 256;                          // tile columns
constexpr int BK = 64;                           // k per stage (128 B rows)
constexpr int A_BYTES = BM * BK * 2;             // one A slice box (16 KB)
constexpr int B_BYTES = BN * BK * 2;             // one B slice box (32 KB)
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int STAGES = 2;
constexpr int CHUNK = 4;                         // k-blocks per acc0 chunk (K = 256)
constexpr int THREADS = 608;                     // 19 warps
constexpr int DRAIN_WARP0 = 3;
constexpr int DRAIN_WARPS = 16;
constexpr int DCOLS = BN / 4;                    // columns per drain thread
constexpr int TMEM_COLS = 512;                   // acc0 chunk | acc1
constexpr int STG_WORDS = 32 * 8;                // per drain warp: 32 rows x 8 columns
constexpr int BAND = 8;                          // row blocks per band of the tile order
constexpr int NBARS = 2 * STAGES + 6;
constexpr int SMEM = 1024 + STAGES * STAGE_BYTES + DRAIN_WARPS * STG_WORDS * 4 + 8 * NBARS;
static_assert(DRAIN_WARPS == 4 * (BN / DCOLS), "four column groups per lane quarter");

struct WideMaps {
  CUtensorMap a[2][2];  // [ping-pong set][slice]: 128 x 64 boxes
  CUtensorMap b[2][2];  //                         256 x 64 boxes
};

__device__ __forceinline__ void mbar_arrive_cta(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

// Per-launch values of the epilogue, in shared memory: the drain warps read them
// when a tile ends instead of holding them in registers across the chunks.
struct WideCtx {
  const uint16_t* xs0;  // slices of X (source set)
  const uint16_t* xs1;
  uint16_t* out0;       // slices of X' (destination set)
  uint16_t* out1;
  double* out64;        // FP64 X' (or its double-float planes)
  unsigned long long wlim;
  int ld, T, bit, want_fp64, df, first_tile, tile_step;
};

// Epilogue of tile j of this CTA for one drain warp: its 32 rows (lanes) and
// 64 columns of S = X*X, read from tensor memory at s_addr in 8-column pieces.
// X' = S or 2X - S (the branch of §IV.A, decided before the product), its
// slices at (r, c) -- staged in shared memory so that the stores run along
// rows -- and at the mirror (c, r), FP64 X' when the schedule may leave the
// split phase next, and the partial traces Tr X', ||X'||_F^2. The tensor
// cores wait for this epilogue (acc1 holds S), so it keeps off the FP64 pipe,
// which is slow on this part: FP32 sums per piece, compensated across pieces,
// one FP64 warp sum per tile into this warp's slot of s_tr.
template <int F>
__device__ __forceinline__ void wide_epilogue(const WideCtx& cx, int j, int dw, int lane,
                                              uint32_t s_addr, uint32_t* stg, double* s_tr) {
  const int ld = cx.ld;
  int I, P;
  wide_tile<BAND>(cx.first_tile + j * cx.tile_step, cx.T, I, P);
  const int quarter = (dw + DRAIN_WARP0) & 3;
  const int rbase = I * BM + quarter * 32;
  const int r = rbase + lane;
  const int bit = cx.bit, want_fp64 = cx.want_fp64, df = cx.df;
  const uint16_t* xs0 = cx.xs0;
  const uint16_t* xs1 = cx.xs1;
  uint16_t* const out0 = cx.out0;
  uint16_t* const out1 = cx.out1;
  double* const out64 = cx.out64;
  float* const out_hi = reinterpret_cast<float*>(out64);
  float* const out_lo = out_hi + (size_t)ld * ld;
  const int cbase = P * BN + (dw >> 2) * DCOLS;
  // X at the mirror (X symmetric: consecutive lanes read consecutive r)
  auto load_mirror = [&](int c0, uint32_t* m) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int c = c0 + i;
      const size_t a = (size_t)c * ld + r;
      m[i] = c < ld ? ((uint32_t)xs0[a] | ((uint32_t)xs1[a] << 16)) : 0u;
    }
  };
  float ts = 0.0f, tc = 0.0f, fs = 0.0f, fc = 0.0f;
  for (int piece = 0; piece < DCOLS / 8; ++piece) {
    const int c0 = cbase + piece * 8;
    uint32_t m01[8];
    if (bit) load_mirror(c0, m01);
    uint32_t u[8];
    tmem_ld8(s_addr + (uint32_t)(piece * 8), u);
    tmem_ld_wait();
    float trf = 0.0f, frf = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int c = c0 + i;
      float x = __uint_as_float(u[i]);
      if (bit)
        x = 2.0f * join_value<F>((uint16_t)(m01[i] & 0xffffu), (uint16_t)(m01[i] >> 16),
                                 (uint16_t)0) -
            x;
      uint16_t a, b2, c2;
      split_value_f<F>(x, a, b2, c2);
      stg[lane * 8 + (i ^ (lane & 7))] = (uint32_t)a | ((uint32_t)b2 << 16);
      if (r <= c && c < ld) {
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
    kahan_add(ts, tc, trf);
    kahan_add(fs, fc, frf);
    // (r, c) slices: 32 rows of 8 columns, four rows per store instruction
    __syncwarp();
    const int cc = c0 + (lane & 7);
#pragma unroll 4
    for (int it = 0; it < 8; ++it) {
      const int i = 4 * it + (lane >> 3);
      if (rbase + i <= cc && cc < ld) {
        const uint32_t v = stg[i * 8 + ((lane & 7) ^ (i & 7))];
        const size_t d = (size_t)(rbase + i) * ld + cc;
        out0[d] = (uint16_t)(v & 0xffffu);
        out1[d] = (uint16_t)(v >> 16);
      }
    }
    __syncwarp();
  }
  // a thread holds at most one diagonal entry per tile: the trace sums it in
  // FP64 (and only in tiles that reach the diagonal), as exactly as an FP64 sum
  // of single entries; ||X'||_F^2 takes the thread's compensated FP32 sum
  const bool diag = 2 * P == (I & ~1);
  const double a = diag ? warp_sum((double)(ts - tc)) : 0.0;
  const double b = warp_sum((double)(fs - fc));
  if (lane == 0) {
    s_tr[0] += a;
    s_tr[1] += b;
  }
}

template <int F>
__global__ void __launch_bounds__(THREADS, 1)
    square_wide_kernel(const __grid_constant__ WideMaps maps, DevBuffers buf,
                       unsigned long long cond) {
  static_assert(!fmt_bf16(F), "two slices");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint32_t s_tmem;
  __shared__ int s_err;
  __shared__ int s_consumed;
  __shared__ int s_issued;  // k-blocks whose loads the producer issued (all tiles)
  __shared__ int s_last;
  __shared__ double s_scratch[2 * THREADS / 32];
  __shared__ double s_tr[DRAIN_WARPS][2];  // per drain warp: Tr X', ||X'||_F^2
  __shared__ WideCtx s_cx;

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
  const int tiles = wide_tile_count(T);
  const int my_tiles = (tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const int KB = ld / BK;
  const int NC = (KB + CHUNK - 1) / CHUNK;

  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t stg_base = base + STAGES * STAGE_BYTES;
  const uint32_t bars = stg_base + DRAIN_WARPS * STG_WORDS * 4;
  auto full_bar = [&](int s) { return bars + 8u * s; };
  auto empty_bar = [&](int s) { return bars + 8u * (STAGES + s); };
  const uint32_t chunk_full = bars + 8u * (2 * STAGES);
  const uint32_t chunk_empty = bars + 8u * (2 * STAGES + 1);
  const uint32_t acc_full = bars + 8u * (2 * STAGES + 2);
  const uint32_t acc_empty = bars + 8u * (2 * STAGES + 3);
  const uint32_t mma_done = bars + 8u * (2 * STAGES + 4);
  const uint32_t stall_bar = bars + 8u * (2 * STAGES + 5);  // nothing arrives on it

  if (threadIdx.x == 0) {
    s_err = 0;
    s_consumed = 0;
    s_issued = 0;
    for (int w = 0; w < DRAIN_WARPS; ++w) s_tr[w][0] = s_tr[w][1] = 0.0;
    const bool odd = src != 0;
    s_cx.xs0 = odd ? buf.sl[1][0] : buf.sl[0][0];
    s_cx.xs1 = odd ? buf.sl[1][1] : buf.sl[0][1];
    s_cx.out0 = odd ? buf.sl[0][0] : buf.sl[1][0];
    s_cx.out1 = odd ? buf.sl[0][1] : buf.sl[1][1];
    s_cx.out64 = odd ? buf.x64[0] : buf.x64[1];
    s_cx.wlim = wlim;
    s_cx.ld = ld;
    s_cx.T = T;
    s_cx.bit = bit;
    s_cx.want_fp64 = want_fp64 ? 1 : 0;
    s_cx.df = st->df64 != 0;
    s_cx.first_tile = (int)blockIdx.x;
    s_cx.tile_step = (int)gridDim.x;
    for (int q = 0; q < STAGES; ++q) {
      mbar_init(full_bar(q), 1);
      mbar_init(empty_bar(q), 1);
    }
    mbar_init(chunk_full, 1);
    mbar_init(chunk_empty, DRAIN_WARPS);
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, DRAIN_WARPS);
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
  // bounded wait of the drain warps: the limit is read only once it may have run out
  auto drain_wait = [&](uint32_t bar, uint32_t parity) -> bool {
    uint64_t t0 = 0;
    for (unsigned i = 1;; ++i) {
      if (mbar_try_wait(bar, parity)) return true;
      if (*err) return false;
      if ((i & 255u) == 0u) {
        const uint64_t t = global_ns();
        if (t0 == 0) {
          t0 = t;
        } else if (t - t0 > s_cx.wlim) {
          *err = 1;
          return false;
        }
      }
    }
  };

  if (warp == 0) {
    if (lane == 0) {
      int g = 0;
      bool ok = true;
      for (int j = 0; j < my_tiles && ok; ++j) {
        int I, P;
        wide_tile<BAND>((int)blockIdx.x + j * (int)gridDim.x, T, I, P);
        const int row_a = I * BM, row_b = P * BN;  // B rows past ld read as zeros
        for (int kb = 0; kb < KB; ++kb, ++g) {
          const int q = g % STAGES;
          if (!mbar_wait(empty_bar(q), ((uint32_t)(g / STAGES) & 1u) ^ 1u, err, true, wlim)) {
            ok = false;
            break;
          }
          mbar_expect_tx(full_bar(q), STAGE_BYTES);
          const uint32_t sa = base + q * STAGE_BYTES;
          const int x = kb * BK;  // 128 B multiple: TMA x alignment holds
          tma_load_2d(sa, &maps.a[src][0], x, row_a, full_bar(q));
          tma_load_2d(sa + A_BYTES, &maps.a[src][1], x, row_a, full_bar(q));
          tma_load_2d(sa + 2 * A_BYTES, &maps.b[src][0], x, row_b, full_bar(q));
          tma_load_2d(sa + 2 * A_BYTES + B_BYTES, &maps.b[src][1], x, row_b, full_bar(q));
        }
      }
      s_issued = g;
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f16(0, BM, BN);
      const uint32_t acc0 = tmem, acc1 = tmem + 256u;
      const int total = my_tiles * KB;
      int h = 0, c = 0;  // next k-block of the H and of the C group
      bool ok = true, stalled = false;
      uint64_t t0 = 0;
      unsigned spin = 0;
      while (ok && (h < total || c < total)) {
        // test of the bounded waits: after the first k-block's products, wait
        // on a barrier that nothing arrives on; it runs out after wlim
        if (stall && !stalled && h >= 1 && c >= 1) {
          stalled = true;
          if (!mbar_wait(stall_bar, 0u, err, true, wlim)) {
            ok = false;
            break;
          }
        }
        bool did = false;
        const bool c_first = c <= h;  // the group that lags goes first: it frees a stage
        for (int pass = 0; pass < 2 && !did; ++pass) {
          if ((pass == 0) == c_first) {
            if (c < total && c - h < STAGES) {
              const int kb = c % KB;
              bool ready = mbar_test_wait(full_bar(c % STAGES), (uint32_t)(c / STAGES) & 1u);
              // a tile's first C products overwrite acc1: the previous epilogue is done
              if (ready && kb == 0)
                ready = mbar_test_wait(acc_empty, ((uint32_t)(c / KB) & 1u) ^ 1u);
              if (ready) {
                tc_fence_after();
                const uint32_t sa = base + (c % STAGES) * STAGE_BYTES;
                const uint64_t a0 = smem_desc_sw128(sa), a1 = smem_desc_sw128(sa + A_BYTES);
                const uint64_t b0 = smem_desc_sw128(sa + 2 * A_BYTES);
                const uint64_t b1 = smem_desc_sw128(sa + 2 * A_BYTES + B_BYTES);
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk) {
                  const uint64_t adv = (uint64_t)(kk * 32) >> 4;  // 32 B per K = 16 step
                  mma_f16(acc1, a0 + adv, b1 + adv, idesc, (kb == 0 && kk == 0) ? 0u : 1u);
                  mma_f16(acc1, a1 + adv, b0 + adv, idesc, 1u);
                }
                if (h > c) {  // both groups of this k-block are issued
                  mma_commit(empty_bar(c % STAGES));
                  if (kb == KB - 1) mma_commit(acc_full);
                }
                ++c;
                did = true;
              }
            }
          } else {
            if (h < total && h - c < STAGES) {
              const int kb = h % KB;
              const bool chunk_first = (kb % CHUNK) == 0;
              const bool chunk_last = (kb % CHUNK) == CHUNK - 1 || kb == KB - 1;
              const int gc = (h / KB) * NC + kb / CHUNK;  // chunk index over all tiles
              bool ready = mbar_test_wait(full_bar(h % STAGES), (uint32_t)(h / STAGES) & 1u);
              // a chunk's first H products overwrite acc0: the previous chunk is drained
              if (ready && chunk_first)
                ready = mbar_test_wait(chunk_empty, ((uint32_t)gc & 1u) ^ 1u);
              if (ready) {
                tc_fence_after();
                const uint32_t sa = base + (h % STAGES) * STAGE_BYTES;
                const uint64_t a0 = smem_desc_sw128(sa);
                const uint64_t b0 = smem_desc_sw128(sa + 2 * A_BYTES);
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk) {
                  const uint64_t adv = (uint64_t)(kk * 32) >> 4;
                  mma_f16(acc0, a0 + adv, b0 + adv, idesc, (chunk_first && kk == 0) ? 0u : 1u);
                }
                if (chunk_last) mma_commit(chunk_full);
                if (c > h) {
                  mma_commit(empty_bar(h % STAGES));
                  if (kb == KB - 1) mma_commit(acc_full);
                }
                ++h;
                did = true;
              }
            }
          }
        }
        if (did) {
          s_consumed = h < c ? h : c;
          t0 = 0;
          spin = 0;
          continue;
        }
        if (*err) {
          ok = false;
          break;
        }
        if ((++spin & 255u) == 0u) {  // no group could go: bounded like every other wait
          const uint64_t t = global_ns();
          if (t0 == 0) {
            t0 = t;
          } else if (t - t0 > wlim) {
            *err = 1;
            ok = false;
          }
        }
      }
      mma_commit(mma_done);  // every MMA issued so far is complete
    }
    __syncwarp();
  }

  // ---- drain + epilogue warps. Registers are the constraint here: 64 FP32 sums
  // per thread live across every chunk, so the loop carries little else (one
  // flat loop over chunks, a slim bounded wait, the epilogue's pointers and
  // flags re-read from shared memory when a tile ends).
  if (warp >= DRAIN_WARP0) {
    const int dw = warp - DRAIN_WARP0;
    const uint32_t lane_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((dw >> 2) * DCOLS);
    const int nchunks = my_tiles * NC;
    float sum0[DCOLS];
#pragma unroll
    for (int i = 0; i < DCOLS; ++i) sum0[i] = 0.0f;
    int left = NC, j = 0;  // chunks left in tile j
    for (int g = 0; g < nchunks; ++g) {
      if (!drain_wait(chunk_full, (uint32_t)g & 1u)) break;
      tc_fence_after();
#pragma unroll
      for (int q = 0; q < DCOLS / 8; ++q) {
        uint32_t u[8];
        tmem_ld8(lane_addr + (uint32_t)(q * 8), u);
        tmem_ld_wait();
        if (q == DCOLS / 8 - 1) {  // the chunk buffer is free again
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive_cta(chunk_empty);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) sum0[q * 8 + i] += __uint_as_float(u[i]);
      }
      if (--left != 0) continue;
      // ---- the tile's last chunk: S = w0 sum0 + w1 acc1 over acc1, then the epilogue
      left = NC;
      if (!drain_wait(acc_full, (uint32_t)j & 1u)) break;
      tc_fence_after();
#pragma unroll
      for (int q = 0; q < DCOLS / 8; ++q) {
        uint32_t u[8];
        tmem_ld8(lane_addr + 256u + (uint32_t)(q * 8), u);
        tmem_ld_wait();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          u[i] = __float_as_uint(sum0[q * 8 + i] * SliceWeights<F>::w0 +
                                 __uint_as_float(u[i]) * SliceWeights<F>::w1);
        }
        tmem_st8(lane_addr + 256u + (uint32_t)(q * 8), u);
      }
      tmem_st_wait();
      wide_epilogue<F>(s_cx, j, dw, lane, lane_addr + 256u,
                       reinterpret_cast<uint32_t*>(smem_raw + (stg_base - smem_u32(smem_raw))) +
                           dw * STG_WORDS,
                       s_tr[dw]);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cta(acc_empty);  // acc1 may be overwritten
      ++j;
#pragma unroll
      for (int i = 0; i < DCOLS; ++i) sum0[i] = 0.0f;
    }
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
      for (int g = s_consumed; g < s_issued; ++g)
        mbar_wait(full_bar(g % STAGES), (uint32_t)(g / STAGES) & 1u, err, false,
                  kWaitLimitNs / 10);
    }
    __syncthreads();
  }
  if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
  if (*err && threadIdx.x == 0) {
    st->status = PROGRESS_ETIMEOUT;
    st->done = 1;
  }

  if (threadIdx.x == 0) {
    double tr = 0.0, fr = 0.0;
    for (int w = 0; w < DRAIN_WARPS; ++w) {
      tr += s_tr[w][0];
      fr += s_tr[w][1];
    }
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
      st->iter = __ldcg(&st->iter) + 1;  // (only this CTA writes it, after every CTA read it)
      st->phase_iters[kPhaseSplit] += 1;
      st->x_fp64_valid = s_cx.want_fp64;
      st->x_slices_valid = 1;
      decide(st);
    }
    if (st->done && cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, 0u);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
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

bool encode_wide_maps(const DevBuffers& b, int ld, WideMaps* maps) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
  if (!enc) return false;
  memset(maps, 0, sizeof *maps);
  for (int k = 0; k < 2; ++k) {
    for (int j = 0; j < 2; ++j) {
      if (!b.sl[k][j]) return false;
      cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)ld};
      cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
      cuuint32_t estr[2] = {1, 1};
      cuuint32_t box_a[2] = {(cuuint32_t)BK, (cuuint32_t)BM};
      cuuint32_t box_b[2] = {(cuuint32_t)BK, (cuuint32_t)BN};
      if (enc(&maps->a[k][j], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, (void*)b.sl[k][j], dims,
              strides, box_a, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
      if (enc(&maps->b[k][j], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, (void*)b.sl[k][j], dims,
              strides, box_b, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    }
  }
  return true;
}

}  // namespace

cudaError_t launch_square_wide(const DevBuffers& b, const SolveParams& p,
                               unsigned long long cond_handle, cudaStream_t s) {
  const int ld = p.ld;
  if (ld % BM || ld <= 0) return cudaErrorInvalidValue;
  if (p.slice_fmt != kFP16x2 && p.slice_fmt != kFP16x2F) return cudaErrorInvalidValue;
  WideMaps maps;
  if (!encode_wide_maps(b, ld, &maps)) return cudaErrorInvalidValue;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int tiles = wide_tile_count(ld / BM);
  const int grid = nsm < tiles ? nsm : tiles;  // one CTA per SM, never more than tiles
  if (grid > b.max_partials) return cudaErrorInvalidValue;
  switch (p.slice_fmt) {
#define SP2_WIDE(F)                                                                        \
  case F:                                                                                  \
    e = cudaFuncSetAttribute(square_wide_kernel<F>,                                        \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);           \
    if (e != cudaSuccess) return e;                                                        \
    square_wide_kernel<F><<<grid, THREADS, SMEM, s>>>(maps, b, cond_handle);               \
    break;
    SP2_WIDE(kFP16x2)
    SP2_WIDE(kFP16x2F)
#undef SP2_WIDE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace sp2
