// Chebyshev Fermi-operator expansion (§IV.B) in the Paterson-Stockmeyer form
// (Eq. 7) on the sm_103a tcgen05 tensor cores.
//
// D = f(H) = sum_{n<=L} c_n T_n(Ht) with Ht = (H - a I) / b mapped into
// [-1, 1] by the Gershgorin bounds, f the Fermi-Dirac occupation at a given
// chemical potential and inverse temperature, and L + 1 = k m:
//
//   D = S_0 + T_k (S_1 + T_k (... + T_k S_{m-1})),  S_j = sum_{i<k} d_ij T_i.
//
// The host computes c_n (interpolation at 2 (L + 1) Chebyshev-Gauss nodes)
// and d_ij (division of the series by T_k with T_n = 2 T_k T_{n-k} -
// T_{|2k-n|}, from the product rule of Eq. 8) in FP64. The device then runs:
//
//   cheb_t1_kernel       T_1 = Ht as operand slices
//   cheb_product_kernel  C = alpha (A B) + beta E + gamma I for a LIST of
//                        independent products in one launch (grid = products
//                        x upper-triangle tiles): T_2..T_k level by level,
//                        T_n = 2 T_a T_b - T_{a-b} with a = ceil(n/2),
//                        b = floor(n/2), so every T_n of (2^(l-1), 2^l]
//                        depends only on lower levels (Eqs. 10-11: the paper
//                        runs them on concurrent streams; here they share one
//                        launch). Then the m - 1 nested products
//                        P_j = S_j + T_k P_{j+1}; the last writes D in FP64.
//   cheb_sum_staged_kernel / cheb_sum_fast_kernel
//                        every S_j in one pass over T_1..T_{k-1} (the sums are
//                        independent, Eq. 9), coefficients in the constant bank; the
//                        staged pass (k <= 16) brings the T inputs by 3D TMA boxes
//
// Every matrix is a polynomial in Ht, so all of them are symmetric and
// commute: a product tile (I, J), I <= J, reads the row panels I of A and J
// of B (both K-major) and writes C at (r, c) and at the mirror (c, r).
//
// Operands are floating-point slices (FP16x2: hi, lo; BF16x3: hi, mid, lo;
// see sp2_slices.cuh) of value / s, with one power-of-two scale s per matrix
// chosen on the host so that the spectral norm of value / s is at most 1
// (every entry of a stored matrix is then at most 1, far inside FP16's range):
// T_n needs s = 1 (|T_n| <= 1 on the spectrum); S_j takes s >= sum_i |d_ij| and
// P_j s >= sum_{j' >= j} sum_i |d_ij'|.
//
// The product kernel has the pipeline of the SP2 split-precision kernel
// (TMA ring, one MMA-issuing thread, FP32 accumulators in tensor memory,
// eight drain warps) with 3D tensor maps over a stack of matrices (the z
// coordinate picks the matrix). The leading hi*hi group is drained from
// tensor memory every k-block (64 k) and summed with round-to-nearest FP32
// adds: the tensor core's own accumulation truncates, and on the diagonal of a
// square whose diagonal entries are near +-1 (T_2, T_4, ...) that became a
// measured bias of -1.9e-6 per product with 256-k chunks, -5.7e-7 with 64-k
// chunks. (Fixed-point slices, whose integer hi*hi sums would be exact in an
// exact FP32 accumulator, measured worse still: -1.1e-5 per square.) Every
// mbarrier wait is bounded; a wait that runs out sets an error word that the
// host reads and that later launches check before doing any work.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "progress_sp2.h"
#include "sp2_launch.h"
#include "sp2_slices.cuh"
#include "sp2_tc.cuh"

namespace sp2 {
namespace {

using namespace tc;

constexpr int BM = 128;
constexpr int BN = 128;
constexpr int BK = 64;                    // 16-bit elements = 128 B rows
constexpr int TILE_BYTES = BM * BK * 2;   // one 128 x 64 slice box (16 KB)
constexpr int THREADS = 384;              // warp 0 TMA, warp 1 MMA, warps 4..11 drain + epilogue
constexpr int DRAIN_WARPS = 8;
constexpr int DRAIN_WARP0 = 4;
constexpr int DCOLS = BN / 2;             // columns per drain thread
constexpr int CHUNK = 1;                  // k-blocks per leading-group chunk
constexpr int TMEM_COLS = 512;
constexpr int MAX_K = 64;                 // T_k order limit
constexpr int MAX_M = 64;                 // nested-product count limit
constexpr int EW_THREADS = 256;
constexpr int EW_BLOCKS = 152 * 8;

template <int F>
struct Cfg {
  static constexpr int NS = fmt_slices(F);
  static constexpr int STAGE_BYTES = 2 * NS * TILE_BYTES;
  static constexpr int STAGES = fmt_bf16(F) ? 2 : 3;
  static constexpr int NBUF = fmt_bf16(F) ? 2 : 3;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 256;
};
// the epilogue stages its (r, c) stores in the idle operand ring
static_assert(DRAIN_WARPS * 32 * 33 * 4 + DRAIN_WARPS * 32 * 34 * 2 <= 2 * 2 * 2 * TILE_BYTES,
              "staging must fit in the smallest ring");

// One product C = alpha * sab * (A B) + beta * se * E + gamma * I, stored as
// slices of C * inv_sc (slot c >= 0) or as FP64 D (c < 0). A, B, E, C are
// stack slots; e < 0 means no E term.
struct Prod {
  int a, b, e, c;
  float alpha, sab, beta, se, gamma, inv_sc;
};

struct Maps {
  CUtensorMap m[3];  // one per slice: the whole stack, box 64 x 128 x 1
};

struct Pool {
  uint16_t* s[3];    // slice stacks: slot z, element (r, c) at z ld^2 + r ld + c
};

__device__ __forceinline__ size_t slot_off(int slot, int ld) {
  return (size_t)slot * (size_t)ld * (size_t)ld;
}

template <int F>
__global__ void __launch_bounds__(THREADS, 1)
    cheb_product_kernel(const __grid_constant__ Maps maps, Pool pool, const Prod* __restrict__ prods,
                        int tiles, int ld, double* __restrict__ D, int64_t n, int* __restrict__ gerr) {
  using C = Cfg<F>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint32_t s_tmem;
  __shared__ int s_err;
  __shared__ int s_consumed;
  __shared__ int s_skip;

  // an earlier launch gave up: the whole CTA leaves before any barrier
  if (threadIdx.x == 0) s_skip = *(volatile int*)gerr;
  __syncthreads();
  if (s_skip) return;
  const int p = blockIdx.x / tiles;
  const int tile = blockIdx.x - p * tiles;
  const Prod pr = prods[p];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int T = ld / BM;
  int I, J;
  tri_tile(tile, T, I, J);
  const int row_a = I * BM, row_b = J * BN;

  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t bars = base + C::STAGES * C::STAGE_BYTES;
  auto full_bar = [&](int s) { return bars + 8u * s; };
  auto empty_bar = [&](int s) { return bars + 8u * (C::STAGES + s); };
  const uint32_t accum_bar = bars + 8u * (2 * C::STAGES);
  const uint32_t chunk_full = bars + 8u * (2 * C::STAGES + 1);
  const uint32_t chunk_empty = bars + 8u * (2 * C::STAGES + 1 + C::NBUF);

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

  const int KB = ld / BK;
  const int NC = (KB + CHUNK - 1) / CHUNK;
  int issued = 0;
  if (warp == 0) {
    if (lane == 0) {
      // TMA producer: row panel I of A and row panel J of B, every slice
      for (int kb = 0; kb < KB; ++kb, ++issued) {
        const int s = kb % C::STAGES;
        const uint32_t ph = (uint32_t)(kb / C::STAGES) & 1u;
        if (!mbar_wait(empty_bar(s), ph ^ 1u, err)) break;
        mbar_expect_tx(full_bar(s), C::STAGE_BYTES);
        const uint32_t sa = base + s * C::STAGE_BYTES;
#pragma unroll
        for (int j = 0; j < C::NS; ++j) {
          tma_load_3d(sa + j * TILE_BYTES, &maps.m[j], kb * BK, row_a, pr.a, full_bar(s));
          tma_load_3d(sa + (C::NS + j) * TILE_BYTES, &maps.m[j], kb * BK, row_b, pr.b,
                      full_bar(s));
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: acc0 (chunked) += hi hi^T, acc1 += hi lo^T + lo hi^T (x2) or
      // hi mid^T + mid hi^T (x3), acc2 += hi lo^T + lo hi^T + mid mid^T (x3)
      constexpr uint32_t idesc = idesc_f16(fmt_bf16(F) ? 1 : 0, BM, BN);
      const uint32_t acc1 = tmem + 128u * C::NBUF, acc2 = acc1 + 128u;
      bool ok = true;
      for (int kb = 0; kb < KB && ok; ++kb) {
        const int c = kb / CHUNK, cb = c % C::NBUF;
        const bool chunk_first = (kb % CHUNK) == 0;
        const bool chunk_last = (kb % CHUNK) == CHUNK - 1 || kb == KB - 1;
        const uint32_t acc0 = tmem + 128u * cb;
        if (chunk_first) {
          if (!mbar_wait(chunk_empty + 8u * cb, ((uint32_t)(c / C::NBUF) & 1u) ^ 1u, err)) {
            ok = false;
            break;
          }
          tc_fence_after();
        }
        const int s = kb % C::STAGES;
        const uint32_t ph = (uint32_t)(kb / C::STAGES) & 1u;
        if (!mbar_wait(full_bar(s), ph, err)) {
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
          const uint64_t adv = (uint64_t)(kk * 32) >> 4;
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
        mma_commit(empty_bar(s));
        if (chunk_last) mma_commit(chunk_full + 8u * cb);
        s_consumed = kb + 1;
      }
      mma_commit(accum_bar);
    }
    __syncwarp();
  }

  // ---- drain warps: lane = tile row, DCOLS columns per thread
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
      if (!mbar_wait(chunk_full + 8u * cb, (uint32_t)(c / C::NBUF) & 1u, err)) break;
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
      for (int j = 0; j < DCOLS; ++j) sum0[j] += v[j];
    }
  }
  const bool ok = mbar_wait(accum_bar, 0u, err, false);
  tc_fence_after();
  if (drain && ok && *err == 0) {
    using W = SliceWeights<F>;
    const int r = row_a + row;
    const float ab = pr.alpha * pr.sab;
    const float be = pr.beta * pr.se;
    const bool has_e = pr.e >= 0;
    const bool to_d = pr.c < 0;
    const size_t eoff = has_e ? slot_off(pr.e, ld) : 0;
    const size_t coff = to_d ? 0 : slot_off(pr.c, ld);
    const uint16_t* e0 = pool.s[0] + eoff;
    const uint16_t* e1 = pool.s[1] + eoff;
    const uint16_t* e2 = pool.s[2] + eoff;
    uint16_t* const o0 = pool.s[0] + coff;
    uint16_t* const o1 = pool.s[1] + coff;
    uint16_t* const o2 = pool.s[2] + coff;
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
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int cs = c0 + hh * 16;
        // E is symmetric: read it at the mirror (c, r), coalesced across lanes,
        // before waiting on tensor memory
        uint32_t m01[16], m2[16];
        if (has_e) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const size_t m = (size_t)(cs + j) * ld + r;
            m01[j] = (uint32_t)e0[m] | ((uint32_t)e1[m] << 16);
            m2[j] = fmt_bf16(F) ? (uint32_t)e2[m] : 0u;
          }
        }
        uint32_t u1[16], u2[16];
        tmem_ld16(lane_addr + 128u * C::NBUF + col + hh * 16, u1);
        if (fmt_bf16(F)) tmem_ld16(lane_addr + 128u * (C::NBUF + 1) + col + hh * 16, u2);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int jj = hh * 16 + j;
          const int c = cs + j;
          float s = sum0[ch * 32 + jj] * W::w0 + __uint_as_float(u1[j]) * W::w1;
          if (fmt_bf16(F)) s += __uint_as_float(u2[j]) * W::w2;
          float x = ab * s;
          if (has_e)
            x += be * join_value<F>((uint16_t)(m01[j] & 0xffffu), (uint16_t)(m01[j] >> 16),
                                    (uint16_t)m2[j]);
          if (r == c) x += pr.gamma;
          if (to_d) {
            if (r <= c && c < n) {  // (r < n follows)
              D[(size_t)r * n + c] = (double)x;
              if (r != c) D[(size_t)c * n + r] = (double)x;
            }
          } else {
            uint16_t a, b2, c2;
            split_value_f<F>(x * pr.inv_sc, a, b2, c2);
            stA[lane * 33 + jj] = (uint32_t)a | ((uint32_t)b2 << 16);
            if (fmt_bf16(F)) stB[lane * 34 + jj] = c2;
            if (r < c) {
              const size_t m = (size_t)c * ld + r;  // mirror: consecutive lanes, consecutive r
              o0[m] = a;
              o1[m] = b2;
              if (fmt_bf16(F)) o2[m] = c2;
            }
          }
        }
      }
      if (!to_d) {
        // (r, c) slices: 32 rows of 32 columns back out, one row per store
        __syncwarp();
        const int cc = c0 + lane;
#pragma unroll 4
        for (int i = 0; i < 32; ++i) {
          if (rb + i <= cc) {
            const uint32_t v = stA[i * 33 + lane];
            const size_t d = (size_t)(rb + i) * ld + cc;
            o0[d] = (uint16_t)(v & 0xffffu);
            o1[d] = (uint16_t)(v >> 16);
            if (fmt_bf16(F)) o2[d] = stB[i * 34 + lane];
          }
        }
        __syncwarp();
      }
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
  if (*err && threadIdx.x == 0) atomicExch(gerr, (int)PROGRESS_ETIMEOUT);
}

// T_1 = (H - a I) / b as slices in slot 0, zero in the padding (r or c >= n).
template <int F>
__global__ void __launch_bounds__(EW_THREADS)
    cheb_t1_kernel(const double* __restrict__ H, int64_t n, int ld, double a, double inv_b,
                   Pool pool) {
  const size_t total = (size_t)ld * ld;
  for (size_t e = (size_t)blockIdx.x * EW_THREADS + threadIdx.x; e < total;
       e += (size_t)gridDim.x * EW_THREADS) {
    const int64_t r = (int64_t)(e / ld), c = (int64_t)(e - (size_t)r * ld);
    double x = 0.0;
    if (r < n && c < n) x = (H[r * n + c] - (r == c ? a : 0.0)) * inv_b;
    uint16_t s0, s1, s2;
    split_value<F>(x, s0, s1, s2);
    pool.s[0][e] = s0;
    pool.s[1][e] = s1;
    if (fmt_bf16(F)) pool.s[2][e] = s2;
  }
}

// S_j = sum_{i<k} d_ij T_i for every j (T_0 = I, T_i in slot i - 1), stored as
// slices of S_j / s_j in slot k + j; with m == 1, S_0 goes to D in FP64.
// The same pass with the coefficients as kernel parameters: a zero-padded
// KB x MB table in the constant bank, so every multiply-add of the fully
// unrolled loops takes its coefficient as an immediate constant operand. Table
// sizes 16 x 16 (two neighbouring elements per thread, 32-bit slice loads and
// stores), 32 x 32 and 64 x 64 (one element per thread; up to 16.6 KB of
// kernel parameters).
template <int KB, int MB>
struct SumTable {
  float d[KB * MB];  // d_ij at i MB + j, zero outside i < k, j < m
  float inv_s[MB];
};

template <int F, int KB, int MB, int EPT>
// the 16 x 16 table runs three CTAs per SM (at most 85 registers): this pass is
// bound by memory, and one CTA per SM kept too few loads in flight
__global__ void __launch_bounds__(EW_THREADS, KB == 16 ? 3 : 1)
    cheb_sum_fast_kernel(Pool pool, int ld, int k, int m,
                         const __grid_constant__ SumTable<KB, MB> tab, double* __restrict__ D,
                         int64_t n, const int* __restrict__ gerr) {
  static_assert(EPT == 1 || EPT == 2, "one or two elements per thread");
  if (*(volatile const int*)gerr) return;  // no barrier below: a per-thread exit is safe
  const size_t area = (size_t)ld * ld;
  const size_t groups = area / EPT;  // ld is even: a pair shares a row
  for (size_t q = (size_t)blockIdx.x * EW_THREADS + threadIdx.x; q < groups;
       q += (size_t)gridDim.x * EW_THREADS) {
    const size_t e = EPT * q;
    const int64_t r = (int64_t)(e / ld), c = (int64_t)(e - (size_t)r * ld);
    float t[EPT][KB];
#pragma unroll
    for (int u = 0; u < EPT; ++u) t[u][0] = (r == c + u) ? 1.0f : 0.0f;
#pragma unroll
    for (int i = 1; i < KB; ++i) {
#pragma unroll
      for (int u = 0; u < EPT; ++u) t[u][i] = 0.0f;
      if (i < k) {
        const size_t o = (size_t)(i - 1) * area + e;
        if (EPT == 2) {
          const uint32_t h = *reinterpret_cast<const uint32_t*>(pool.s[0] + o);
          const uint32_t l = *reinterpret_cast<const uint32_t*>(pool.s[1] + o);
          const uint32_t w =
              fmt_bf16(F) ? *reinterpret_cast<const uint32_t*>(pool.s[2] + o) : 0u;
          t[0][i] = join_value<F>((uint16_t)(h & 0xffffu), (uint16_t)(l & 0xffffu),
                                  (uint16_t)(w & 0xffffu));
          t[EPT - 1][i] = join_value<F>((uint16_t)(h >> 16), (uint16_t)(l >> 16),
                                        (uint16_t)(w >> 16));
        } else {
          t[0][i] = join_value<F>(pool.s[0][o], pool.s[1][o],
                                  fmt_bf16(F) ? pool.s[2][o] : (uint16_t)0);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < MB; ++j) {
      if (j < m) {
        float acc[EPT];
#pragma unroll
        for (int u = 0; u < EPT; ++u) acc[u] = 0.0f;
#pragma unroll
        for (int i = 0; i < KB; ++i) {
#pragma unroll
          for (int u = 0; u < EPT; ++u) acc[u] += tab.d[i * MB + j] * t[u][i];
        }
        if (m == 1) {
#pragma unroll
          for (int u = 0; u < EPT; ++u)
            if (r < n && c + u < n) D[r * n + c + u] = (double)acc[u];
        } else {
          uint16_t x[EPT][3];
#pragma unroll
          for (int u = 0; u < EPT; ++u)
            split_value_f<F>(acc[u] * tab.inv_s[j], x[u][0], x[u][1], x[u][2]);
          const size_t o = (size_t)(k + j) * area + e;
          if (EPT == 2) {
#pragma unroll
            for (int sl = 0; sl < fmt_slices(F); ++sl)
              *reinterpret_cast<uint32_t*>(pool.s[sl] + o) =
                  (uint32_t)x[0][sl] | ((uint32_t)x[EPT - 1][sl] << 16);
          } else {
#pragma unroll
            for (int sl = 0; sl < fmt_slices(F); ++sl) pool.s[sl][o] = x[0][sl];
          }
        }
      }
    }
  }
}

template <int F, int KB, int MB, int EPT>
cudaError_t launch_sum_fast(const Pool& pool, int ld, int k, int m, const std::vector<float>& d,
                            const std::vector<float>& inv_s, double* D, int64_t n,
                            const int* err, cudaStream_t s) {
  SumTable<KB, MB> tab;
  memset(&tab, 0, sizeof tab);
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < m; ++j) tab.d[i * MB + j] = d[(size_t)i * m + j];
  for (int j = 0; j < m; ++j) tab.inv_s[j] = inv_s[j];
  const unsigned blocks = (unsigned)std::min<size_t>(
      EW_BLOCKS, ((size_t)ld * ld / EPT + EW_THREADS - 1) / EW_THREADS);
  cheb_sum_fast_kernel<F, KB, MB, EPT><<<blocks, EW_THREADS, 0, s>>>(pool, ld, k, m, tab, D, n,
                                                                     err);
  return cudaGetLastError();
}

// The 16 x 16 pass with its T inputs staged through shared memory. Measured on
// cheb_sum_fast_kernel at N = 4096: its 30 slice streams of 4-byte loads per
// element ran at about 1.1 TB/s (the loads alone took as long as the whole pass,
// 0.95 ms; the stores alone 0.29 ms). Here one 3D TMA box per slice brings
// T_1 .. T_{k-1} of a 4 x 128 chunk (k - 1 planes of 1 KB each) in long
// sequential requests, SG_STAGES chunks ahead, and the threads compute from
// shared memory with the same arithmetic and the same stores as the fast pass.
// Persistent: CTA b takes chunks b, b + grid, ...; every wait is bounded.
constexpr int SG_ROWS = 4;
constexpr int SG_COLS = 128;
constexpr int SG_STAGES = 3;
static_assert(SG_ROWS * SG_COLS == 2 * EW_THREADS, "two elements per thread");

struct SumMaps {
  CUtensorMap m[3];  // per slice: the slot stack, boxes of SG_COLS x SG_ROWS x (k - 1)
};

template <int F>
__global__ void __launch_bounds__(EW_THREADS, 2)
    cheb_sum_staged_kernel(const __grid_constant__ SumMaps maps, Pool pool, int ld, int k,
                           int m, const __grid_constant__ SumTable<16, 16> tab,
                           double* __restrict__ D, int64_t n, int* __restrict__ gerr) {
  constexpr int NS = fmt_slices(F);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t s_full[SG_STAGES];
  __shared__ int s_err;
  __shared__ int s_skip;
  if (threadIdx.x == 0) s_skip = *(volatile const int*)gerr;
  __syncthreads();
  if (s_skip) return;  // an earlier launch of this solve failed (uniform)

  const int nz = k - 1;  // T_1 .. T_{k-1} sit in slots 0 .. k - 2
  constexpr uint32_t kPlane = SG_ROWS * SG_COLS * 2;  // bytes of one z plane of one slice
  const uint32_t stage_bytes = (uint32_t)(NS * nz) * kPlane;
  const int cpr = ld / SG_COLS;  // chunks per band of SG_ROWS rows
  const int chunks = (ld / SG_ROWS) * cpr;
  const int my = (chunks - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  auto full = [&](int q) { return smem_u32(&s_full[q]); };
  if (threadIdx.x == 0) {
    s_err = 0;
    for (int q = 0; q < SG_STAGES; ++q) mbar_init(full(q), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  }
  __syncthreads();
  volatile int* err = &s_err;
  // thread 0: the loads of this CTA's chunk `it` into stage it % SG_STAGES
  auto issue = [&](int it) {
    const int g = (int)blockIdx.x + it * (int)gridDim.x;
    const int r0 = (g / cpr) * SG_ROWS, c0 = (g % cpr) * SG_COLS;  // c0: 256 B multiple
    const int q = it % SG_STAGES;
    const uint32_t dst = base + (uint32_t)q * stage_bytes;
    mbar_expect_tx(full(q), stage_bytes);
#pragma unroll
    for (int sl = 0; sl < NS; ++sl)
      tma_load_3d(dst + (uint32_t)(sl * nz) * kPlane, &maps.m[sl], c0, r0, 0, full(q));
  };
  int issued = 0;
  if (threadIdx.x == 0)
    for (; issued < SG_STAGES && issued < my; ++issued) issue(issued);

  const int row = threadIdx.x / (SG_COLS / 2), col = 2 * (threadIdx.x % (SG_COLS / 2));
  int it = 0;
  for (; it < my; ++it) {
    const int q = it % SG_STAGES;
    const bool fail = !mbar_wait(full(q), (uint32_t)(it / SG_STAGES) & 1u, err);
    if (__syncthreads_or(fail)) break;  // uniform
    const uint16_t* sb = reinterpret_cast<const uint16_t*>(
        smem_raw + (base + (uint32_t)q * stage_bytes - smem_u32(smem_raw)));
    const int g = (int)blockIdx.x + it * (int)gridDim.x;
    const int64_t r = (int64_t)(g / cpr) * SG_ROWS + row;
    const int64_t c = (int64_t)(g % cpr) * SG_COLS + col;
    const size_t e = (size_t)r * ld + (size_t)c;
    const size_t area = (size_t)ld * ld;
    float t[2][16];
#pragma unroll
    for (int u = 0; u < 2; ++u) t[u][0] = (r == c + u) ? 1.0f : 0.0f;
#pragma unroll
    for (int i = 1; i < 16; ++i) {
      t[0][i] = t[1][i] = 0.0f;
      if (i < k) {
        const int off = ((i - 1) * SG_ROWS + row) * SG_COLS + col;  // elements in a slice box
        const int sls = nz * SG_ROWS * SG_COLS;                     // elements per slice box
        const uint32_t h = *reinterpret_cast<const uint32_t*>(sb + off);
        const uint32_t l = *reinterpret_cast<const uint32_t*>(sb + sls + off);
        const uint32_t w =
            fmt_bf16(F) ? *reinterpret_cast<const uint32_t*>(sb + 2 * sls + off) : 0u;
        t[0][i] = join_value<F>((uint16_t)(h & 0xffffu), (uint16_t)(l & 0xffffu),
                                (uint16_t)(w & 0xffffu));
        t[1][i] = join_value<F>((uint16_t)(h >> 16), (uint16_t)(l >> 16), (uint16_t)(w >> 16));
      }
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (j < m) {
        float acc[2] = {0.0f, 0.0f};
#pragma unroll
        for (int i = 0; i < 16; ++i) {
#pragma unroll
          for (int u = 0; u < 2; ++u) acc[u] += tab.d[i * 16 + j] * t[u][i];
        }
        if (m == 1) {
#pragma unroll
          for (int u = 0; u < 2; ++u)
            if (r < n && c + u < n) D[r * n + c + u] = (double)acc[u];
        } else {
          uint16_t x[2][3];
#pragma unroll
          for (int u = 0; u < 2; ++u)
            split_value_f<F>(acc[u] * tab.inv_s[j], x[u][0], x[u][1], x[u][2]);
          const size_t o = (size_t)(k + j) * area + e;
#pragma unroll
          for (int sl = 0; sl < NS; ++sl)
            *reinterpret_cast<uint32_t*>(pool.s[sl] + o) =
                (uint32_t)x[0][sl] | ((uint32_t)x[1][sl] << 16);
        }
      }
    }
    __syncthreads();  // every thread has read stage q: it may be refilled
    if (threadIdx.x == 0 && issued < my) {
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      issue(issued++);
    }
  }
  if (*err) {
    // failure path: let the copies still in flight land before the CTA exits
    if (threadIdx.x == 0) {
      for (int g = it; g < issued; ++g)
        mbar_wait(full(g % SG_STAGES), (uint32_t)(g / SG_STAGES) & 1u, err, false,
                  kWaitLimitNs / 10);
      atomicExch(gerr, (int)PROGRESS_ETIMEOUT);
    }
  }
}

__global__ void cheb_trace_kernel(const double* __restrict__ D, int64_t n, double* out) {
  __shared__ double s[EW_THREADS / 32];
  double v = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += EW_THREADS) v += D[i * n + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < EW_THREADS / 32; ++w) t += s[w];
    *out = t;
  }
}

// ---------------------------------------------------------------- host side

// Fermi-Dirac occupation (§III) as (1 - tanh(beta (e - mu) / 2)) / 2.
double fermi(double e, double mu, double beta) {
  return 0.5 * (1.0 - tanh(0.5 * beta * (e - mu)));
}

// Coefficients c_0..c_L of the interpolant of f(b x + a) at the M = 2 (L + 1)
// Chebyshev-Gauss nodes x_j = cos(pi (j + 1/2) / M):
// c_q = (2 - [q = 0]) / M sum_j f(b x_j + a) T_q(x_j), with T_q(x_j) from the
// three-term recursion (O(M L) multiply-adds instead of M L cosines).
std::vector<double> coefficients(int L, double a, double b, double mu, double beta) {
  const int M = 2 * (L + 1);
  std::vector<double> c(L + 1, 0.0);
  for (int j = 0; j < M; ++j) {
    const double x = cos(M_PI * (j + 0.5) / M);
    const double g = fermi(b * x + a, mu, beta);
    double t0 = 1.0, t1 = x;
    c[0] += g;
    if (L >= 1) c[1] += g * x;
    for (int q = 2; q <= L; ++q) {
      const double t2 = 2.0 * x * t1 - t0;
      c[q] += g * t2;
      t0 = t1;
      t1 = t2;
    }
  }
  for (int q = 0; q <= L; ++q) c[q] *= (q ? 2.0 : 1.0) / M;
  return c;
}

// d[i][j] (k x m, row-major): column j = remainder of the j-th division of the
// series by T_k, using T_n = 2 T_k T_{n-k} - T_{|2k-n|} (and T_k = T_k T_0).
std::vector<double> ps_split(std::vector<double> series, int k, int m) {
  std::vector<double> d((size_t)k * m, 0.0);
  for (int j = 0; j < m; ++j) {
    const int deg = (int)series.size() - 1;
    if (j == m - 1) {
      for (int i = 0; i < k && i <= deg; ++i) d[(size_t)i * m + j] = series[i];
      break;
    }
    std::vector<double> quot(std::max(deg - k + 1, 1), 0.0);
    for (int q = deg; q >= k; --q) {
      const double v = series[q];
      series[q] = 0.0;
      if (q == k) {
        quot[0] += v;
      } else {
        quot[q - k] += 2.0 * v;
        series[std::abs(2 * k - q)] -= v;
      }
    }
    for (int i = 0; i < k && i <= deg; ++i) d[(size_t)i * m + j] = series[i];
    series.swap(quot);
  }
  return d;
}

double pow2_at_least(double v) {
  if (!(v > 1.0)) return 1.0;
  return ldexp(1.0, (int)ceil(log2(v)));
}

struct ChebWs {
  uint16_t* pool = nullptr;  // NS slice stacks, contiguous
  size_t pool_cap = 0;       // elements
  Prod* prods = nullptr;
  size_t prods_cap = 0;
  int* err = nullptr;
  double* scal = nullptr;    // [0..1] bounds, [2] trace
  int last_ld = 0, last_slots = 0, last_ns = 0;  // layout of the last solve's stack
};

std::mutex g_cmu;
std::map<std::pair<int, cudaStream_t>, ChebWs*> g_cws;

progress_status_t cfail(progress_status_t s, const char* what) {
  set_last_error(what);
  return s;
}

progress_status_t ccuda(cudaError_t e, const char* where) {
  set_last_error(where);
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? PROGRESS_ENOMEM : PROGRESS_ECUDA;
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

bool encode_stack(const Pool& pool, int ns, int ld, int nslots, bool bf16, Maps* maps) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
  if (!enc) return false;
  memset(maps, 0, sizeof *maps);
  for (int j = 0; j < ns; ++j) {
    cuuint64_t dims[3] = {(cuuint64_t)ld, (cuuint64_t)ld, (cuuint64_t)nslots};
    cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)ld * (cuuint64_t)ld * 2};
    cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)BM, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(&maps->m[j],
                     bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3,
                     (void*)pool.s[j], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
  }
  return true;
}

// The staged 16 x 16 sum pass (2 <= k <= 16, m <= 16): maps of boxes
// SG_COLS x SG_ROWS x (k - 1) over each slice's slot stack.
template <int F>
cudaError_t launch_sum_staged(const Pool& pool, int ld, int nslots, int k, int m,
                              const std::vector<float>& d, const std::vector<float>& inv_s,
                              double* D, int64_t n, int* err, cudaStream_t s) {
  constexpr int NS = fmt_slices(F);
  if (k < 2 || k > 16 || m > 16 || ld % SG_COLS || nslots < k - 1) return cudaErrorInvalidValue;
  PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
  if (!enc) return cudaErrorInvalidValue;
  SumMaps maps;
  memset(&maps, 0, sizeof maps);
  for (int j = 0; j < NS; ++j) {
    cuuint64_t dims[3] = {(cuuint64_t)ld, (cuuint64_t)ld, (cuuint64_t)nslots};
    cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)ld * (cuuint64_t)ld * 2};
    cuuint32_t box[3] = {(cuuint32_t)SG_COLS, (cuuint32_t)SG_ROWS, (cuuint32_t)(k - 1)};
    cuuint32_t estr[3] = {1, 1, 1};
    if (enc(&maps.m[j], fmt_bf16(F) ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                    : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
            3, (void*)pool.s[j], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  SumTable<16, 16> tab;
  memset(&tab, 0, sizeof tab);
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < m; ++j) tab.d[i * 16 + j] = d[(size_t)i * m + j];
  for (int j = 0; j < m; ++j) tab.inv_s[j] = inv_s[j];
  const int smem = 1024 + SG_STAGES * NS * (k - 1) * SG_ROWS * SG_COLS * 2;
  cudaError_t e = cudaFuncSetAttribute(cheb_sum_staged_kernel<F>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  const int chunks = (ld / SG_ROWS) * (ld / SG_COLS);
  const int grid = std::min(2 * nsm, chunks);
  cheb_sum_staged_kernel<F><<<grid, EW_THREADS, smem, s>>>(maps, pool, ld, k, m, tab, D, n, err);
  return cudaGetLastError();
}

template <int F>
cudaError_t launch_products(const Maps& maps, const Pool& pool, const Prod* d_prods, int count,
                            int ld, double* D, int64_t n, int* err, cudaStream_t s) {
  const int T = ld / BM;
  const int tiles = T * (T + 1) / 2;
  const int smem = Cfg<F>::SMEM;
  cudaError_t e = cudaFuncSetAttribute(cheb_product_kernel<F>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  cheb_product_kernel<F><<<count * tiles, THREADS, smem, s>>>(maps, pool, d_prods, tiles, ld, D,
                                                              n, err);
  return cudaGetLastError();
}

// The whole schedule of one solve, computed on the host from the bounds.
struct Plan {
  double a = 0.0, b = 1.0;     // Ht = (H - a I) / b
  double growth = 0.0;         // sum_j sum_i |d_ij|
  double coef_last = 0.0;      // |c_L|
  int nslots = 0;              // T_1..T_k | S_0..S_{m-1} | two nested-product buffers
  int t_products = 0;          // products of the T levels (the rest are nested)
  std::vector<Prod> prods;
  std::vector<int> level_end;  // prods index after each T-level launch
  std::vector<double> d;       // d_ij at i m + j
  std::vector<double> inv_s;   // 1 / scale of S_j
};

bool make_plan(int k, int m, double mu, double beta, double emin, double emax, Plan* P) {
  if (!isfinite(emin) || !isfinite(emax) || emin > emax) return false;
  double lo = emin, hi = emax;
  if (!(hi > lo)) {
    lo -= 1.0;
    hi += 1.0;
  }
  P->a = 0.5 * (hi + lo);
  P->b = 0.5 * (hi - lo);
  P->nslots = k + m + 2;
  // coefficients, nested-form split and scales (FP64)
  const int L = k * m - 1;
  const std::vector<double> c = coefficients(L, P->a, P->b, mu, beta);
  P->coef_last = fabs(c[L]);
  P->d = ps_split(c, k, m);
  std::vector<double> colsum(m, 0.0), tail(m, 0.0), sS(m), sP(m);
  for (int j = 0; j < m; ++j)
    for (int i = 0; i < k; ++i) colsum[j] += fabs(P->d[(size_t)i * m + j]);
  for (int j = m - 1; j >= 0; --j) tail[j] = colsum[j] + (j + 1 < m ? tail[j + 1] : 0.0);
  for (int j = 0; j < m; ++j) {
    sS[j] = pow2_at_least(colsum[j]);
    sP[j] = pow2_at_least(tail[j]);
  }
  sP[m - 1] = sS[m - 1];  // P_{m-1} is S_{m-1}
  P->growth = tail[0];
  P->inv_s.resize(m);
  for (int j = 0; j < m; ++j) P->inv_s[j] = 1.0 / sS[j];
  // T_2..T_k by levels (T_k itself only when the nested products need it)
  const int k_top = (m > 1) ? k : k - 1;
  P->prods.clear();
  P->level_end.clear();
  for (int lvl = 1; lvl < k_top; lvl *= 2) {
    // level: n in (lvl, 2 lvl]; a = ceil(n/2) <= lvl was made by an earlier launch
    const int hi_n = std::min(2 * lvl, k_top);
    for (int q = lvl + 1; q <= hi_n; ++q) {
      const int ta = (q + 1) / 2, tb = q / 2;
      Prod p;
      p.a = ta - 1;
      p.b = tb - 1;
      p.e = (ta - tb == 1) ? 0 : -1;  // - T_1, or - T_0 = - I
      p.c = q - 1;
      p.alpha = 2.0f;
      p.sab = 1.0f;
      p.beta = -1.0f;
      p.se = 1.0f;
      p.gamma = (ta - tb == 1) ? 0.0f : -1.0f;
      p.inv_sc = 1.0f;
      P->prods.push_back(p);
    }
    P->level_end.push_back((int)P->prods.size());
  }
  P->t_products = (int)P->prods.size();
  // the nested products P_j = S_j + T_k P_{j+1}, j = m - 2 .. 0
  for (int j = m - 2; j >= 0; --j) {
    Prod p;
    p.a = k - 1;                                             // T_k
    p.b = (j == m - 2) ? k + m - 1 : k + m + ((j + 1) & 1);  // P_{j+1}
    p.e = k + j;                                             // S_j
    p.c = (j == 0) ? -1 : k + m + (j & 1);
    p.alpha = 1.0f;
    p.sab = (float)sP[j + 1];
    p.beta = 1.0f;
    p.se = (float)sS[j];
    p.gamma = 0.0f;
    p.inv_sc = (j == 0) ? 1.0f : (float)(1.0 / sP[j]);
    P->prods.push_back(p);
  }
  return true;
}

template <int F>
progress_status_t run(const double* dH, int64_t n, double mu, double beta, int k, int m,
                      const double* h_bounds, double* dD, progress_cheb_info_t* info,
                      cudaStream_t s) {
  constexpr int NS = fmt_slices(F);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return ccuda(e, "cudaGetDevice");
  ChebWs* w = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_cmu);
    auto key = std::make_pair(dev, s);
    auto it = g_cws.find(key);
    if (it == g_cws.end()) {
      w = new ChebWs();
      g_cws[key] = w;
    } else {
      w = it->second;
    }
  }
  const int ld = (int)((n + BM - 1) / BM) * BM;
  const int nslots = k + m + 2;
  const int nprod_max = (k - 1) + (m - 1);
  // the previous call on this stream may still read the buffers
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return ccuda(e, "stream synchronize");
  if (!w->err) {
    if ((e = cudaMalloc(&w->err, sizeof(int))) != cudaSuccess) return ccuda(e, "cheb alloc");
    if ((e = cudaMalloc(&w->scal, 4 * sizeof(double))) != cudaSuccess) return ccuda(e, "cheb alloc");
  }
  const size_t need = (size_t)NS * nslots * (size_t)ld * ld;
  if (need > w->pool_cap) {
    if (w->pool) cudaFree(w->pool);
    w->pool = nullptr;
    w->pool_cap = 0;
    if ((e = cudaMalloc(&w->pool, need * sizeof(uint16_t))) != cudaSuccess)
      return ccuda(e, "cheb operand stack allocation");
    w->pool_cap = need;
  }
  if ((size_t)std::max(nprod_max, 1) > w->prods_cap) {
    if (w->prods) cudaFree(w->prods);
    w->prods = nullptr;
    w->prods_cap = 0;
    if ((e = cudaMalloc(&w->prods, (size_t)std::max(nprod_max, 1) * sizeof(Prod))) != cudaSuccess)
      return ccuda(e, "cheb product table allocation");
    w->prods_cap = std::max(nprod_max, 1);
  }
  // spectral bounds: the caller's, or Gershgorin (one read-back)
  double emin, emax;
  if (h_bounds) {
    emin = h_bounds[0];
    emax = h_bounds[1];
  } else {
    progress_status_t st = progress_gershgorin_bounds(dH, n, w->scal, w->scal + 1, s);
    if (st != PROGRESS_OK) return st;
    double hb[2];
    e = cudaMemcpyAsync(hb, w->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return ccuda(e, "bounds read-back");
    emin = hb[0];
    emax = hb[1];
  }
  Plan plan;
  if (!make_plan(k, m, mu, beta, emin, emax, &plan))
    return cfail(PROGRESS_EINVAL, "spectral bounds must be finite with emin <= emax");
  const std::vector<Prod>& prods = plan.prods;
  const int nprod = (int)prods.size();
  const int t_products = plan.t_products;
  const double a = plan.a, b = plan.b;
  std::vector<float> dcoef((size_t)k * m), inv_s(m);
  for (size_t i = 0; i < dcoef.size(); ++i) dcoef[i] = (float)plan.d[i];
  for (int j = 0; j < m; ++j) inv_s[j] = (float)plan.inv_s[j];
  Pool pool;
  for (int j = 0; j < 3; ++j) pool.s[j] = w->pool + (size_t)std::min(j, NS - 1) * nslots * ld * ld;
  w->last_ld = ld;
  w->last_slots = nslots;
  w->last_ns = NS;
  Maps maps;
  if (!encode_stack(pool, NS, ld, nslots, fmt_bf16(F), &maps))
    return cfail(PROGRESS_ECUDA, "tensor map encoding failed");
  e = cudaMemsetAsync(w->err, 0, sizeof(int), s);
  if (e == cudaSuccess && nprod > 0)
    e = cudaMemcpyAsync(w->prods, prods.data(), prods.size() * sizeof(Prod),
                        cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return ccuda(e, "cheb set-up upload");
  int launches = h_bounds ? 0 : 2;  // state init + Gershgorin
  const unsigned ew_blocks =
      (unsigned)std::min<size_t>(EW_BLOCKS, ((size_t)ld * ld + EW_THREADS - 1) / EW_THREADS);
  cheb_t1_kernel<F><<<ew_blocks, EW_THREADS, 0, s>>>(dH, n, ld, a, 1.0 / b, pool);
  if ((e = cudaGetLastError()) != cudaSuccess) return ccuda(e, "cheb_t1 launch");
  ++launches;
  int first = 0;
  for (int end : plan.level_end) {
    e = launch_products<F>(maps, pool, w->prods + first, end - first, ld, dD, n, w->err, s);
    if (e != cudaSuccess) return ccuda(e, "cheb product launch (T levels)");
    ++launches;
    first = end;
  }
  if (k >= 2 && k <= 16 && m <= 16)
    e = launch_sum_staged<F>(pool, ld, plan.nslots, k, m, dcoef, inv_s, dD, n, w->err, s);
  else if (k <= 16 && m <= 16)
    e = launch_sum_fast<F, 16, 16, 2>(pool, ld, k, m, dcoef, inv_s, dD, n, w->err, s);
  else if (k <= 32 && m <= 32)
    e = launch_sum_fast<F, 32, 32, 1>(pool, ld, k, m, dcoef, inv_s, dD, n, w->err, s);
  else
    e = launch_sum_fast<F, 64, 64, 1>(pool, ld, k, m, dcoef, inv_s, dD, n, w->err, s);
  if (e != cudaSuccess) return ccuda(e, "cheb_sum launch");
  ++launches;
  for (int q = t_products; q < nprod; ++q) {
    e = launch_products<F>(maps, pool, w->prods + q, 1, ld, dD, n, w->err, s);
    if (e != cudaSuccess) return ccuda(e, "cheb product launch (nested)");
    ++launches;
  }
  cheb_trace_kernel<<<1, EW_THREADS, 0, s>>>(dD, n, w->scal + 2);
  if ((e = cudaGetLastError()) != cudaSuccess) return ccuda(e, "cheb_trace launch");
  ++launches;
  int herr = 0;
  double tr = 0.0;
  e = cudaMemcpyAsync(&herr, w->err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&tr, w->scal + 2, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return ccuda(e, "cheb result read-back");
  if (info) {
    memset(info, 0, sizeof *info);
    info->emin = emin;
    info->emax = emax;
    info->trace = tr;
    info->growth = plan.growth;
    info->products = nprod;
    info->launches = launches;
    info->coef_last = plan.coef_last;
  }
  if (herr) return cfail((progress_status_t)herr, "a bounded device-side wait gave up");
  return PROGRESS_OK;
}

}  // namespace

void cheb_release(int dev, cudaStream_t s, bool all_streams) {
  std::lock_guard<std::mutex> lk(g_cmu);
  for (auto it = g_cws.begin(); it != g_cws.end();) {
    if (it->first.first == dev && (all_streams || it->first.second == s)) {
      ChebWs* w = it->second;
      void* ptrs[] = {w->pool, w->prods, w->err, w->scal};
      for (void* p : ptrs)
        if (p) cudaFree(p);
      delete w;
      it = g_cws.erase(it);
    } else {
      ++it;
    }
  }
}

}  // namespace sp2

extern "C" progress_status_t progress_cheb_fermi(const double* dH, int64_t n, double mu,
                                                 double beta, int32_t k, int32_t m, int32_t prec,
                                                 const double* h_bounds, double* dD,
                                                 progress_cheb_info_t* info, void* stream) {
  using namespace sp2;
  if (n < 1 || n > 32768) return cfail(PROGRESS_EINVAL, "n must be in [1, 32768]");
  if (k < 1 || k > MAX_K || m < 1 || m > MAX_M)
    return cfail(PROGRESS_EINVAL, "k and m must be in [1, 64]");
  if (!dH || !dD) return cfail(PROGRESS_EINVAL, "NULL matrix pointer");
  if (dD == dH) return cfail(PROGRESS_EINVAL, "dD must not overlap dH");
  if (!isfinite(mu) || !isfinite(beta) || beta < 0.0)
    return cfail(PROGRESS_EINVAL, "mu must be finite and beta finite and >= 0");
  if (prec != PROGRESS_FP32_SPLIT && prec != PROGRESS_FP32_SPLIT_BF16)
    return cfail(PROGRESS_EINVAL, "prec must be PROGRESS_FP32_SPLIT or PROGRESS_FP32_SPLIT_BF16");
  int dev = 0, major = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  if (e != cudaSuccess) return ccuda(e, "device query");
  if (major != 10) return cfail(PROGRESS_EUNSUPPORTED, "the Chebyshev solver needs an sm_10x GPU");
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == PROGRESS_FP32_SPLIT)
    return run<kFP16x2>(dH, n, mu, beta, k, m, h_bounds, dD, info, s);
  return run<kBF16x3>(dH, n, mu, beta, k, m, h_bounds, dD, info, s);
}

extern "C" progress_status_t progress_cheb_plan(int32_t k, int32_t m, double mu, double beta,
                                                double emin, double emax, int32_t cap,
                                                int32_t* prods, float* params, double* dcoef,
                                                double* inv_s, double* ab, int32_t* counts) {
  using namespace sp2;
  if (k < 1 || k > MAX_K || m < 1 || m > MAX_M)
    return cfail(PROGRESS_EINVAL, "k and m must be in [1, 64]");
  if (!isfinite(mu) || !isfinite(beta) || beta < 0.0)
    return cfail(PROGRESS_EINVAL, "mu must be finite and beta finite and >= 0");
  if (!prods || !params || !dcoef || !inv_s || !ab || !counts)
    return cfail(PROGRESS_EINVAL, "NULL output pointer");
  Plan plan;
  if (!make_plan(k, m, mu, beta, emin, emax, &plan))
    return cfail(PROGRESS_EINVAL, "spectral bounds must be finite with emin <= emax");
  const int np = (int)plan.prods.size();
  if (cap < np) return cfail(PROGRESS_EINVAL, "cap is smaller than the product count");
  int launch = 0, q = 0;
  for (int end : plan.level_end) {
    for (; q < end; ++q) prods[5 * q + 4] = launch;
    ++launch;
  }
  for (; q < np; ++q) prods[5 * q + 4] = launch++;
  for (int i = 0; i < np; ++i) {
    const Prod& p = plan.prods[i];
    prods[5 * i + 0] = p.a;
    prods[5 * i + 1] = p.b;
    prods[5 * i + 2] = p.e;
    prods[5 * i + 3] = p.c;
    const float v[6] = {p.alpha, p.sab, p.beta, p.se, p.gamma, p.inv_sc};
    for (int j = 0; j < 6; ++j) params[6 * i + j] = v[j];
  }
  for (size_t i = 0; i < plan.d.size(); ++i) dcoef[i] = plan.d[i];
  for (int j = 0; j < m; ++j) inv_s[j] = plan.inv_s[j];
  ab[0] = plan.a;
  ab[1] = plan.b;
  counts[0] = np;
  counts[1] = launch;
  counts[2] = plan.nslots;
  counts[3] = plan.t_products;
  return PROGRESS_OK;
}

extern "C" progress_status_t progress_cheb_choose(int32_t terms, double mu, double beta,
                                                  double emin, double emax, double max_growth,
                                                  int32_t* k_out, int32_t* m_out,
                                                  int32_t* products_out, double* growth_out) {
  using namespace sp2;
  if (terms < 1 || terms > MAX_K * MAX_M) return cfail(PROGRESS_EINVAL, "terms must be in [1, 4096]");
  if (!isfinite(mu) || !isfinite(beta) || beta < 0.0)
    return cfail(PROGRESS_EINVAL, "mu must be finite and beta finite and >= 0");
  if (!(max_growth > 0.0)) return cfail(PROGRESS_EINVAL, "max_growth must be > 0");
  if (!k_out || !m_out) return cfail(PROGRESS_EINVAL, "NULL output pointer");
  // every split k m >= terms (m = ceil(terms / k)); the plan that progress_cheb_fermi
  // would run, ranked by its product count, then by its term count
  int best_k = 0, best_m = 0, best_p = 0, best_terms = 0;
  double best_g = 0.0;
  for (int k = 1; k <= MAX_K; ++k) {
    const int m = (terms + k - 1) / k;
    if (m > MAX_M) continue;
    Plan plan;
    if (!make_plan(k, m, mu, beta, emin, emax, &plan))
      return cfail(PROGRESS_EINVAL, "spectral bounds must be finite with emin <= emax");
    if (!(plan.growth <= max_growth)) continue;
    const int np = (int)plan.prods.size();
    if (best_k == 0 || np < best_p || (np == best_p && k * m < best_terms)) {
      best_k = k;
      best_m = m;
      best_p = np;
      best_terms = k * m;
      best_g = plan.growth;
    }
  }
  if (best_k == 0)
    return cfail(PROGRESS_EINVAL, "no (k, m) with k m >= terms keeps the growth within max_growth");
  *k_out = best_k;
  *m_out = best_m;
  if (products_out) *products_out = best_p;
  if (growth_out) *growth_out = best_g;
  return PROGRESS_OK;
}

extern "C" progress_status_t progress_cheb_slot(int32_t slot, int32_t slice, uint16_t* host_out,
                                                void* stream) {
  using namespace sp2;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return ccuda(e, "cudaGetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  ChebWs* w = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_cmu);
    auto it = g_cws.find(std::make_pair(dev, s));
    if (it != g_cws.end()) w = it->second;
  }
  if (!w || !w->pool || w->last_ld == 0) return cfail(PROGRESS_EINVAL, "no Chebyshev solve on this stream");
  if (slot < 0 || slot >= w->last_slots || slice < 0 || slice >= w->last_ns || !host_out)
    return cfail(PROGRESS_EINVAL, "slot or slice out of range, or NULL output");
  const size_t area = (size_t)w->last_ld * w->last_ld;
  const uint16_t* src = w->pool + ((size_t)slice * w->last_slots + slot) * area;
  e = cudaMemcpyAsync(host_out, src, area * sizeof(uint16_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return ccuda(e, "slot read-back");
  return PROGRESS_OK;
}
