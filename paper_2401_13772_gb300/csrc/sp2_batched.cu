// Batched SP2: thousands of independent dense sub-Hamiltonians of uneven size
// (the parts of a graph-partitioned system, §VIII.B, which are independent
// problems solved concurrently) in ONE persistent kernel launch.
//
// Scheduling: the grid is a set of thread-block clusters of C CTAs (C = 1, 2,
// 4 or 8, one CTA per SM). Instances sit in a device work queue ordered by
// decreasing size (greedy longest-processing-time). A large instance (at
// least `share` 128-row blocks) is taken by a whole cluster: its product
// tiles are dealt round-robin to the cluster's CTAs, the partial traces are
// exchanged through distributed shared memory and every CTA takes the same
// branch decision from the same sums. Fewer instances are then in flight,
// so their operand slices stay resident in L2 across the tiles of an
// iteration. Once the queue reaches the small instances the cluster splits
// and each CTA takes whole instances by itself. No CTA waits on a flag in
// global memory: cluster barriers are hardware barriers.
//
// Layout: every instance i is padded to m_i = round_up(n_i, 128) and stored as
// operand slices (FP16x2 or BF16x3) in "tall" matrices of pitch P = max m_i:
// instance i owns rows [row0_i, row0_i + m_i), columns [0, m_i). One TMA
// tensor map per slice, set and operand box therefore serves every instance.
//
// Roles inside a CTA (384 threads), per product tile (128 x BN outputs):
//   warp 0 lane 0 : TMA producer into a STAGES-deep ring (continues across
//                   tiles, so the next tile's operands stream in during the
//                   current tile's epilogue)
//   warp 1 lane 0 : tcgen05.mma issuer, M = 128, N = BN, K = 16, FP32
//                   accumulators in one of two tensor-memory buffers
//                   (double-buffered across tiles)
//   warps 4..11   : epilogue, two warps per 32-lane quarter of tensor memory
//                   (each takes half of the tile's columns): S = X^2 from the
//                   accumulators, X' = S or 2X - S, the new slices of X' at
//                   (r, c) (staged through shared memory so that the stores
//                   run along rows) and at the mirror (c, r), partial traces.
// At the end of an iteration the traces are reduced (CTA, then cluster) and
// the next step is decided; generic-proxy stores are fenced before the next
// iteration's TMA reads them.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <string.h>

#include "sp2_batched.h"
#include "sp2_common.cuh"
#include "sp2_slices.cuh"
#include "sp2_tc.cuh"

namespace sp2 {
namespace batched {

using namespace tc;

namespace {

constexpr int BM = 128;
constexpr int BK = 64;
constexpr int A_BYTES = BM * BK * 2;  // one 128 x 64 slice box
constexpr int THREADS = 384;
constexpr int NWARPS = THREADS / 32;
constexpr int EPI_WARP0 = 4;  // warps 4..11
constexpr int NEPI = 8;
constexpr int MAX_CLUSTER = 8;
constexpr int MAX_STAGES = 4;

template <int F, int BN>
struct BCfg {
  static constexpr int NS = fmt_slices(F);
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE_BYTES = NS * (A_BYTES + B_BYTES);
  static constexpr int STAGES = fmt_bf16(F) ? 2 : (BN == 128 ? 3 : 4);
  // Two accumulators per buffer: acc0 = hi*hi and acc1 = the correction
  // products (FP16x2: hi*lo + lo*hi, weight 2^-11; BF16x3: hi*mid + mid*hi +
  // hi*lo + lo*hi + mid*mid, weight 1). The tensor core's FP32 accumulation
  // truncates; adding the small correction terms into the leading sum would
  // drop their low bits every time (a systematic bias), so they are summed on
  // their own scale.
  static constexpr int ACC_COLS = 2 * BN;
  static constexpr int TMEM_COLS = 2 * ACC_COLS;
  static constexpr int COLS_PER_WARP = BN / 2;
  // epilogue staging per warp: 32 rows x 16 columns of packed (slice0,
  // slice1) words (row stride 17 words) and, for BF16x3, of slice-2 half
  // words (row stride 18)
  static constexpr int EPI_A = 32 * 17;
  static constexpr int EPI_B = 32 * 18;
  static constexpr int EPI_BYTES = NEPI * (EPI_A * 4 + (NS == 3 ? EPI_B * 2 : 0));
  static constexpr int SMEM = STAGES * STAGE_BYTES + EPI_BYTES + 1024;
  static_assert(STAGES <= MAX_STAGES, "ring too deep");
  static_assert(TMEM_COLS >= 32 && (TMEM_COLS & (TMEM_COLS - 1)) == 0, "tensor memory columns");
};

struct Maps {
  CUtensorMap a[2][3];  // [set][slice], 64 x 128 boxes (rows of block I)
  CUtensorMap b[2][3];  // [set][slice], 64 x BN boxes (rows of block J)
};

struct Shared {
  State st;  // control state of the instance in flight
  double red[2 * NWARPS];
  double lo[NWARPS], hi[NWARPS];
  double xch[2][MAX_CLUSTER][4];  // cluster exchange slots [parity][rank][value]
  uint64_t bars[2 * MAX_STAGES + 5];
  int kb_consumed;
  uint32_t tmem;
  int err;
  int inst;
  int share;
};

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void fence_async_global() {
  asm volatile("fence.proxy.async.global;\n" ::: "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
  return r;
}

__device__ __forceinline__ uint32_t cluster_size() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;\n" : "=r"(r));
  return r;
}

// All threads of all CTAs of the cluster; release/acquire at cluster scope.
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n"
      "barrier.cluster.wait.acquire.aligned;\n" ::
          : "memory");
}

__device__ __forceinline__ uint32_t map_rank(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}

__device__ __forceinline__ void st_cluster_f64(uint32_t addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;\n" ::"r"(addr), "d"(v) : "memory");
}

__device__ __forceinline__ void st_cluster_s32(uint32_t addr, int v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;\n" ::"r"(addr), "r"(v) : "memory");
}

// Product tiles of an instance with T row blocks: (I, J) with rows
// [128 I, 128 I + 128) and columns [BN J, BN J + BN) that hold at least one
// element on or above the diagonal, row-major.
template <int BN>
__device__ __forceinline__ int tile_count(int T) {
  constexpr int R = BM / BN;
  return R * T * (T + 1) / 2;
}

template <int BN>
__device__ __forceinline__ void tile_of(int t, int T, int& I, int& J) {
  if (BN == BM) {
    tri_tile(t, T, I, J);
    return;
  }
  constexpr int R = BM / BN;
  const int C = R * T;
  int i = 0;
  while (t >= C - R * i) {
    t -= C - R * i;
    ++i;
  }
  I = i;
  J = R * i + t;
}

// Thread 0 of a CTA: write (a, b, c) into slot [par][rank] of every CTA of
// the cluster (the caller then runs cluster_sync_all()).
__device__ __forceinline__ void xch_put(Shared& sh, int par, int rank, int G, double a, double b,
                                        double c) {
  const uint32_t loc = smem_u32(&sh.xch[par][rank][0]);
  for (int r = 0; r < G; ++r) {
    const uint32_t p = map_rank(loc, (uint32_t)r);
    st_cluster_f64(p, a);
    st_cluster_f64(p + 8u, b);
    st_cluster_f64(p + 16u, c);
  }
}

template <int F, int BN>
__global__ void __launch_bounds__(THREADS, 1)
    batched_kernel(const __grid_constant__ Maps maps, Params prm) {
  using Cfg = BCfg<F, BN>;
  constexpr int NS = Cfg::NS;
  constexpr int STAGES = Cfg::STAGES;
  constexpr int STAGE_BYTES = Cfg::STAGE_BYTES;
  constexpr int ACC_COLS = Cfg::ACC_COLS;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ Shared sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool epi = warp >= EPI_WARP0;
  const int quarter = warp & 3;                        // tensor-memory lanes 32q .. 32q + 31
  const int half = epi ? (warp - EPI_WARP0) >> 2 : 0;  // column half of the tile
  const int erow = quarter * 32 + lane;                // tile row of an epilogue thread
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  unsigned char* const epi_base = smem_raw + (base - smem_u32(smem_raw)) + STAGES * STAGE_BYTES;
  const int ew = epi ? warp - EPI_WARP0 : 0;
  uint32_t* const epA = reinterpret_cast<uint32_t*>(epi_base) + ew * Cfg::EPI_A;
  uint16_t* const epB =
      reinterpret_cast<uint16_t*>(epi_base + NEPI * Cfg::EPI_A * 4) + ew * Cfg::EPI_B;
  const uint32_t bars = smem_u32(&sh.bars[0]);
  auto full_bar = [&](int s) { return bars + 8u * s; };
  auto empty_bar = [&](int s) { return bars + 8u * (STAGES + s); };
  const uint32_t tfull = bars + 8u * (2 * STAGES);          // [2] MMA -> epilogue
  const uint32_t tempty = bars + 8u * (2 * STAGES + 2);     // [2] epilogue -> MMA
  const uint32_t drain_bar = bars + 8u * (2 * STAGES + 4);  // failure path only
  const int G = (int)cluster_size();
  const int rank = (int)cluster_rank();

  if (threadIdx.x == 0) {
    sh.err = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull + 8u * b, 1);
      mbar_init(tempty + 8u * b, NEPI);
    }
    mbar_init(drain_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(&sh.tmem), Cfg::TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh.tmem;
  volatile int* err = &sh.err;
  constexpr uint32_t idesc = idesc_f16(fmt_bf16(F) ? 1 : 0, BM, BN);

  // ring / buffer counters, each kept by the thread that uses it
  uint32_t kb_prod = 0, kb_mma = 0, tile_mma = 0, tile_epi = 0;
  int xk = 0;             // cluster exchanges so far (the same count in every CTA of a cluster)
  bool together = G > 1;  // the cluster still takes its instances jointly
  if (together) cluster_sync_all();  // every CTA of the cluster is running

  for (;;) {
    // ---- next work item
    int inst, gsz, grank;
    if (together) {
      cluster_sync_all();  // every CTA is done with the previous item
      if (*err) break;     // the same in every CTA of the cluster (exchanged)
      if (rank == 0 && threadIdx.x == 0) {
        const int q = atomicAdd(prm.queue, 1);
        const int i = q < prm.batch ? prm.order[q] : -1;
        const int shr = (i >= 0 && prm.inst[i].m / BM >= prm.share) ? 1 : 0;
        for (int r = 0; r < G; ++r) {
          // a small instance stays with rank 0; the others then take their own
          st_cluster_s32(map_rank(smem_u32(&sh.inst), (uint32_t)r),
                         (r == 0 || shr || i < 0) ? i : -2);
          st_cluster_s32(map_rank(smem_u32(&sh.share), (uint32_t)r), shr);
        }
      }
      cluster_sync_all();
      inst = sh.inst;
      const int shr = sh.share;
      __syncthreads();  // every thread has read sh.inst
      if (!shr) together = false;  // the queue is sorted: no larger instance follows
      if (inst == -2) {
        if (threadIdx.x == 0) {
          const int q = atomicAdd(prm.queue, 1);
          sh.inst = q < prm.batch ? prm.order[q] : -1;
        }
        __syncthreads();
        inst = sh.inst;
      }
      gsz = shr ? G : 1;
      grank = shr ? rank : 0;
    } else {
      __syncthreads();  // every thread has read the previous sh.inst
      if (threadIdx.x == 0) {
        const int q = atomicAdd(prm.queue, 1);
        sh.inst = q < prm.batch ? prm.order[q] : -1;
      }
      __syncthreads();
      inst = sh.inst;
      gsz = 1;
      grank = 0;
      if (*err) break;
    }
    if (inst < 0) break;
    const long long c_start = clock64();
    const Instance in = prm.inst[inst];
    const int n = in.n, m = in.m, T = m / BM;
    const double* __restrict__ H = prm.H + in.offset;
    State& st = sh.st;
    // A run with predicted bounds/bits that the judge rejects (or that
    // diverges) is restarted once on the plain path.
    bool predicted = prm.bounds_in != nullptr || prm.pred_bits != nullptr;
    bool fell_back = false;
    int wasted = 0;  // products of a rejected predicted run
  restart:

    // ---- set-up: state, Gershgorin bounds, X0 (rows dealt over the group)
    {
      unsigned int* w = reinterpret_cast<unsigned int*>(&st);
      for (int i = threadIdx.x; i < (int)(sizeof(State) / 4); i += THREADS) w[i] = 0u;
    }
    __syncthreads();
    double lo = INFINITY, hi = -INFINITY;
    for (int r = grank * NWARPS + warp; r < n; r += gsz * NWARPS) {
      const double* row = H + (size_t)r * n;
      double s = 0.0;
      for (int j = lane; j < n; j += 32) s += (j == r) ? 0.0 : fabs(row[j]);
      s = warp_sum(s);
      lo = fmin(lo, row[r] - s);
      hi = fmax(hi, row[r] + s);
    }
    lo = warp_min(lo);
    hi = warp_max(hi);
    if (lane == 0) {
      sh.lo[warp] = lo;
      sh.hi[warp] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < NWARPS; ++w) {
        lo = fmin(lo, sh.lo[w]);
        hi = fmax(hi, sh.hi[w]);
      }
      if (gsz > 1) xch_put(sh, xk & 1, grank, gsz, lo, hi, 0.0);
    }
    if (gsz > 1) {
      cluster_sync_all();
      if (threadIdx.x == 0) {
        lo = INFINITY;
        hi = -INFINITY;
        for (int r = 0; r < gsz; ++r) {
          lo = fmin(lo, sh.xch[xk & 1][r][0]);
          hi = fmax(hi, sh.xch[xk & 1][r][1]);
        }
      }
      ++xk;
    }
    if (threadIdx.x == 0) {
      if (!(hi > lo)) {  // zero-width enclosure: widen (as the dense solver does)
        lo -= 1.0;
        hi += 1.0;
      }
      st.n = n;
      st.ld = m;
      st.nocc = in.nocc;
      st.rule = prm.rule;
      st.maxiter = prm.maxiter;
      st.prec = PROGRESS_FP32_SPLIT;
      st.tol = prm.tol;
      st.emin = lo;
      st.emax = hi;
      if (predicted && prm.bounds_in) {
        const double e0 = prm.bounds_in[2 * inst], e1 = prm.bounds_in[2 * inst + 1];
        if (isfinite(e0) && isfinite(e1) && e1 > e0) {
          st.emin = e0;
          st.emax = e1;
        }
      }
      if (predicted && prm.pred_bits && prm.pred_len) {
        for (int b = 0; b < 4; ++b) st.pred_bits[b] = prm.pred_bits[4 * inst + b];
        st.pred_len = min(prm.pred_len[inst], kMaxHist);
        st.judge_delta = prm.judge_delta;
      }
      if (prm.rule == PROGRESS_RULE_MU) {
        // theta(mu I - H): mu must map strictly inside (0, 1)
        const double mu = prm.mu_in[inst];
        if (!(st.emin < mu && mu < st.emax)) {
          st.emin = fmin(st.emin, mu - 1.0);
          st.emax = fmax(st.emax, mu + 1.0);
        }
        st.y_mu = (st.emax - mu) / (st.emax - st.emin);
      }
      st.best_split_idem = INFINITY;
      st.phase = kPhaseSplit;
    }
    __syncthreads();
    {
      // X0 = (emax I - H) / (emax - emin) in FP32 (the slices carry 22 bits);
      // one warp per row, partial traces in FP32 per row, folded into FP64.
      const float emax_f = (float)st.emax, inv_f = (float)(1.0 / (st.emax - st.emin));
      uint16_t* s0 = prm.sl[0][0];
      uint16_t* s1 = prm.sl[0][1];
      uint16_t* s2 = prm.sl[0][2];
      double tr = 0.0, fr = 0.0;
      for (int r = grank * NWARPS + warp; r < m; r += gsz * NWARPS) {
        float trf = 0.0f, frf = 0.0f;
        const size_t g0 = (size_t)(in.row0 + r) * prm.pitch;
        for (int c = lane; c < m; c += 32) {
          float x = 0.0f;
          if (r < n && c < n) {
            const float h = (float)H[(size_t)r * n + c];
            x = ((r == c) ? (emax_f - h) : -h) * inv_f;
            if (r == c) trf += x;
            frf += x * x;
          }
          uint16_t a, b, c2;
          split_value_f<F>(x, a, b, c2);
          s0[g0 + c] = a;
          s1[g0 + c] = b;
          if (NS == 3) s2[g0 + c] = c2;
        }
        tr += (double)trf;
        fr += (double)frf;
      }
      fence_async_global();
      block_sum2(tr, fr, sh.red);
      if (gsz > 1) {
        if (threadIdx.x == 0) xch_put(sh, xk & 1, grank, gsz, tr, fr, 0.0);
        cluster_sync_all();
        if (threadIdx.x == 0) {
          tr = 0.0;
          fr = 0.0;
          for (int r = 0; r < gsz; ++r) {
            tr += sh.xch[xk & 1][r][0];
            fr += sh.xch[xk & 1][r][1];
          }
        }
        ++xk;
      }
      if (threadIdx.x == 0) {
        st.t1 = tr;
        st.t2 = fr;
        st.iter = 0;
        decide(&st);
      }
    }
    __syncthreads();

    // ---- SP2 iterations
    while (!st.done) {
      const int k = st.iter;
      const int bit = st.bit;
      const int src = k & 1, dst = (k + 1) & 1;
      const int ntiles = tile_count<BN>(T);
      const int KB = m / BK;
      if (warp == 0) {
        if (lane == 0) {
          fence_async_global();  // slices written by the group before the barrier
          for (int t = grank; t < ntiles && !*err; t += gsz) {
            int I, J;
            tile_of<BN>(t, T, I, J);
            for (int kb = 0; kb < KB; ++kb, ++kb_prod) {
              const int s = kb_prod % STAGES;
              const uint32_t ph = (kb_prod / STAGES) & 1u;
              if (!mbar_wait(empty_bar(s), ph ^ 1u, err)) break;
              mbar_expect_tx(full_bar(s), STAGE_BYTES);
              const uint32_t sa = base + s * STAGE_BYTES;
              for (int j = 0; j < NS; ++j) {
                tma_load_2d(sa + j * A_BYTES, &maps.a[src][j], kb * BK, (int)(in.row0 + I * BM),
                            full_bar(s));
                tma_load_2d(sa + NS * A_BYTES + j * Cfg::B_BYTES, &maps.b[src][j], kb * BK,
                            (int)(in.row0 + J * BN), full_bar(s));
              }
            }
          }
        }
        __syncwarp();
      } else if (warp == 1) {
        if (lane == 0) {
          for (int t = grank; t < ntiles && !*err; t += gsz, ++tile_mma) {
            const uint32_t tb = tile_mma & 1u;
            if (!mbar_wait(tempty + 8u * tb, ((tile_mma >> 1) & 1u) ^ 1u, err)) break;
            tc_fence_after();
            const uint32_t acc0 = tmem + ACC_COLS * tb, acc1 = acc0 + BN;
            for (int kb = 0; kb < KB; ++kb, ++kb_mma) {
              const int s = kb_mma % STAGES;
              const uint32_t ph = (kb_mma / STAGES) & 1u;
              if (!mbar_wait(full_bar(s), ph, err)) break;
              tc_fence_after();
              const uint32_t sa = base + s * STAGE_BYTES;
              uint64_t a[NS], b[NS];
#pragma unroll
              for (int j = 0; j < NS; ++j) {
                a[j] = smem_desc_sw128(sa + j * A_BYTES);
                b[j] = smem_desc_sw128(sa + NS * A_BYTES + j * Cfg::B_BYTES);
              }
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk) {
                const uint64_t adv = (uint64_t)(kk * 32) >> 4;
                const uint32_t acc = (kb == 0 && kk == 0) ? 0u : 1u;
                if (NS == 2) {
                  mma_f16(acc0, a[0] + adv, b[0] + adv, idesc, acc);
                  mma_f16(acc1, a[0] + adv, b[1] + adv, idesc, acc);
                  mma_f16(acc1, a[1] + adv, b[0] + adv, idesc, 1u);
                } else {
                  // the corrections, small terms first, then the leading product
                  mma_f16(acc1, a[0] + adv, b[2 % NS] + adv, idesc, acc);
                  mma_f16(acc1, a[2 % NS] + adv, b[0] + adv, idesc, 1u);
                  mma_f16(acc1, a[1] + adv, b[1] + adv, idesc, 1u);
                  mma_f16(acc1, a[0] + adv, b[1] + adv, idesc, 1u);
                  mma_f16(acc1, a[1] + adv, b[0] + adv, idesc, 1u);
                  mma_f16(acc0, a[0] + adv, b[0] + adv, idesc, acc);
                }
              }
              mma_commit(empty_bar(s));
            }
            mma_commit(tfull + 8u * tb);
          }
        }
        __syncwarp();
      }
      // partial traces of this iteration: the FP32 sum of each 32-column chunk
      // (the same chunks in every launch configuration) is added exactly on the
      // 2^-40 grid in 64-bit integers, converted to FP64 once per iteration (FP64
      // adds per tile held up the epilogue; the exact sums keep the traces, and
      // with them the branch decisions, independent of the configuration)
      long long tfix = 0, ffix = 0;
      if (epi) {
        const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
        const uint16_t* xs0 = prm.sl[src][0];
        const uint16_t* xs1 = prm.sl[src][1];
        const uint16_t* xs2 = prm.sl[src][2];
        uint16_t* o0 = prm.sl[dst][0];
        uint16_t* o1 = prm.sl[dst][1];
        uint16_t* o2 = prm.sl[dst][2];
        const size_t P = prm.pitch;
        for (int t = grank; t < ntiles; t += gsz, ++tile_epi) {
          const uint32_t tb = tile_epi & 1u;
          const bool ok = mbar_wait(tfull + 8u * tb, (tile_epi >> 1) & 1u, err);
          tc_fence_after();
          int I, J;
          tile_of<BN>(t, T, I, J);
          const int r = I * BM + erow;  // row within the instance
          const int rb = I * BM + quarter * 32;
          if (ok && !*err) {
#pragma unroll 1
            for (int ch = 0; ch < Cfg::COLS_PER_WARP / 32; ++ch) {
              const int cofs = half * Cfg::COLS_PER_WARP + ch * 32;  // column in the tile
              const int c0 = J * BN + cofs;
              float trf = 0.0f, frf = 0.0f;
              // X at the mirror (for 2X - X^2) does not depend on the products:
              // load it before the tensor-memory reads (packed slice0 | slice1
              // << 16; coalesced across the warp's rows). Two slices: both
              // 16-column halves at once (one round of load latency per chunk)
              uint32_t mm01[2][16], mm2[2][16];
              auto load_mirror = [&](int hh) {
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                  const size_t mi = (size_t)(in.row0 + c0 + hh * 16 + jj) * P + r;
                  mm01[hh][jj] = (uint32_t)xs0[mi] | ((uint32_t)xs1[mi] << 16);
                  mm2[hh][jj] = NS == 3 ? (uint32_t)xs2[mi] : 0u;
                }
              };
              if (bit && NS == 2) {
                load_mirror(0);
                load_mirror(1);
              }
#pragma unroll
              for (int hh = 0; hh < 2; ++hh) {
                if (bit && NS == 3) load_mirror(hh);
                const uint32_t* m01 = mm01[hh];
                const uint32_t* m2 = mm2[hh];
                uint32_t u0[16], u1[16];
                tmem_ld16(tmem + lane_base + ACC_COLS * tb + cofs + hh * 16, u0);
                tmem_ld16(tmem + lane_base + ACC_COLS * tb + BN + cofs + hh * 16, u1);
                tmem_ld_wait();
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                  const int c = c0 + hh * 16 + jj;
                  float x = (NS == 2)
                                ? __uint_as_float(u0[jj]) + __uint_as_float(u1[jj]) * (1.0f / 2048.0f)
                                : __uint_as_float(u0[jj]) + __uint_as_float(u1[jj]);
                  if (bit)
                    x = 2.0f * join_value<F>((uint16_t)(m01[jj] & 0xffffu),
                                             (uint16_t)(m01[jj] >> 16), (uint16_t)m2[jj]) -
                        x;
                  if (r <= c) {
                    uint16_t a, b, c2;
                    split_value_f<F>(x, a, b, c2);
                    // (r, c) and its mirror (c, r) go through the staging planes
                    // and are written as 16-byte vectors below
                    epA[lane * 17 + jj] = (uint32_t)a | ((uint32_t)b << 16);
                    if (NS == 3) epB[lane * 18 + jj] = c2;
                    if (r == c) {
                      trf += x;
                      frf += x * x;
                    } else {
                      frf += 2.0f * x * x;
                    }
                  }
                }
                __syncwarp();
                {
                  // 32 rows x 16 columns of (slice0 | slice1 << 16) are staged (and
                  // slice 2 beside them): each lane writes runs of 8 values of one
                  // slice as 16-byte vectors (2-byte stores made the epilogue
                  // store-bound). Pitch and row offsets are multiples of 128, so
                  // every run is 16-byte aligned; a run that crosses the diagonal
                  // is written element by element.
                  const int cb = c0 + hh * 16;
                  auto pack = [](const uint32_t* w, bool hi) {
                    uint4 v;
                    uint32_t* pv = reinterpret_cast<uint32_t*>(&v);
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                      pv[t] = hi ? ((w[2 * t] >> 16) | (w[2 * t + 1] & 0xffff0000u))
                                 : ((w[2 * t] & 0xffffu) | (w[2 * t + 1] << 16));
                    return v;
                  };
                  // 8 slice-2 values at p, p + stride, ..., packed for one store
                  auto pack16 = [](const uint16_t* p, int stride) {
                    uint4 v;
                    uint32_t* pv = reinterpret_cast<uint32_t*>(&v);
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                      pv[t] = (uint32_t)p[2 * t * stride] | ((uint32_t)p[(2 * t + 1) * stride] << 16);
                    return v;
                  };
#pragma unroll
                  for (int q = 0; q < 2; ++q) {  // (r, c): row i, columns cb + 8 g ..
                    const int task = lane + 32 * q;
                    const int i = task >> 1, g = task & 1;
                    const int rr = rb + i, cs = cb + 8 * g;
                    if (rr <= cs + 7) {
                      uint32_t w[8];
#pragma unroll
                      for (int t = 0; t < 8; ++t) w[t] = epA[i * 17 + 8 * g + t];
                      const size_t dd = (size_t)(in.row0 + rr) * P + cs;
                      if (rr <= cs) {
                        *reinterpret_cast<uint4*>(o0 + dd) = pack(w, false);
                        *reinterpret_cast<uint4*>(o1 + dd) = pack(w, true);
                        if (NS == 3)
                          *reinterpret_cast<uint4*>(o2 + dd) = pack16(epB + i * 18 + 8 * g, 1);
                      } else {
#pragma unroll
                        for (int t = 0; t < 8; ++t)
                          if (rr <= cs + t) {
                            o0[dd + t] = (uint16_t)(w[t] & 0xffffu);
                            o1[dd + t] = (uint16_t)(w[t] >> 16);
                            if (NS == 3) o2[dd + t] = epB[i * 18 + 8 * g + t];
                          }
                      }
                    }
                  }
#pragma unroll
                  for (int q = 0; q < 2; ++q) {  // mirror (c, r): column cb + j, rows rb + 8 g ..
                    const int task = lane + 32 * q;
                    const int j = task >> 2, g = task & 3;
                    const int cc = cb + j, r0 = rb + 8 * g;
                    if (r0 < cc) {
                      uint32_t w[8];
#pragma unroll
                      for (int t = 0; t < 8; ++t) w[t] = epA[(8 * g + t) * 17 + j];
                      const size_t mi = (size_t)(in.row0 + cc) * P + r0;
                      if (r0 + 7 < cc) {
                        *reinterpret_cast<uint4*>(o0 + mi) = pack(w, false);
                        *reinterpret_cast<uint4*>(o1 + mi) = pack(w, true);
                        if (NS == 3)
                          *reinterpret_cast<uint4*>(o2 + mi) = pack16(epB + (8 * g) * 18 + j, 18);
                      } else {
#pragma unroll
                        for (int t = 0; t < 8; ++t)
                          if (r0 + t < cc) {
                            o0[mi + t] = (uint16_t)(w[t] & 0xffffu);
                            o1[mi + t] = (uint16_t)(w[t] >> 16);
                            if (NS == 3) o2[mi + t] = epB[(8 * g + t) * 18 + j];
                          }
                      }
                    }
                  }
                }
                __syncwarp();
              }
              tfix += fixed40(trf);
              ffix += fixed40(frf);
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(tempty + 8u * tb);
        }
        fence_async_global();  // this iteration's slices feed the next TMA reads
      }
      double tr = (double)tfix * 9.094947017729282e-13, fr = (double)ffix * 9.094947017729282e-13;  // 2^-40
      block_sum2(tr, fr, sh.red);  // all threads of the CTA meet here
      if (gsz > 1) {
        if (threadIdx.x == 0) xch_put(sh, xk & 1, grank, gsz, tr, fr, *err ? 1.0 : 0.0);
        cluster_sync_all();  // also publishes every CTA's slice stores to the group
        if (threadIdx.x == 0) {
          tr = 0.0;
          fr = 0.0;
          double e = 0.0;
          for (int r = 0; r < gsz; ++r) {
            tr += sh.xch[xk & 1][r][0];
            fr += sh.xch[xk & 1][r][1];
            e += sh.xch[xk & 1][r][2];
          }
          if (e != 0.0) *err = 1;
        }
        ++xk;
      }
      if (threadIdx.x == 0) {
        if (*err) {
          st.status = PROGRESS_ETIMEOUT;
          st.done = 1;
        } else {
          st.t1 = tr;
          st.t2 = fr;
          st.iter = k + 1;
          st.phase_iters[kPhaseSplit] += 1;
          decide(&st);
        }
      }
      __syncthreads();
    }

    if (predicted && !*err &&
        (st.judge_fail || st.status == PROGRESS_EBOUNDS || st.status == PROGRESS_ENOCONV)) {
      predicted = false;
      fell_back = true;
      wasted = st.iter;
      __syncthreads();
      goto restart;
    }

    // ---- D (FP64, n x n at the instance's offset) from the final slices
    {
      const int fin = st.iter & 1;
      const uint16_t* s0 = prm.sl[fin][0];
      const uint16_t* s1 = prm.sl[fin][1];
      const uint16_t* s2 = prm.sl[fin][2];
      double* D = prm.D + in.offset;
      for (int idx = grank * THREADS + threadIdx.x; idx < n * n; idx += gsz * THREADS) {
        const int r = idx / n, c = idx - r * n;
        const size_t g = (size_t)(in.row0 + r) * prm.pitch + c;
        D[idx] = (double)join_value<F>(s0[g], s1[g], NS == 3 ? s2[g] : (uint16_t)0);
      }
      if (threadIdx.x == 0 && grank == 0) {
        if (prm.iters) prm.iters[inst] = st.iter;
        if (prm.fallback) prm.fallback[inst] = fell_back ? 1 : 0;
        if (prm.products) prm.products[inst] = st.iter + wasted;
        if (prm.bits_out)
          for (int b = 0; b < 4; ++b) prm.bits_out[4 * inst + b] = st.bits[b];
        if (prm.bounds_out) {
          prm.bounds_out[2 * inst] = st.emin;
          prm.bounds_out[2 * inst + 1] = st.emax;
        }
        if (prm.status) prm.status[inst] = st.status;
        if (prm.info) {
          InstanceInfo& o = prm.info[inst];
          o.emin = st.emin;
          o.emax = st.emax;
          o.idem = st.idem;
          o.converged = st.converged;
          for (int b = 0; b < 4; ++b) o.bits[b] = st.bits[b];
        }
        if (prm.cycles) prm.cycles[inst] = clock64() - c_start;
      }
    }
    __syncthreads();
  }
  if (*err) {
    // Failure path (a bounded wait ran out): no MMA may still write tensor
    // memory and no TMA copy may still land in shared memory when the CTA
    // frees them and exits.
    if (warp == 1 && lane == 0) {
      mma_commit(drain_bar);
      mbar_wait(drain_bar, 0u, err, false, kWaitLimitNs / 10);
      sh.kb_consumed = (int)kb_mma;
    }
    __syncthreads();
    if (warp == 0 && lane == 0) {
      for (uint32_t kb = (uint32_t)sh.kb_consumed; kb < kb_prod; ++kb)
        mbar_wait(full_bar(kb % STAGES), (kb / STAGES) & 1u, err, false, kWaitLimitNs / 10);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, Cfg::TMEM_COLS);
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

void* pick_kernel(int fmt, int tile_n, int* smem) {
  if (fmt_bf16(fmt)) {
    if (tile_n == 64) {
      *smem = BCfg<kBF16x3, 64>::SMEM;
      return reinterpret_cast<void*>(&batched_kernel<kBF16x3, 64>);
    }
    *smem = BCfg<kBF16x3, 128>::SMEM;
    return reinterpret_cast<void*>(&batched_kernel<kBF16x3, 128>);
  }
  if (tile_n == 64) {
    *smem = BCfg<kFP16x2, 64>::SMEM;
    return reinterpret_cast<void*>(&batched_kernel<kFP16x2, 64>);
  }
  *smem = BCfg<kFP16x2, 128>::SMEM;
  return reinterpret_cast<void*>(&batched_kernel<kFP16x2, 128>);
}

void fill_config(cudaLaunchConfig_t& lc, cudaLaunchAttribute* attr, const Config& cfg, int grid,
                 int smem, cudaStream_t s) {
  memset(&lc, 0, sizeof lc);
  lc.gridDim = dim3((unsigned)grid, 1, 1);
  lc.blockDim = dim3(THREADS, 1, 1);
  lc.dynamicSmemBytes = (size_t)smem;
  lc.stream = s;
  memset(attr, 0, sizeof(cudaLaunchAttribute));
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cfg.cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
}

}  // namespace

bool config_ok(const Config& c) {
  return (c.tile_n == 64 || c.tile_n == 128) &&
         (c.cluster == 1 || c.cluster == 2 || c.cluster == 4 || c.cluster == 8) && c.share >= 1;
}

int grid_size(const Config& cfg, int fmt, int batch) {
  if (!config_ok(cfg) || batch < 1) return 0;
  int smem = 0;
  void* k = pick_kernel(fmt, cfg.tile_n, &smem);
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  int clusters = sms / cfg.cluster;
  if (cfg.cluster > 1) {
    cudaLaunchConfig_t lc;
    cudaLaunchAttribute attr[1];
    fill_config(lc, attr, cfg, cfg.cluster, smem, nullptr);
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, k, &lc) != cudaSuccess || nc < 1) {
      cudaGetLastError();
      return 0;
    }
    clusters = nc < clusters ? nc : clusters;
  }
  // one CTA per instance at most (rounded up to whole clusters)
  int g = clusters * cfg.cluster;
  if (g > batch) g = (batch + cfg.cluster - 1) / cfg.cluster * cfg.cluster;
  return g;
}

cudaError_t launch(const Params& prm, const Config& cfg, int grid, cudaStream_t s) {
  if (!config_ok(cfg) || grid < cfg.cluster || grid % cfg.cluster) return cudaErrorInvalidValue;
  PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
  if (!enc) return cudaErrorNotSupported;
  const bool bf = fmt_bf16(prm.fmt);
  const int ns = fmt_slices(prm.fmt);
  Maps maps;
  memset(&maps, 0, sizeof maps);
  for (int k = 0; k < 2; ++k)
    for (int j = 0; j < ns; ++j) {
      cuuint64_t dims[2] = {(cuuint64_t)prm.pitch, (cuuint64_t)prm.total_rows};
      cuuint64_t strides[1] = {(cuuint64_t)prm.pitch * 2};
      cuuint32_t estr[2] = {1, 1};
      for (int op = 0; op < 2; ++op) {
        cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)(op == 0 ? BM : cfg.tile_n)};
        CUtensorMap* mp = op == 0 ? &maps.a[k][j] : &maps.b[k][j];
        if (enc(mp, bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                (void*)prm.sl[k][j], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
          return cudaErrorInvalidValue;
      }
    }
  int smem = 0;
  void* k = pick_kernel(prm.fmt, cfg.tile_n, &smem);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t lc;
  cudaLaunchAttribute attr[1];
  fill_config(lc, attr, cfg, grid, smem, s);
  Params p = prm;
  p.share = cfg.share;
  void* args[2] = {(void*)&maps, (void*)&p};
  return cudaLaunchKernelExC(&lc, k, args);
}

}  // namespace batched
}  // namespace sp2
