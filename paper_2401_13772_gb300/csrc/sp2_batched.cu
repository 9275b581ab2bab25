// Batched SP2: thousands of independent dense sub-Hamiltonians of uneven size
// (the parts of a graph-partitioned system, §VIII.B: the parts are "solved
// for independently and concurrently") in ONE persistent kernel launch.
//
// Scheduling: one CTA per SM. A CTA takes the next instance from a device
// work queue (instances ordered by decreasing cost n^3, so the largest start
// first -- greedy longest-processing-time) and runs the whole SP2 solve of
// that instance by itself: Gershgorin bounds, the X0 map, every product tile
// of every iteration, the device-side branch/convergence decision (the same
// rule as the dense solver) and the FP64 copy of D. No CTA ever waits for
// another, so nothing spins on a global flag.
//
// Layout: every instance i is padded to m_i = round_up(n_i, 128) and stored as
// FP16x2 operand slices in "tall" matrices of pitch P = max_i m_i: instance i
// owns rows [row0_i, row0_i + m_i), columns [0, m_i). One TMA tensor map per
// slice and ping-pong set therefore serves every instance.
//
// Roles inside a CTA (256 threads), per product tile (I <= J) of an iteration:
//   warp 0 lane 0 : TMA producer into a STAGES-deep ring (continues across
//                   tiles, so the next tile's operands stream in during the
//                   current tile's epilogue)
//   warp 1 lane 0 : tcgen05.mma issuer, M = N = 128, K = 16, FP32 accumulators
//                   acc0 (hi*hi) and acc1 (hi*lo + lo*hi) in one of two tensor
//                   memory buffers (double-buffered across tiles)
//   warps 4..7    : epilogue -- S = acc0 + 2^-11 acc1, X' = S or 2X - S, the
//                   new slices of X' at (r, c) and its mirror, partial traces.
// At the end of an iteration all threads meet, the traces are reduced and the
// next step is decided; generic-proxy stores are fenced before the next
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
constexpr int TILE_BYTES = BM * BK * 2;  // one 128 x 64 slice box
constexpr int THREADS = 256;
constexpr int EPI_WARP0 = 4;             // warps 4..7 own tensor-memory lanes 0..127
constexpr int TMEM_COLS = 512;           // 2 buffers x 256 columns

// FP16x2: acc0 (hi*hi) and acc1 (hi*lo + lo*hi, weight 2^-11) per buffer.
// BF16x3: the slices carry their own magnitudes, so all six products go to
// one accumulator per buffer.
template <int F>
struct BCfg {
  static constexpr int NS = fmt_slices(F);
  static constexpr int STAGE_BYTES = 2 * NS * TILE_BYTES;
  static constexpr int STAGES = fmt_bf16(F) ? 2 : 3;
  // epilogue staging (per epilogue warp): a 32 x 33 word plane holding the
  // packed (slice0, slice1) of a 32 x 32 chunk, and for BF16x3 a 32 x 34
  // half-word plane for slice 2; used to turn row-wise results into
  // column-contiguous (coalesced) stores
  static constexpr int EPI_A = 32 * 33;
  static constexpr int EPI_B = 32 * 34;
  static constexpr int EPI_BYTES = 4 * (EPI_A * 4 + (NS == 3 ? EPI_B * 2 : 0));
  static constexpr int SMEM = STAGES * STAGE_BYTES + EPI_BYTES + 1024;
};

struct Maps {
  CUtensorMap m[2][3];  // [set][slice]
};

struct Shared {
  State st;             // control state of the instance in flight
  double red[2 * THREADS / 32];
  double lo[THREADS / 32], hi[THREADS / 32];
  uint64_t bars[2 * 3 + 5];
  int kb_consumed;
  uint32_t tmem;
  int err;
  int inst;
};

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void fence_async_global() {
  asm volatile("fence.proxy.async.global;\n" ::: "memory");
}

template <int F>
__global__ void __launch_bounds__(THREADS, 1)
    batched_kernel(const __grid_constant__ Maps maps, Params prm) {
  constexpr int NS = BCfg<F>::NS;
  constexpr int STAGES = BCfg<F>::STAGES;
  constexpr int STAGE_BYTES = BCfg<F>::STAGE_BYTES;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ Shared sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool epi = warp >= EPI_WARP0;
  const int erow = threadIdx.x - EPI_WARP0 * 32;  // tile row of an epilogue thread
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  unsigned char* const epi_base = smem_raw + (base - smem_u32(smem_raw)) + STAGES * STAGE_BYTES;
  uint32_t* const epA = reinterpret_cast<uint32_t*>(epi_base) +
                        (epi ? (warp - EPI_WARP0) * BCfg<F>::EPI_A : 0);
  uint16_t* const epB = reinterpret_cast<uint16_t*>(epi_base + 4 * BCfg<F>::EPI_A * 4) +
                        (epi ? (warp - EPI_WARP0) * BCfg<F>::EPI_B : 0);
  const uint32_t bars = smem_u32(&sh.bars[0]);
  auto full_bar = [&](int s) { return bars + 8u * s; };
  auto empty_bar = [&](int s) { return bars + 8u * (STAGES + s); };
  const uint32_t tfull = bars + 8u * (2 * STAGES);      // [2] MMA -> epilogue
  const uint32_t tempty = bars + 8u * (2 * STAGES + 2); // [2] epilogue -> MMA
  const uint32_t drain_bar = bars + 8u * (2 * STAGES + 4);  // failure path only

  if (threadIdx.x == 0) {
    sh.err = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull + 8u * b, 1);
      mbar_init(tempty + 8u * b, 4);
    }
    mbar_init(drain_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(&sh.tmem), TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh.tmem;
  volatile int* err = &sh.err;
  constexpr uint32_t idesc = idesc_f16(fmt_bf16(F) ? 1 : 0, BM, BM);

  // ring / buffer counters, each kept by the thread that uses it
  uint32_t kb_prod = 0, kb_mma = 0, tile_mma = 0, tile_epi = 0;

  for (;;) {
    if (threadIdx.x == 0) {
      const int q = atomicAdd(prm.queue, 1);
      sh.inst = q < prm.batch ? prm.order[q] : -1;
    }
    __syncthreads();
    const int inst = sh.inst;
    if (inst < 0 || *err) break;
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

    // ---- set-up: state, Gershgorin bounds, X0 (all threads)
    {
      unsigned int* w = reinterpret_cast<unsigned int*>(&st);
      for (int i = threadIdx.x; i < (int)(sizeof(State) / 4); i += THREADS) w[i] = 0u;
    }
    __syncthreads();
    double lo = INFINITY, hi = -INFINITY;
    for (int r = warp; r < n; r += THREADS / 32) {
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
      for (int w = 1; w < THREADS / 32; ++w) {
        lo = fmin(lo, sh.lo[w]);
        hi = fmax(hi, sh.hi[w]);
      }
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
      for (int r = warp; r < m; r += THREADS / 32) {
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
      block_sum2(tr, fr, sh.red);
      if (threadIdx.x == 0) {
        st.t1 = tr;
        st.t2 = fr;
        st.iter = 0;
        decide(&st);
      }
    }
    fence_async_global();
    __syncthreads();

    // ---- SP2 iterations
    while (!st.done) {
      const int k = st.iter;
      const int bit = st.bit;
      const int src = k & 1, dst = (k + 1) & 1;
      const int ntiles = T * (T + 1) / 2;
      const int KB = m / BK;
      if (warp == 0) {
        if (lane == 0) {
          for (int t = 0; t < ntiles && !*err; ++t) {
            int I, J;
            tri_tile(t, T, I, J);
            for (int kb = 0; kb < KB; ++kb, ++kb_prod) {
              const int s = kb_prod % STAGES;
              const uint32_t ph = (kb_prod / STAGES) & 1u;
              if (!mbar_wait(empty_bar(s), ph ^ 1u, err)) break;
              mbar_expect_tx(full_bar(s), STAGE_BYTES);
              const uint32_t sa = base + s * STAGE_BYTES;
              for (int j = 0; j < NS; ++j) {
                tma_load_2d(sa + j * TILE_BYTES, &maps.m[src][j], kb * BK, in.row0 + I * BM,
                            full_bar(s));
                tma_load_2d(sa + (NS + j) * TILE_BYTES, &maps.m[src][j], kb * BK,
                            in.row0 + J * BM, full_bar(s));
              }
            }
          }
        }
        __syncwarp();
      } else if (warp == 1) {
        if (lane == 0) {
          for (int t = 0; t < ntiles && !*err; ++t, ++tile_mma) {
            const uint32_t tb = tile_mma & 1u;
            if (!mbar_wait(tempty + 8u * tb, ((tile_mma >> 1) & 1u) ^ 1u, err)) break;
            tc_fence_after();
            const uint32_t acc0 = tmem + 256u * tb, acc1 = acc0 + 128u;
            for (int kb = 0; kb < KB; ++kb, ++kb_mma) {
              const int s = kb_mma % STAGES;
              const uint32_t ph = (kb_mma / STAGES) & 1u;
              if (!mbar_wait(full_bar(s), ph, err)) break;
              tc_fence_after();
              const uint32_t sa = base + s * STAGE_BYTES;
              uint64_t a[NS], b[NS];
#pragma unroll
              for (int j = 0; j < NS; ++j) {
                a[j] = smem_desc_sw128(sa + j * TILE_BYTES);
                b[j] = smem_desc_sw128(sa + (NS + j) * TILE_BYTES);
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
                  // small terms first, the leading product last
                  mma_f16(acc0, a[0] + adv, b[2 % NS] + adv, idesc, acc);
                  mma_f16(acc0, a[2 % NS] + adv, b[0] + adv, idesc, 1u);
                  mma_f16(acc0, a[1] + adv, b[1] + adv, idesc, 1u);
                  mma_f16(acc0, a[0] + adv, b[1] + adv, idesc, 1u);
                  mma_f16(acc0, a[1] + adv, b[0] + adv, idesc, 1u);
                  mma_f16(acc0, a[0] + adv, b[0] + adv, idesc, 1u);
                }
              }
              mma_commit(empty_bar(s));
            }
            mma_commit(tfull + 8u * tb);
          }
        }
        __syncwarp();
      }
      double tr = 0.0, fr = 0.0;
      if (epi) {
        const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
        const uint16_t* xs0 = prm.sl[src][0];
        const uint16_t* xs1 = prm.sl[src][1];
        const uint16_t* xs2 = prm.sl[src][2];
        uint16_t* o0 = prm.sl[dst][0];
        uint16_t* o1 = prm.sl[dst][1];
        uint16_t* o2 = prm.sl[dst][2];
        const size_t P = prm.pitch;
        for (int t = 0; t < ntiles; ++t, ++tile_epi) {
          const uint32_t tb = tile_epi & 1u;
          const bool ok = mbar_wait(tfull + 8u * tb, (tile_epi >> 1) & 1u, err);
          tc_fence_after();
          int I, J;
          tri_tile(t, T, I, J);
          const int r = I * BM + erow;  // row within the instance
          if (ok && !*err) {
#pragma unroll 1
            for (int ch = 0; ch < BM / 32; ++ch) {
              float v0[32], v1[32];
              tmem_ld32(tmem + lane_base + 256u * tb + ch * 32, v0);
              if (NS == 2) tmem_ld32(tmem + lane_base + 256u * tb + 128u + ch * 32, v1);
              tmem_ld_wait();
              const int c0 = J * BM + ch * 32;
              float trf = 0.0f, frf = 0.0f;
#pragma unroll
              for (int j = 0; j < 32; ++j) {
                const int c = c0 + j;
                float x = (NS == 2) ? v0[j] + v1[j] * (1.0f / 2048.0f) : v0[j];
                if (bit) {
                  const size_t mi = (size_t)(in.row0 + c) * P + r;
                  x = 2.0f * join_value<F>(xs0[mi], xs1[mi], NS == 3 ? xs2[mi] : (uint16_t)0) - x;
                }
                if (r <= c) {
                  uint16_t a, b, c2;
                  split_value_f<F>(x, a, b, c2);
                  // (r, c) goes through the staging planes; its mirror
                  // (c, r) is already contiguous across the warp's lanes
                  epA[lane * 33 + j] = (uint32_t)a | ((uint32_t)b << 16);
                  if (NS == 3) epB[lane * 34 + j] = c2;
                  if (r == c) {
                    trf += x;
                    frf += x * x;
                  } else {
                    frf += 2.0f * x * x;
                    const size_t mi = (size_t)(in.row0 + c) * P + r;
                    o0[mi] = a;
                    o1[mi] = b;
                    if (NS == 3) o2[mi] = c2;
                  }
                }
              }
              tr += (double)trf;
              fr += (double)frf;
              // rows of the chunk, one per store instruction, lanes along c
              __syncwarp();
              const int rb = I * BM + (warp - EPI_WARP0) * 32;
              const int cc = c0 + lane;
#pragma unroll 4
              for (int i = 0; i < 32; ++i) {
                if (rb + i <= cc) {
                  const uint32_t v = epA[i * 33 + lane];
                  const size_t dd = (size_t)(in.row0 + rb + i) * P + cc;
                  o0[dd] = (uint16_t)(v & 0xffffu);
                  o1[dd] = (uint16_t)(v >> 16);
                  if (NS == 3) o2[dd] = epB[i * 34 + lane];
                }
              }
              __syncwarp();
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(tempty + 8u * tb);
        }
        fence_async_global();  // this iteration's slices feed the next TMA reads
      }
      block_sum2(tr, fr, sh.red);  // all threads meet here
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

    if (predicted && !*err && (st.judge_fail || st.status == PROGRESS_EBOUNDS ||
                               st.status == PROGRESS_ENOCONV)) {
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
      for (int idx = threadIdx.x; idx < n * n; idx += THREADS) {
        const int r = idx / n, c = idx - r * n;
        const size_t g = (size_t)(in.row0 + r) * prm.pitch + c;
        D[idx] = (double)join_value<F>(s0[g], s1[g], NS == 3 ? s2[g] : (uint16_t)0);
      }
      if (threadIdx.x == 0) {
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
  if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
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

}  // namespace

cudaError_t launch(const Params& prm, int grid, cudaStream_t s) {
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
      cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)BM};
      cuuint32_t estr[2] = {1, 1};
      if (enc(&maps.m[k][j], bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
              2, (void*)prm.sl[k][j], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    }
  if (bf) {
    cudaFuncSetAttribute(batched_kernel<kBF16x3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         BCfg<kBF16x3>::SMEM);
    batched_kernel<kBF16x3><<<grid, THREADS, BCfg<kBF16x3>::SMEM, s>>>(maps, prm);
  } else {
    cudaFuncSetAttribute(batched_kernel<kFP16x2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         BCfg<kFP16x2>::SMEM);
    batched_kernel<kFP16x2><<<grid, THREADS, BCfg<kFP16x2>::SMEM, s>>>(maps, prm);
  }
  return cudaGetLastError();
}

}  // namespace batched
}  // namespace sp2
