// FP64 SP2 product step: X' = X*X or 2X - X*X with the traces of X' (§IV.A).
//
// Only the upper-triangle tiles of the symmetric product are computed
// (n^2 (n+1) flops instead of 2 n^3). Because X is symmetric, both operands of
// tile (I, J) are row panels of X (K-major): S_IJ = sum_k X[I, k] X[J, k]^T.
// The epilogue applies the branch chosen on the device, writes the tile and
// its mirror, emits the operand slices of the next product when the precision
// schedule needs them, and reduces Tr X' and ||X'||_F^2 (diagonal elements
// once, off-diagonal ones twice). The last CTA sums the per-tile partials in
// tile order and decides the next step.
//
// Arithmetic: FP64 DMMA (mma.sync m8n8k4 f64), the only FP64 matrix
// instruction of sm_103a; tcgen05 has no FP64 kind.
#include "sp2_common.cuh"
#include "sp2_launch.h"
#include "sp2_slices.cuh"

namespace sp2 {

namespace {

constexpr int BM = 64;        // tile edge (square tiles)
constexpr int BK = 16;        // k depth per pipeline stage
constexpr int PADK = BK + 4;  // smem row pitch in doubles (conflict-free fragment loads)
constexpr int STAGES = 3;
constexpr int THREADS = 128;  // 4 warps, 2 x 2, each 32 x 32

__device__ __forceinline__ void dmma(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// Row-major enumeration of the upper-triangle tiles (I <= J) of a T x T grid.
__device__ __forceinline__ void tri_tile(int t, int T, int& I, int& J) {
  const double b = 2.0 * T + 1.0;
  int i = (int)floor((b - sqrt(b * b - 8.0 * (double)t)) * 0.5);
  if (i < 0) i = 0;
  while (i > 0 && i * T - i * (i - 1) / 2 > t) --i;
  while ((i + 1) * T - (i + 1) * i / 2 <= t) ++i;
  I = i;
  J = i + (t - (i * T - i * (i - 1) / 2));
}

struct Smem {
  double A[STAGES][BM][PADK];
  double B[STAGES][BM][PADK];
  double scratch[2 * THREADS / 32];
  int last;
};

__device__ __forceinline__ void load_stage(Smem& sm, int stage, const double* __restrict__ X,
                                           int ld, int row_a, int row_b, int k0, bool same) {
  // 64 rows x 16 doubles per operand = 512 chunks of 16 B; 4 per thread
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int c = threadIdx.x + i * THREADS;
    const int r = c >> 3, col = (c & 7) * 2;
    cp_async16(&sm.A[stage][r][col], X + (size_t)(row_a + r) * ld + k0 + col);
    if (!same) cp_async16(&sm.B[stage][r][col], X + (size_t)(row_b + r) * ld + k0 + col);
  }
}

template <int F>
__global__ void __launch_bounds__(THREADS) square_fp64_kernel(DevBuffers buf,
                                                              unsigned long long cond) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
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
  // Slices of X' are needed when the next product will be split (MIXED, end
  // of the FP64 prefix).
  const bool want_slices =
      (prec == PROGRESS_MIXED_FP16 || prec == PROGRESS_MIXED_BF16) && phase == kPhaseFP64 &&
      (k_iter + 1 >= st->fp64_prefix);
  const double* __restrict__ X = buf.x64[k_iter & 1];
  double* __restrict__ Y = buf.x64[(k_iter + 1) & 1];
  Slices S;
  for (int i = 0; i < 3; ++i) S.s[i] = buf.sl[(k_iter + 1) & 1][i];

  const int T = ld / BM;
  int I, J;
  tri_tile(blockIdx.x, T, I, J);
  const int row_a = I * BM, row_b = J * BM;
  const bool same = (I == J);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = warp >> 1, wn = warp & 1;
  const int g = lane >> 2, t4 = lane & 3;

  double acc[4][4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;

  const int KT = ld / BK;
#pragma unroll
  for (int s = 0; s < STAGES - 1; ++s) {
    if (s < KT) load_stage(sm, s, X, ld, row_a, row_b, s * BK, same);
    cp_async_commit();
  }
  for (int kt = 0; kt < KT; ++kt) {
    cp_async_wait<STAGES - 2>();
    __syncthreads();
    const int pf = kt + STAGES - 1;
    if (pf < KT) load_stage(sm, pf % STAGES, X, ld, row_a, row_b, pf * BK, same);
    cp_async_commit();
    const int s = kt % STAGES;
    const double(*As)[PADK] = sm.A[s];
    const double(*Bs)[PADK] = same ? sm.A[s] : sm.B[s];
#pragma unroll
    for (int kk = 0; kk < BK; kk += 4) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[wm * 32 + i * 8 + g][kk + t4];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[wn * 32 + j * 8 + g][kk + t4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) dmma(acc[i][j][0], acc[i][j][1], a[i], b[j]);
    }
  }
  cp_async_wait<0>();

  // epilogue: branch, mirror store, slices, partial traces
  double tr = 0.0, fr = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = row_a + wm * 32 + i * 8 + g;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int c = row_b + wn * 32 + j * 8 + 2 * t4 + e;
        if (r > c) continue;  // covered by the mirror of the tile above the diagonal
        const double s = acc[i][j][e];
        double x = s;
        if (bit) x = 2.0 * X[(size_t)r * ld + c] - s;
        Y[(size_t)r * ld + c] = x;
        if (r != c) Y[(size_t)c * ld + r] = x;
        if (want_slices) {
          store_slices<F>(S, (size_t)r * ld + c, x);
          if (r != c) store_slices<F>(S, (size_t)c * ld + r, x);
        }
        if (r == c) {
          tr += x;
          fr += x * x;
        } else {
          fr += 2.0 * x * x;
        }
      }
    }
  }
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

int fp64_tile_count(int ld) {
  const int T = ld / BM;
  return T * (T + 1) / 2;
}

cudaError_t launch_square_fp64(const DevBuffers& b, int ld, int slice_fmt,
                               unsigned long long cond_handle, cudaStream_t s) {
  const int tiles = fp64_tile_count(ld);
  if (tiles > b.max_partials || ld % BM) return cudaErrorInvalidValue;
  const int smem = (int)sizeof(Smem);
  switch (slice_fmt) {
#define SP2_SQ64(F)                                                                        \
  case F:                                                                                  \
    cudaFuncSetAttribute(square_fp64_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                         smem);                                                            \
    square_fp64_kernel<F><<<tiles, THREADS, smem, s>>>(b, cond_handle);                    \
    break;
    SP2_SQ64(kFP16x2)
    SP2_SQ64(kBF16x3)
    SP2_SQ64(kFP16x2F)
    SP2_SQ64(kBF16x3F)
#undef SP2_SQ64
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace sp2
