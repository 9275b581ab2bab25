/*
 * progress_sp2.h -- C ABI of the GB300 (sm_103a) SP2 density-matrix solver.
 *
 * The operation (arXiv 2401.13772):
 *   §III   D = V f V^T, the zero-temperature density matrix of a symmetric H
 *          with Nocc occupied states (the insulating limit: f = 1 below the
 *          gap, 0 above).
 *   §IV.A  SP2 reaches that D with matrix products only: X0 = (emax I - H) /
 *          (emax - emin), then X <- X^2 when the trace is above Nocc and
 *          X <- 2X - X^2 when it is below, until X is idempotent (Listing 1,
 *          prg_sp2, gives the loop).
 *   §VIII.A  emin, emax come from Gershgorin circles.
 *
 * Conventions shared by every entry point
 *   - Matrices are dense, real, FP64, square n x n, row-major with leading
 *     dimension n. H and D are symmetric, so row-major equals column-major.
 *   - All matrix pointers are DEVICE pointers owned by the caller, except where
 *     a comment says host. The library never frees caller memory.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Every call is
 *     asynchronous on that stream unless its comment says it synchronizes.
 *   - Work buffers (ping-pong iterates, operand slices, partial traces) are
 *     allocated by the library on first use per (device, stream) and cached;
 *     progress_release() frees them. Calls on one stream are serialized by the
 *     stream; concurrent calls on different streams use different workspaces.
 *   - Nothing aborts. Each call returns a progress_status_t; argument errors
 *     are reported before any work is queued. A failed CUDA call returns
 *     PROGRESS_ECUDA and progress_last_error() describes it.
 *   - The GPU decides each SP2 branch and the stopping point itself: no host
 *     round trip per iteration (the paper's listing reads the trace on the host
 *     every iteration).
 */
#ifndef PROGRESS_SP2_H
#define PROGRESS_SP2_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PROGRESS_OK = 0,
  PROGRESS_EINVAL = 1,      /* bad argument (sizes, nocc outside [0, n], NULL pointer) */
  PROGRESS_ENOCONV = 2,     /* maxiter products without reaching tol; D holds the last iterate */
  PROGRESS_EBOUNDS = 3,     /* the iterate left [0, 1] (bounds do not enclose the spectrum) or is not finite */
  PROGRESS_ECUDA = 4,       /* a CUDA runtime call failed */
  PROGRESS_ENOMEM = 5,      /* device workspace allocation failed */
  PROGRESS_ETIMEOUT = 6,    /* a bounded device-side wait gave up */
  PROGRESS_EUNSUPPORTED = 7 /* the requested mode is not available on this device */
} progress_status_t;

/* Arithmetic of the squarings X*X. Traces, branch decisions, the convergence
 * test and the bounds are FP64 in every mode. */
typedef enum {
  PROGRESS_FP64 = 0,        /* every product in FP64 */
  PROGRESS_FP32_SPLIT = 1,  /* every product as fp16 hi+lo operand splits on tcgen05 tensor
                               cores with FP32 accumulation (~FP32 accuracy) */
  PROGRESS_MIXED_FP16 = 2,  /* fp64_prefix FP64 products, then fp16 hi+lo split products, then
                               FP64 refinement products until idempotent in FP64 */
  PROGRESS_MIXED_BF16 = 3,  /* as MIXED_FP16 with bf16 hi+mid+lo (3-way) splits */
  PROGRESS_FP32_SPLIT_BF16 = 4, /* as FP32_SPLIT with bf16 hi+mid+lo splits: six products
                               instead of three, but FP32's exponent range (fp16 slices
                               flush entries below ~6e-8, which runs with nocc << n reach
                               by repeated squaring) */
  PROGRESS_DF64 = 5         /* every product in double-float (pairs of FP32, ~47 bits) on
                               the FP32 pipe: FP64-class accuracy, several times the FP64
                               pipe's rate on this part */
} progress_prec_t;

typedef enum {
  PROGRESS_RULE_NEARER = 0, /* take the branch whose trace lands nearer Nocc; needs no extra
                               work because Tr X^2 = ||X||_F^2 is known before the product */
  PROGRESS_RULE_PAPER = 1,  /* 2X - X^2 iff Tr X - Nocc <= 0 (Listing 1's test) */
  PROGRESS_RULE_MU = 2      /* batched and graph solves only: D = theta(mu I - H) at a given
                               chemical potential mu instead of a given Nocc. The X0 map sends
                               mu to y = (emax - mu) / (emax - emin) (bounds widened to
                               mu -/+ 1 if they do not hold mu strictly inside); each product
                               is X^2 if y > 1/2, else 2X - X^2, and y follows the same map */
} progress_rule_t;

typedef struct {
  int32_t prec;         /* progress_prec_t */
  int32_t rule;         /* progress_rule_t */
  int32_t fp64_prefix;  /* MIXED_*: FP64 products before the split phase (default 12) */
  int32_t maxiter;      /* cap on products (default 100, at most 250) */
  double emin, emax;    /* spectral bounds; NaN (default) = Gershgorin estimate */
  int32_t loop_mode;    /* 0 = CUDA graph with a device-side WHILE node (default),
                           1 = maxiter plain launches that exit early once done */
  int32_t slice_fixed;  /* split operand encoding: 0 = floating-point hi/lo slices
                           (default), 1 = fixed-point slices (exact FP32 accumulation
                           of the leading hi*hi group; absolute, not relative, precision) */
  void* loop_events[2]; /* optional cudaEvent_t pair (or NULL) recorded on the stream
                           right before and right after the product loop, so a
                           caller can time the products alone */
  int32_t fp64_impl;    /* MIXED_*: arithmetic of the FP64-accurate products (prefix and
                           refinement): 0 = library default (3 for n <= 8192, else 2),
                           1 = native FP64 (DMMA), 2 = double-float on the FP32 pipe,
                           3 = exact products of BF16 fixed-point digits on the tensor
                           cores (Ozaki scheme; ~2^-40 absolute accuracy; n <= 8192, else
                           PROGRESS_EUNSUPPORTED) */
  float tau;            /* cutoff of thresholded SP2 (Listing 1's tau): every product X*X and
                           every 2X - X^2 drops the elements with |x| < tau; X0 is not
                           pruned. 0 (default) = dense. tau > 0 needs prec FP32_SPLIT or
                           FP32_SPLIT_BF16 (else EINVAL); the product then skips every
                           128 x 128 block pair of X that holds no non-zero and leaves a
                           result tile that stays zero unwritten */
  int32_t wait_limit_us; /* bound on each pipeline wait (mbarrier) of the tensor-core product
                           kernels, in microseconds; 0 (default) = 2 s. A wait that runs out
                           ends the solve with PROGRESS_ETIMEOUT (D is then not valid): the
                           kernel stops its loads and products, lets copies already in flight
                           land and frees its tensor memory before it exits */
  int32_t stall_test;   /* fault-injection test of those bounded waits: 0 (default) = off;
                           1 = the first CTA of the first tensor-core product waits on a
                           barrier that nothing arrives on, so the solve must end with
                           PROGRESS_ETIMEOUT after wait_limit_us. Needs a mode with
                           tensor-core products (not FP64 or DF64), else PROGRESS_EINVAL */
  int32_t split_tile;   /* tile of the dense FP16 split products (FP32_SPLIT, MIXED_FP16):
                           0 (default) or 1 = 128 x 128 tiles; 2 = 128 x 256 tiles (one
                           tensor-core product of N = 256, so the 128-row operand is read
                           once per 256 columns; slower on GB300: 1.26 against 1.13 ms
                           per product at n = 8192). Both issue the same products per
                           element in the same order: D is the same bit for bit. Other
                           values: PROGRESS_EINVAL; ignored by the other modes */
  int32_t prefix_full;  /* MIXED_* with digit products (fp64_impl 3, the default up to
                           n = 8192): 0 (default) = the FP64-accurate prefix products take
                           13 of the 15 digit products: x0 x4^T + x4 x0^T is dropped, at
                           most 2 sqrt(n) 2^-36 per entry (random sign, ~1e-11), and digit
                           4 is not loaded; the refinement always takes all 15 (~2^-40).
                           1 = all 15 in the prefix too. Other values: PROGRESS_EINVAL */
} progress_opts_t;

/* Result of one solve, read back from the device by the calls that take it. */
typedef struct {
  int32_t status;        /* progress_status_t of the solve */
  int32_t iters;         /* products performed */
  int32_t converged;     /* 1 if |Tr X^2 - Tr X| < tol was reached; 2 (MIXED modes) if the
                            refinement stopped on the round-off floor of its FP64-accurate
                            products before reaching tol: |Tr X^2 - Tr X| < 2 n u and
                            |Tr X - nocc| < n u / 2 (u = 2^-40 for digit products, 2^-44
                            double-float, 2^-52 native FP64), or two refinement products
                            that did not halve |Tr X^2 - Tr X|. The reached
                            value is in `idempotency`; the status is still PROGRESS_OK */
  int32_t phase_iters[3];/* products in FP64 prefix / split phase / FP64 refinement */
  double emin, emax;     /* bounds used */
  double trace;          /* Tr D */
  double idempotency;    /* |Tr D^2 - Tr D| of the returned D */
  uint64_t bits[4];      /* branch of product k is bit (k % 64) of bits[k / 64]; 1 = 2X - X^2 */
  uint64_t kblocks;      /* thresholded SP2 (tau > 0): 128 x 128 x 64 tile steps streamed over
                            all products (a dense product streams T (T + 1) / 2 x ld / 64 of
                            them, ld = n rounded up to 128, T = ld / 128); 0 otherwise */
} progress_info_t;

/* Fill *opts with the defaults listed above. */
void progress_opts_default(progress_opts_t* opts);

/*
 * Gershgorin enclosure of the spectrum of the symmetric H (§VIII.A; the emin,
 * emax that Listing 1 uses): R_i = sum_{j != i} |H_ij|,
 * *d_emin = min_i (H_ii - R_i), *d_emax = max_i (H_ii + R_i).
 *   dH              device, n x n FP64 row-major, read only
 *   d_emin, d_emax  device, one double each, written
 * Asynchronous. Errors: EINVAL if n < 1 or a pointer is NULL.
 */
progress_status_t progress_gershgorin_bounds(const double* dH, int64_t n, double* d_emin,
                                             double* d_emax, void* stream);

/*
 * SP2 density matrix with default options (FP64 products, nearer rule,
 * Gershgorin bounds, maxiter 100). Asynchronous: the convergence status of
 * the solve is available from progress_sp2_query().
 *   dH    device, n x n FP64, read only (H is never written)
 *   n     matrix order, >= 0 (n = 0 is a no-op)
 *   nocc  occupied states (spin factor excluded), 0 <= nocc <= n
 *   tol   stop once |Tr X^2 - Tr X| < tol (tol >= 0)
 *   dD    device, n x n FP64, written; must not overlap dH
 * Errors: EINVAL for bad sizes/pointers; ENOMEM; ECUDA.
 */
progress_status_t progress_sp2_dense(const double* dH, int64_t n, int64_t nocc, double tol,
                                     double* dD, void* stream);

/*
 * SP2 with options. If info is not NULL the call synchronizes the stream,
 * fills *info (host memory) and returns the solve's status (ENOCONV, EBOUNDS
 * ...); otherwise it is asynchronous like progress_sp2_dense. opts may be NULL
 * (defaults). dD may equal dH (in place) in this entry point only.
 * Errors: as progress_sp2_dense, plus EUNSUPPORTED when a split-precision mode
 * is asked on a device without tcgen05 tensor cores (sm_100 family).
 */
progress_status_t progress_sp2_dense_ex(const double* dH, int64_t n, int64_t nocc, double tol,
                                        double* dD, const progress_opts_t* opts,
                                        progress_info_t* info, void* stream);

/*
 * FP64 SP2 solve (same arithmetic and defaults as progress_sp2_dense) that
 * allocates no memory at all. The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc -- applications whose own
 * memory pool already owns the whole device, so an allocation by the library
 * would fail or fragment it, and time-stepping codes (QMD calls the solver
 * every step) that must not pay allocation latency or the device-wide
 * synchronization of cudaFree. The caller still passes H and D.
 *   Limit: n <= 1024; larger n returns PROGRESS_EINVAL.
 *   Work space: one static device array of about 16.1 MiB inside the library
 *   (every GPU that loads the library holds it until the process exits). Its
 *   device address is looked up on the first call on each device, so make
 *   that first call before any stream capture begins.
 *   Every call shares that array and it keeps the previous call's contents;
 *   the solve clears what has to start at zero. Calls whose work overlaps on
 *   the GPU (e.g. on two streams at once) race on it: serialize them.
 *   Asynchronous on `stream`; no status readback (no host-side state).
 */
progress_status_t progress_sp2_dense_noalloc(const double* dH, int64_t n, int64_t nocc,
                                             double tol, double* dD, void* stream);

/*
 * Batched SP2: `batch` independent dense problems of uneven size -- the parts
 * of a graph-partitioned system, which are independent and solved concurrently
 * (§VIII.B) -- in one persistent kernel launch (captured once in a CUDA graph
 * and replayed while the batch layout and pointers stay the same). Instances
 * are taken largest first from a device work queue by thread-block clusters:
 * a large instance by a whole cluster (its product tiles spread over the
 * cluster's CTAs, traces exchanged through distributed shared memory), a
 * small one by a single CTA, which runs its full SP2 loop (split FP16 hi+lo
 * products on tcgen05 tensor cores, FP32 accumulation, FP64 traces and
 * decisions). The tile shape, cluster size and sharing threshold are the
 * ones progress_sp2_batched_tune chose for this batch signature, else a
 * default (largest part below 1024: 128 x 64 tiles, clusters of 2, sharing
 * from 2 row blocks of 128; otherwise 128 x 128 tiles, clusters of 2, sharing
 * from 3 row blocks); the _ex entry point can set them explicitly.
 *   h_n, h_offset, h_nocc  HOST arrays [batch]: order n_i (1..4096), element
 *                          offset of instance i in dH/dD, occupied states
 *   dH  device, packed FP64 inputs: instance i is n_i x n_i row-major at
 *       dH + h_offset[i]; read only
 *   dD  device, packed outputs with the same layout; written
 *   d_iters, d_status  device int32 [batch] or NULL: products performed and
 *       progress_status_t per instance (-1 if the instance was not reached)
 *   opts  NULL or prec = PROGRESS_FP32_SPLIT (fp16 hi+lo) or
 *         PROGRESS_FP32_SPLIT_BF16 (bf16 hi+mid+lo), rule, maxiter; other fields
 *         ignored
 * Asynchronous on `stream`. Errors: EINVAL (bad sizes), EUNSUPPORTED (other
 * precisions or a GPU without tcgen05), ENOMEM, ECUDA.
 */
progress_status_t progress_sp2_batched(int32_t batch, const int32_t* h_n, const int64_t* h_offset,
                                       const int32_t* h_nocc, const double* dH, double tol,
                                       double* dD, int32_t* d_iters, int32_t* d_status,
                                       const progress_opts_t* opts, void* stream);

/* Learned-sequence inputs and outputs of a batched solve (all optional). */
typedef struct {
  const double* d_bounds;      /* device [batch][2]: emin, emax to use for X0 (NaN = Gershgorin) */
  const uint64_t* d_pred_bits; /* device [batch][4]: predicted branch of product k = bit k */
  const int32_t* d_pred_len;   /* device [batch]: number of predicted branches */
  double judge_delta;          /* a predicted branch that disagrees with the trace rule by a
                                  margin > judge_delta (trace units) rejects the prediction */
  uint64_t* d_bits_out;        /* device [batch][4]: branches taken, or NULL */
  double* d_bounds_out;        /* device [batch][2]: bounds used, or NULL */
  int32_t* d_fallback;         /* device [batch]: 1 if the instance reverted to the plain
                                  path (Gershgorin bounds, trace rule), or NULL */
  int32_t* d_products;         /* device [batch]: products executed in total, including a
                                  rejected predicted run (d_iters counts the final run only),
                                  or NULL */
  int32_t tile_n;              /* launch configuration (0 = the tuned or default one): product
                                  tile width, 64 or 128 (tiles are 128 x tile_n) */
  int32_t cluster;             /* CTAs per thread-block cluster: 1, 2, 4 or 8 */
  int32_t share;               /* an instance of at least `share` 128-row blocks is solved by
                                  a whole cluster (tiles dealt to its CTAs), a smaller one by
                                  one CTA; >= 1 */
  int32_t reserved0;           /* must be zero */
  int64_t* d_cycles;           /* device [batch]: SM clock cycles spent on each instance (by
                                  the CTA that owns it, or cluster rank 0), or NULL */
  const double* d_mu;          /* device [batch]: chemical potential of each instance; needed
                                  with opts->rule = PROGRESS_RULE_MU (h_nocc is then ignored),
                                  else NULL */
} progress_batch_ex_t;

/*
 * progress_sp2_batched with learned inputs. An instance given predicted
 * bounds and/or branch bits runs SP2 with them; the trace rule is still
 * evaluated at every product and judges each predicted branch. On a
 * disagreement beyond judge_delta, or if the run leaves [0, 1] or does not
 * converge, that instance alone restarts from X0 with Gershgorin bounds and
 * the plain trace-driven rule (d_fallback = 1).
 */
progress_status_t progress_sp2_batched_ex(int32_t batch, const int32_t* h_n,
                                          const int64_t* h_offset, const int32_t* h_nocc,
                                          const double* dH, double tol, double* dD,
                                          int32_t* d_iters, int32_t* d_status,
                                          const progress_opts_t* opts,
                                          const progress_batch_ex_t* ex, void* stream);

/*
 * Autotuner of the batched solver's launch configuration. No part of the
 * paper corresponds to it: it picks the tile shape (128 x 64 or 128 x 128
 * product tiles), the cluster size (1, 2, 4 or 8 CTAs) and the sharing
 * threshold of progress_sp2_batched for a batch by timing candidate
 * configurations on the GPU.
 *   Arguments as progress_sp2_batched (H and D as there; D is overwritten for
 *   the instances of the sample). sample_stride >= 1: the calibration runs on
 *   every sample_stride-th instance in size order (1 = the whole batch).
 *   The best configuration is cached in the library under the batch's size
 *   signature (device, slice format, largest padded order, log2 of the batch
 *   size); later progress_sp2_batched(_ex) calls with the same signature and
 *   no explicit configuration use it.
 *   out (host, may be NULL): the chosen configuration and each candidate's
 *   time per launch (milliseconds, median of `reps` timed launches after one
 *   untimed one).
 * Synchronizes the stream (it measures with CUDA events). Errors as
 * progress_sp2_batched.
 */
typedef struct {
  int32_t tile_n, cluster, share; /* chosen configuration */
  int32_t ncand;                   /* candidates timed (<= 16) */
  int32_t cand[16][3];             /* tile_n, cluster, share of each candidate */
  float ms[16];                    /* time per launch of each candidate */
} progress_batch_tune_t;

progress_status_t progress_sp2_batched_tune(int32_t batch, const int32_t* h_n,
                                            const int64_t* h_offset, const int32_t* h_nocc,
                                            const double* dH, double tol, double* dD,
                                            const progress_opts_t* opts, int32_t sample_stride,
                                            int32_t reps, progress_batch_tune_t* out,
                                            void* stream);

/*
 * Graph-based divide-and-conquer density matrix (§VIII.B): P ~ theta(mu I - H)
 * for a large H from small dense parts.
 *   1. adjacency of the auxiliary matrix G (H itself, an overlap matrix, or a
 *      previously computed density matrix): A_ij = |G_ij| >= tau, i != j;
 *   2. core partition: nparts regular segments of the index list (part k
 *      holds [floor(k n / nparts), floor((k + 1) n / nparts)));
 *   3. core-halo parts: each core plus every node adjacent to it;
 *   4. the dense submatrices H[part, part], solved together in one batched
 *      SP2 launch at the chemical potential mu (PROGRESS_RULE_MU; precision
 *      from opts->prec, FP32_SPLIT or FP32_SPLIT_BF16; NULL = FP32_SPLIT);
 *   5. the columns of each core copied into P, then P = (P + P^T) / 2.
 *   dH, dG  device n x n row-major FP64 (read only); dD device n x n output
 *   (must not overlap dH or dG). A part may hold at most 4096 nodes
 *   (PROGRESS_EUNSUPPORTED otherwise). info (host, may be NULL): part
 *   statistics. Synchronizes the stream (the part layout is built on the
 *   host from the adjacency rows). The part buffers are cached per (device,
 *   stream) like the other work spaces.
 */
typedef struct {
  int32_t nparts;       /* parts solved */
  int32_t max_part;     /* largest core-halo part (nodes) */
  double mean_part;     /* mean core-halo part size */
  int32_t max_iters;    /* most SP2 products of a part */
  int32_t failed_parts; /* parts whose SP2 status was not PROGRESS_OK */
  int64_t sub_elements; /* elements of all dense submatrices */
} progress_graph_info_t;

progress_status_t progress_sp2_graph(const double* dH, const double* dG, int64_t n, double tau,
                                     int32_t nparts, double mu, double tol, double* dD,
                                     const progress_opts_t* opts, progress_graph_info_t* info,
                                     void* stream);

/*
 * Finite-temperature density matrix by the Chebyshev Fermi-operator expansion
 * (§IV.B) in the Paterson-Stockmeyer form (Eqs. 7-11):
 *   D = f(H),  f(e) = 1 / (1 + exp(beta (e - mu)))  (§III, at a known mu),
 *   Ht = (H - a I) / b with a, b the midpoint and half-width of the bounds,
 *   f(b x + a) ~ sum_{n<=L} c_n T_n(x), L + 1 = k m, c_n from interpolation at
 *   the 2 (L + 1) Chebyshev-Gauss nodes (no damping kernel),
 *   D = S_0 + T_k (S_1 + T_k (... + T_k S_{m-1})), S_j = sum_{i<k} d_ij T_i,
 *   with d_ij from dividing the series by T_k (T_n = 2 T_k T_{n-k} - T_{|2k-n|}).
 * T_2..T_k come from T_n = 2 T_a T_b - T_{a-b} (a = ceil(n/2), b = floor(n/2)),
 * all T_n of one doubling level in one launch; then the m - 1 nested products.
 * Matrix products: (k - 1) + (m - 1) (k - 2 when m = 1), against L for the
 * serial recursion of Eq. 6.
 *   dH        device, n x n FP64 symmetric, read only
 *   n         1 <= n <= 32768
 *   mu, beta  chemical potential (finite) and inverse temperature (finite,
 *             >= 0), in the units of H
 *   k, m      1..64 each. Stability: the nested sums grow like
 *             info->growth; keep k >= m (k of about 2 sqrt(L) or more) for a
 *             sharp Fermi function
 *   prec      PROGRESS_FP32_SPLIT: fp16 hi+lo operand slices on the tensor
 *             cores, FP32 accumulate (leading group summed every 64 k);
 *             PROGRESS_FP32_SPLIT_BF16: bf16 hi+mid+lo slices (six products per
 *             tile step instead of three). Any other value: EINVAL. The error
 *             of D is about (growth) (beta b / 4) 2^-23 with b the half-width
 *             of the bounds: the Fermi function's slope times the FP32-class
 *             product error
 *   h_bounds  HOST, 2 doubles {emin, emax} enclosing the spectrum, or NULL for
 *             the Gershgorin bounds (one device-to-host read of 2 doubles)
 *   dD        device, n x n FP64, written (must not be dH)
 *   info      host, optional: bounds used, Tr D, growth, products, launches,
 *             |c_L| (truncation indicator)
 * Synchronizes the stream before it returns (the work buffers of a previous
 * call on the stream are reused; info is read back).
 * Errors: EINVAL (sizes, k, m, prec, beta < 0, non-finite mu or bounds, NULL
 * pointers, dD == dH), EUNSUPPORTED (not an sm_10x GPU), ENOMEM,
 * ETIMEOUT (a bounded device wait gave up; D is not valid), ECUDA.
 */
typedef struct {
  double emin, emax;    /* bounds used (before a zero-width interval is widened by 1) */
  double trace;         /* Tr D: the electron count at mu (spin factor excluded) */
  double growth;        /* sum over j of sum_i |d_ij|: bound on the nested sums' norms */
  double coef_last;     /* |c_L|, the last expansion coefficient */
  int32_t products;     /* matrix products performed */
  int32_t launches;     /* kernel launches */
} progress_cheb_info_t;

progress_status_t progress_cheb_fermi(const double* dH, int64_t n, double mu, double beta,
                                      int32_t k, int32_t m, int32_t prec,
                                      const double* h_bounds, double* dD,
                                      progress_cheb_info_t* info, void* stream);

/*
 * The schedule progress_cheb_fermi runs for bounds {emin, emax} (host only, no
 * GPU): every matrix lives in a stack slot (T_i in slot i - 1, S_j in slot
 * k + j, nested results in slots k + m and k + m + 1). Product q computes
 *   C = alpha sab (A B) + beta se E + gamma I   (E term absent if e < 0)
 * from the stored (scaled) A, B, E and stores C * inv_sc in slot c, or writes
 * D (c < 0). Launch order: T_1 = (H - a I) / b in slot 0, the T-level product
 * launches, the S_j pass (S_j stored as S_j * inv_s[j]; with m = 1 it writes D),
 * then the nested product launches; products sharing a launch index read only
 * slots written by earlier launches.
 *   cap     capacity of prods / params in products ((k - 1) + (m - 1) suffice)
 *   prods   host int32 [cap][5]: a, b, e, c, launch index
 *   params  host float [cap][6]: alpha, sab, beta, se, gamma, inv_sc
 *   dcoef   host double [k m]: d_ij at i m + j;  inv_s: host double [m]
 *   ab      host double [2]: a, b;  counts: host int32 [4]: products, product
 *           launches, slots, T-level products
 * Errors: EINVAL (k, m, mu, beta, bounds, NULL pointers, cap too small).
 */
/*
 * Copy one operand slice of one stack slot of the last progress_cheb_fermi
 * solve on `stream` (ld x ld uint16, ld = n rounded up to 128, row-major) into
 * host_out, for inspection of the intermediate T_i, S_j and nested results
 * (slot layout as in progress_cheb_plan; slice 0 = hi, 1 = lo (fp16) or mid,
 * 2 = lo (bf16); value = scale * (hi + lo / 2048) for fp16, scale * (hi + mid +
 * lo) for bf16, the slot's scale from the plan). Synchronizes the stream.
 * Errors: EINVAL (no solve on the stream, slot or slice out of range, NULL).
 */
progress_status_t progress_cheb_slot(int32_t slot, int32_t slice, uint16_t* host_out,
                                     void* stream);

progress_status_t progress_cheb_plan(int32_t k, int32_t m, double mu, double beta, double emin,
                                     double emax, int32_t cap, int32_t* prods, float* params,
                                     double* dcoef, double* inv_s, double* ab, int32_t* counts);

/*
 * Choice of the Paterson-Stockmeyer split for progress_cheb_fermi (host only,
 * no GPU): among the splits k m >= terms (k = 1..64, m = ceil(terms / k) <= 64)
 * whose nested sums stay bounded -- the plan's growth sum_ij |d_ij| <=
 * max_growth, since a large growth multiplies the products' rounding error --
 * the one whose plan (progress_cheb_plan) has the fewest matrix products, ties
 * to fewer terms. Writes k, m and (if not NULL) the product count and growth.
 * Errors: EINVAL (terms outside [1, 4096], bad mu, beta or bounds, max_growth
 * <= 0, no split qualifies).
 */
progress_status_t progress_cheb_choose(int32_t terms, double mu, double beta, double emin,
                                       double emax, double max_growth, int32_t* k_out,
                                       int32_t* m_out, int32_t* products_out,
                                       double* growth_out);

/*
 * Features of the learned predictor, 37 floats per instance (device output
 * [batch][37]): Gershgorin emin/w, emax/w (w = emax - emin, §VIII.A),
 * Tr H/(n w), ||H||_F/(sqrt(n) w), a 32-bin histogram of diag(H) over
 * [emin, emax] divided by n, and n/2048. d_n, d_offset are DEVICE arrays,
 * H packed as for progress_sp2_batched.
 */
progress_status_t progress_features(int32_t batch, const int32_t* d_n, const int64_t* d_offset,
                                    const double* dH, float* d_feat, void* stream);

/* d_out[i] = Tr(H_i D_i) for packed symmetric H and D (device arrays). With D
 * the projector onto the lowest state (nocc = 1) this is that state's energy. */
progress_status_t progress_trace_hd(int32_t batch, const int32_t* d_n, const int64_t* d_offset,
                                    const double* dH, const double* dD, double* d_out,
                                    void* stream);

/*
 * The predictor: a perceptron in -> hidden (ReLU) -> hidden (ReLU) -> out.
 * Parameters are one flat FP32 vector: W1 [hidden][in], b1, W2 [hidden][hidden],
 * b2, W3 [out][hidden], b3. Outputs 0 and 1 are the bound fractions
 * u_min = (eps_1 - emin)/w and u_max = (emax - eps_N)/w; outputs 2.. are the
 * logits of the branch bits. The loss (mean over the batch) is
 *   sum_{j<2} c (y_j - t_j)^2, c = 10 if y_j > t_j else 1   (over-shooting a
 *   bound would cut the spectrum)
 * + sum_{j>=2} mask_j BCE_with_logits(y_j, t_j) / max(1, sum_j mask_j).
 */
int32_t progress_mlp_param_count(int32_t in, int32_t hidden, int32_t out);
/* Floats of device scratch that progress_mlp_train_step / _forward need. */
int64_t progress_mlp_scratch_floats(int32_t in, int32_t hidden, int32_t out, int32_t batch);
/* FP16 copy of the parameters (the inference weights). */
progress_status_t progress_mlp_to_fp16(const float* d_params, int32_t count,
                                       uint16_t* d_params_fp16, void* stream);
/* y = mlp(x) with FP16 weights, FP32 arithmetic; x [batch][in], y [batch][out]. */
progress_status_t progress_mlp_forward(int32_t in, int32_t hidden, int32_t out,
                                       const uint16_t* d_params_fp16, int32_t batch,
                                       const float* d_x, float* d_y, float* d_scratch,
                                       void* stream);
/* One training step: forward, loss (d_loss, 1 float, may be NULL), gradient
 * into d_grad, then Adam (beta 0.9/0.999, eps 1e-8, bias-corrected with
 * `step` >= 1) on d_params with moments d_m, d_v. lr = 0 computes the
 * gradient only. All arrays are device FP32. */
progress_status_t progress_mlp_train_step(int32_t in, int32_t hidden, int32_t out,
                                          float* d_params, float* d_grad, float* d_m,
                                          float* d_v, int32_t step, float lr, int32_t batch,
                                          const float* d_x, const float* d_target,
                                          const float* d_mask, float* d_scratch, float* d_loss,
                                          void* stream);

/*
 * Solve inputs of the learned sequence (a12) from the predictor's outputs,
 * one row of `nout` floats per instance (device d_y [batch][nout]: u_min, u_max,
 * then nout - 2 <= 256 branch logits), and the Gershgorin enclosure of each
 * instance (device d_gersh [batch][2], §VIII.A), w = emax - emin:
 *   d_bounds [batch][2] (device, written): emin + w max(u_min - margin, 0) and
 *     emax - w max(u_max - margin, 0), each operation rounded on its own (no
 *     fused multiply-add); an empty interval is replaced by the enclosure, so
 *     the bounds never leave it;
 *   d_bits [batch][4] (device, written, or NULL): branch k = bit k, 1 (2X - X^2)
 *     iff logit k > 0;
 *   d_len [batch] (device, written, or NULL): the number of leading logits with
 *     |logit| >= logit_tau -- the predicted prefix; later branches are left to
 *     the trace rule.
 * These are the d_bounds, d_pred_bits, d_pred_len of progress_batch_ex_t.
 * Asynchronous. Errors: EINVAL (batch < 0, nout outside [3, 258], margin < 0 or
 * not finite, NULL pointer).
 */
progress_status_t progress_learned_inputs(int32_t batch, int32_t nout, const float* d_y,
                                          const double* d_gersh, double margin, float logit_tau,
                                          double* d_bounds, uint64_t* d_bits, int32_t* d_len,
                                          void* stream);

/*
 * Training targets and masks of the predictor (device d_target, d_mask
 * [batch][2 + kmax], written): targets 0 and 1 are d_ub[i * ld_ub + 0..1]
 * (device float; the bound fractions of progress_learned_labels, or the
 * predictor's own outputs when later training must keep its bounds), mask 1;
 * targets 2 + k are bit k of d_bits [batch][4] (device, or NULL = 0), masked
 * (0) for k >= d_iters[i] (device, or NULL = 0) and for every k when
 * d_reject[i] != 0 (device, or NULL: none rejected). 1 <= kmax <= 256.
 * Asynchronous. Errors: EINVAL.
 */
progress_status_t progress_learned_targets(int32_t batch, int32_t kmax, const float* d_ub,
                                           int32_t ld_ub, const uint64_t* d_bits,
                                           const int32_t* d_iters, const int32_t* d_reject,
                                           float* d_target, float* d_mask, void* stream);

/*
 * Bound labels of the predictor from SP2 runs of this library: the projector D1
 * onto the lowest state of H (a batched solve with nocc = 1, bf16 hi+mid+lo
 * split products) gives eps_1 = Tr(H D1), the projector onto the lowest state
 * of -H gives eps_N = Tr(H D1'); then u_min = max((eps_1 - emin)/w, 0) and
 * u_max = max((emax - eps_N)/w, 0) with the Gershgorin enclosure [emin, emax],
 * w = emax - emin.
 *   h_n, h_offset  HOST [batch]: the batch layout (as progress_sp2_batched)
 *   d_n, d_offset  DEVICE [batch]: the same layout
 *   dH             device, packed FP64 instances, read only
 *   d_u            device float [batch][2], written: u_min, u_max
 *   d_gersh        device double [batch][2], written: emin, emax
 *   d_eps          device double [2][batch], written (eps_1 then eps_N), or NULL
 * Allocates and frees its own work space (two packed copies) and synchronizes
 * the stream. Errors: EINVAL, ENOMEM/ECUDA, and those of progress_sp2_batched.
 */
progress_status_t progress_learned_labels(int32_t batch, const int32_t* h_n,
                                          const int64_t* h_offset, const int32_t* d_n,
                                          const int64_t* d_offset, const double* dH, double tol,
                                          float* d_u, double* d_gersh, double* d_eps,
                                          void* stream);

/*
 * Safety margin of the predicted bounds, calibrated on held-out instances
 * (host computation, no GPU): with predictions h_y and targets h_t (HOST
 * float arrays, rows of ld_y / ld_t entries whose first two are the bound
 * fractions), the overshoot of instance i is max(y_i0 - t_i0, y_i1 - t_i1, 0);
 * *margin_out = the `quantile` of the overshoots (linear interpolation
 * between order statistics), at least `floor`. A bound that cuts the spectrum
 * makes the judge reject the run, so the quantile sets the expected fallback
 * rate of that cause. Errors: EINVAL.
 */
progress_status_t progress_learned_margin(int32_t batch, const float* h_y, int32_t ld_y,
                                          const float* h_t, int32_t ld_t, double quantile,
                                          double floor, double* margin_out);

/* Synchronize `stream` and report the last solve queued on it. */
progress_status_t progress_sp2_query(void* stream, progress_info_t* info);

/*
 * Synchronize `stream` and copy the per-iteration history of the last solve
 * queued on it into host arrays of capacity `cap` (either may be NULL):
 *   idem[k]   |Tr X_k^2 - Tr X_k| of iterate X_k, k = 0..iters
 *   margin[k] signed margin of the branch rule at product k, k < iters
 *             (nearer rule: |Tr X^2 - Nocc| - |2 Tr X - Tr X^2 - Nocc|,
 *              paper rule: Nocc - Tr X); a positive margin selects 2X - X^2
 * Returns the number of iterates written to idem (iters + 1, at most cap).
 */
int32_t progress_sp2_history(void* stream, double* idem, double* margin, int32_t cap);

/* Free the cached work spaces (dense, batched, graph and Chebyshev solves) of `stream` on the
 * current device (synchronizes it). */
progress_status_t progress_release(void* stream);

/* Free every cached work space of the current device (synchronizes the device). */
progress_status_t progress_release_all(void);

/* Text of the last error recorded by this thread (never NULL). */
const char* progress_last_error(void);

/* Library version, e.g. "0.1.0". */
const char* progress_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PROGRESS_SP2_H */
