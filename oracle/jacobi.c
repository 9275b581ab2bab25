/*
 * oracle/jacobi.c -- FP64 cyclic Jacobi eigensolver for a real symmetric matrix.
 *
 * TEST INFRASTRUCTURE ONLY. Part of the CPU oracle that checks the CUDA path;
 * the product path never links or calls it.
 *
 * Step 1 of the paper's density-matrix procedure (§III) is "compute all the
 * eigenvalues and eigenvectors of H". This file does that with the classical
 * two-sided Jacobi method (Golub & Van Loan, Matrix Computations, §8.5: the
 * symmetric Schur 2x2 rotation and the cyclic Jacobi sweep), in the parallel
 * "round-robin tournament" ordering: in each of the m-1 steps of a sweep
 * (m = n rounded up to even) the indices are split into m/2 disjoint pairs, so
 * the m/2 rotations of one step commute and each one annihilates its own
 * off-diagonal entry exactly. Every index pair meets once per sweep.
 *
 * A is overwritten (its diagonal ends as the eigenvalues, unsorted);
 * V accumulates the rotations, V[:, i] is the eigenvector of w[i].
 * An entry is rotated only when it is not negligible next to its two pivots,
 * |a_pq| > 1e-17 sqrt(|a_pp a_qq|) (the relative test of Demmel & Veselic,
 * "Jacobi's method is more accurate than QR", 1992); sweeps stop after a
 * sweep that rotates nothing, or after max_sweeps.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

static double off_norm2(int n, const double* A) {
  double s = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      if (i != j) s += A[(size_t)i * n + j] * A[(size_t)i * n + j];
  return s;
}

/* Tournament pairing: player 0 is fixed, players 1..m-1 rotate by one seat per
 * step. Pair k of step s is (seat k, seat m-1-k). Index m-1 is a dummy when n
 * is odd (pairs touching it are skipped). */
static void tournament_pairs(int m, int step, int* P, int* Q) {
  for (int k = 0; k < m / 2; ++k) {
    int a = (k == 0) ? 0 : 1 + ((k - 1 + step) % (m - 1));
    int bseat = m - 1 - k;
    int b = 1 + ((bseat - 1 + step) % (m - 1));
    if (a > b) { int t = a; a = b; b = t; }
    P[k] = a;
    Q[k] = b;
  }
}

int oracle_jacobi_eigh(int n, double* A, double* w, double* V, int max_sweeps,
                       int* sweeps_out, double* off_out) {
  if (n <= 0) return -1;
  const int m = (n % 2) ? n + 1 : n;
  const int npair = m / 2;
  int* P = (int*)malloc(sizeof(int) * npair);
  int* Q = (int*)malloc(sizeof(int) * npair);
  double* C = (double*)malloc(sizeof(double) * npair);
  double* S = (double*)malloc(sizeof(double) * npair);
  double* DP = (double*)malloc(sizeof(double) * npair);
  double* DQ = (double*)malloc(sizeof(double) * npair);
  if (!P || !Q || !C || !S || !DP || !DQ) {
    free(P); free(Q); free(C); free(S); free(DP); free(DQ);
    return -2;
  }

  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[(size_t)i * n + j] = (i == j) ? 1.0 : 0.0;

  double off_prev = sqrt(off_norm2(n, A));
  int sweep = 0;
  for (; sweep < max_sweeps && off_prev > 0.0;) {
    long rotations = 0;
    for (int step = 0; step < m - 1; ++step) {
      tournament_pairs(m, step, P, Q);
      /* Rotation parameters from the current matrix (symmetric Schur 2x2). */
      for (int k = 0; k < npair; ++k) {
        int p = P[k], q = Q[k];
        C[k] = 1.0;
        S[k] = 0.0;
        if (q >= n) continue;
        double apq = A[(size_t)p * n + q];
        double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
        /* Skip an entry that is negligible next to its pivots (a rotation by
         * an angle below round-off would only add rounding error). */
        if (fabs(apq) <= 1e-17 * sqrt(fabs(app * aqq)) || fabs(apq) < 1e-300) continue;
        double tau = (aqq - app) / (2.0 * apq);
        double t = (tau >= 0.0) ? 1.0 / (tau + sqrt(1.0 + tau * tau))
                                : -1.0 / (-tau + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t);
        C[k] = c;
        S[k] = t * c;
        /* Exact diagonal of the rotated 2x2 block (GVL 8.5.2 update form). */
        DP[k] = app - t * apq;
        DQ[k] = aqq + t * apq;
        ++rotations;
      }
      /* A <- J^T A : rows p and q of each pair. */
#pragma omp parallel for schedule(static)
      for (int k = 0; k < npair; ++k) {
        int p = P[k], q = Q[k];
        if (q >= n || S[k] == 0.0) continue;
        double c = C[k], s = S[k];
        double* rp = A + (size_t)p * n;
        double* rq = A + (size_t)q * n;
        for (int j = 0; j < n; ++j) {
          double ap = rp[j], aq = rq[j];
          rp[j] = c * ap - s * aq;
          rq[j] = s * ap + c * aq;
        }
      }
      /* A <- A J and V <- V J : columns p and q, parallel over rows. */
#pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i) {
        double* ra = A + (size_t)i * n;
        double* rv = V + (size_t)i * n;
        for (int k = 0; k < npair; ++k) {
          int p = P[k], q = Q[k];
          if (q >= n || S[k] == 0.0) continue;
          double c = C[k], s = S[k];
          double ap = ra[p], aq = ra[q];
          ra[p] = c * ap - s * aq;
          ra[q] = s * ap + c * aq;
          double vp = rv[p], vq = rv[q];
          rv[p] = c * vp - s * vq;
          rv[q] = s * vp + c * vq;
        }
      }
      /* The rotation annihilates its pivot exactly in exact arithmetic. */
      for (int k = 0; k < npair; ++k) {
        int p = P[k], q = Q[k];
        if (q >= n || S[k] == 0.0) continue;
        A[(size_t)p * n + q] = 0.0;
        A[(size_t)q * n + p] = 0.0;
        A[(size_t)p * n + p] = DP[k];
        A[(size_t)q * n + q] = DQ[k];
      }
    }
    ++sweep;
    off_prev = sqrt(off_norm2(n, A));
    if (rotations == 0) break;
  }
  for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
  if (sweeps_out) *sweeps_out = sweep;
  if (off_out) *off_out = off_prev;
  free(P); free(Q); free(C); free(S); free(DP); free(DQ);
  return 0;
}
