"""Thresholded SP2 -- TEST INFRASTRUCTURE ONLY.

Plain FP64 statement of the thresholded SP2 of arXiv 2401.13772 (§IV.A,
Listing 1 with its cutoff tau; the sparse solvers of §VII keep the same
thresholding criterion): the matrix product and the branch update each drop
the elements whose magnitude is below tau,

    X2 <- prune(X X),   X <- prune(2 X - X2)  or  X <- X2,

prune(A)_ij = 0 if |A_ij| < tau else A_ij. The starting matrix
X0 = (emax I - H) / (emax - emin) is not pruned (the listing builds it with a
copy, an identity shift and a scale, none of which takes tau). Branch rule,
convergence test and Gershgorin bounds as in ``sp2.sp2_plain``.

numpy's matmul is the only library primitive.
"""

from __future__ import annotations

import numpy as np

from .sp2 import NEARER, branch_bit, gershgorin_bounds, x0_map


def prune(A, tau):
    """Elements with |a| < tau set to zero."""
    A = np.asarray(A, dtype=np.float64)
    return np.where(np.abs(A) < tau, 0.0, A)


def sp2_thresholded(H, nocc, tol, tau, rule=NEARER, maxiter=100, bounds=None,
                    keep_iterates=False):
    """Thresholded SP2. Returns dict(D, iters, converged, bits, nnz, iterates):
    nnz[k] = non-zeros of X_k; iterates = [X_0, X_1, ...] if keep_iterates."""
    H = np.asarray(H, dtype=np.float64)
    n = H.shape[0]
    emin, emax = gershgorin_bounds(H) if bounds is None else bounds
    if not emax > emin:
        emin, emax = emin - 1.0, emax + 1.0
    X = x0_map(H, emin, emax)
    bits, nnz, its = [], [int(np.count_nonzero(X))], [X] if keep_iterates else []
    converged = False
    k = 0
    while True:
        t1 = float(np.trace(X))
        t2 = float(np.sum(X * X))
        if abs(t2 - t1) < tol:
            converged = True
            break
        if k >= maxiter:
            break
        b = branch_bit(t1, t2, nocc, n, rule)
        X2 = prune(X @ X, tau)
        X = prune(2.0 * X - X2, tau) if b else X2
        bits.append(b)
        nnz.append(int(np.count_nonzero(X)))
        if keep_iterates:
            its.append(X)
        k += 1
    return {"D": X, "iters": k, "converged": converged, "bits": bits, "nnz": nnz,
            "iterates": its, "emin": emin, "emax": emax}
