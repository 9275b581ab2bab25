"""Plain FP64 statements of the SP2 density-matrix method -- TEST INFRASTRUCTURE ONLY.

Written from arXiv 2401.13772:

* §III (Eq. 2 and the insulating limit after it): D = V f V^T with
  f = 1 for the Nocc lowest eigenvalues and 0 above, when the spectrum has a
  gap at the Fermi level. ``density_projector``.
* §IV.A: D_0 = (eps_N I - H) / (eps_N - eps_1), then D_{m+1} = D_m^2 when the
  trace of D_m exceeds the electron count and D_{m+1} = 2 D_m - D_m^2 when it
  falls short; Listing 1 (prg_sp2) takes the trace before the product and
  uses the 2D - D^2 branch when Tr D - Nocc <= 0. ``x0_map``, ``sp2_plain``.
* §VIII.A names Gershgorin circles as the eigenvalue-bound estimate that
  Listing 1 needs for emin, emax. ``gershgorin_bounds``.

Readings where the paper is silent (each also listed in the design notes):

* Branch rule NEARER (default): the iteration takes the branch whose trace
  lands nearer Nocc. Both candidate traces are known before the product
  because Tr(X^2) = ||X||_F^2 for symmetric X:
  Tr(X^2) = t2, Tr(2X - X^2) = 2 t1 - t2. Take 2X - X^2 iff
  |t2 - Nocc| - |2 t1 - t2 - Nocc| > 1e-12 * n; a tie takes X^2.
* Branch rule PAPER: 2X - X^2 iff t1 - Nocc <= 0 (the listing's test).
* A zero-width Gershgorin interval (H = c I, n = 1) is widened by 1 on each
  side before the X0 map.
* Convergence ("check for convergence", elided in the listing): stop before
  the next product once |Tr X^2 - Tr X| = |t2 - t1| < tol. The iteration count
  is the number of products performed.

numpy's matmul is the only library primitive used (the product X @ X); no
blocking, fusion or symmetric shortcut.
"""

from __future__ import annotations

import numpy as np

NEARER = 0
PAPER = 1


def gershgorin_bounds(H):
    """Gershgorin enclosure of the spectrum (§VIII.A; emin/emax of Listing 1).

    R_i = sum_{j != i} |H_ij|, emin = min_i (H_ii - R_i), emax = max_i (H_ii + R_i).
    """
    H = np.asarray(H, dtype=np.float64)
    d = np.diag(H).copy()
    R = np.abs(H).sum(axis=1) - np.abs(d)
    return float(np.min(d - R)), float(np.max(d + R))


def x0_map(H, emin, emax):
    """Shifted, rescaled Hamiltonian D_0 = (emax I - H) / (emax - emin) (§IV.A)."""
    H = np.asarray(H, dtype=np.float64)
    n = H.shape[0]
    return (emax * np.eye(n) - H) / (emax - emin)


def branch_bit(t1, t2, nocc, n, rule=NEARER):
    """1 selects X <- 2X - X^2, 0 selects X <- X^2, from t1 = Tr X, t2 = Tr X^2."""
    if rule == PAPER:
        return 1 if (t1 - nocc) <= 0.0 else 0
    d_square = abs(t2 - nocc)
    d_expand = abs(2.0 * t1 - t2 - nocc)
    return 1 if (d_square - d_expand) > 1e-12 * max(n, 1) else 0


def sp2_plain(H, nocc, tol, rule=NEARER, maxiter=100, bounds=None, stop_after=None):
    """Plain FP64 SP2 (§IV.A), one full matrix product per iteration.

    Returns a dict with D (the last iterate), iters (products performed),
    converged, bits (branch per product), t1/t2 histories (traces of each
    iterate X_0, X_1, ...), emin, emax. ``stop_after`` ends after that many
    products (used to compare intermediate iterates).
    """
    H = np.asarray(H, dtype=np.float64)
    n = H.shape[0]
    emin, emax = gershgorin_bounds(H) if bounds is None else bounds
    if not emax > emin:
        # zero-width enclosure (H = c I, n = 1): widen by 1 on each side so the
        # X0 map is defined and the spectrum is still enclosed
        emin, emax = emin - 1.0, emax + 1.0
    X = x0_map(H, emin, emax)
    bits, t1s, t2s = [], [], []
    converged = False
    it = 0
    while True:
        t1 = float(np.trace(X))
        t2 = float(np.sum(X * X))  # Tr(X^2) = ||X||_F^2 for symmetric X
        t1s.append(t1)
        t2s.append(t2)
        if abs(t2 - t1) < tol:
            converged = True
            break
        if it >= maxiter or (stop_after is not None and it >= stop_after):
            break
        b = branch_bit(t1, t2, nocc, n, rule)
        S = X @ X
        X = 2.0 * X - S if b else S
        bits.append(b)
        it += 1
    return {"D": X, "iters": it, "converged": converged, "bits": bits,
            "t1": t1s, "t2": t2s, "emin": emin, "emax": emax}


def spectral_sp2(eigvals, nocc, tol, emin, emax, rule=NEARER, maxiter=100):
    """SP2 acting on the eigenvalues alone.

    Every iterate is a polynomial in H, X_k = V p_k(Lambda) V^T, so its traces
    are sums over the mapped eigenvalues x_i = (emax - eps_i) / (emax - emin)
    and the branch sequence and iteration count depend on the spectrum only.
    Returns a dict like ``sp2_plain`` with ``x`` (final mapped eigenvalues)
    and ``margins`` (the signed rule margin at each decision).
    """
    w = np.asarray(eigvals, dtype=np.float64)
    n = w.size
    x = (emax - w) / (emax - emin)
    bits, t1s, t2s, margins = [], [], [], []
    converged = False
    it = 0
    while True:
        t1 = float(np.sum(x))
        t2 = float(np.sum(x * x))
        t1s.append(t1)
        t2s.append(t2)
        if abs(t2 - t1) < tol:
            converged = True
            break
        if it >= maxiter:
            break
        b = branch_bit(t1, t2, nocc, n, rule)
        if rule == PAPER:
            margins.append(nocc - t1)
        else:
            margins.append(abs(t2 - nocc) - abs(2.0 * t1 - t2 - nocc))
        x = 2.0 * x - x * x if b else x * x
        bits.append(b)
        it += 1
    return {"x": x, "iters": it, "converged": converged, "bits": bits,
            "t1": t1s, "t2": t2s, "margins": margins}


def density_projector(w, V, nocc):
    """Zero-temperature density matrix D = sum_{i <= Nocc} v_i v_i^T (§III).

    ``w`` ascending with V[:, i] its eigenvector. Returns (D, gap) where
    gap = w[nocc] - w[nocc - 1] (the HOMO-LUMO gap; inf when nocc is 0 or n).
    """
    w = np.asarray(w, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    n = w.size
    if not 0 <= nocc <= n:
        raise ValueError("nocc out of range")
    Vo = V[:, :nocc]
    D = Vo @ Vo.T
    gap = float(w[nocc] - w[nocc - 1]) if 0 < nocc < n else float("inf")
    return D, gap


def invariants(D, H, nocc):
    """Properties the exact density matrix has at any size (§III).

    D = D^T, D^2 = D, Tr D = Nocc, and D commutes with H.
    """
    D = np.asarray(D, dtype=np.float64)
    H = np.asarray(H, dtype=np.float64)
    hmax = max(float(np.abs(H).max()), 1e-300)
    return {
        "symmetry": float(np.abs(D - D.T).max()),
        "idempotency": float(np.abs(D @ D - D).max()),
        "trace_err": abs(float(np.trace(D)) - nocc),
        "commutator": float(np.abs(H @ D - D @ H).max()) / hmax,
    }
