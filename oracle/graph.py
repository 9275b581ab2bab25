"""Graph-based divide-and-conquer density matrix -- TEST INFRASTRUCTURE ONLY.

Plain FP64 statement of §VIII.B of arXiv 2401.13772 (graph-based divide
electronic structure), step by step:

1. The adjacency matrix of an auxiliary matrix G (the Hamiltonian, or a
   previously computed density matrix) at threshold tau:
   A_ij = 1 if |G_ij| >= tau and i != j, else 0.       ``threshold_graph``
2. A core partition: every node in exactly one part. The paper's simplest
   option divides the index list into regular segments.  ``core_partition``
3. The core-halo partition: each core extended by every node directly
   connected to one of its nodes.                        ``core_halo``
4. For each part k the dense submatrix h_k = H[ch_k, ch_k]; a matrix function
   of it -- here the zero-temperature density matrix theta(mu I - h_k) at the
   global chemical potential mu, computed by SP2 -- and the columns of the
   cores mapped back into the full matrix P.             ``graph_density``
5. P is symmetrized as (P + P^T) / 2: each column of P comes from the part
   whose core holds it, so P is not symmetric before this step (a reading:
   the paper sums the parts' contributions without saying how the two
   triangles are reconciled).

SP2 at a fixed chemical potential (``sp2_fixed_mu``, a reading: the paper's
sub-problems apply a Fermi function at the system's mu, while the SP2 of
§IV.A fixes the occupation instead). The X0 map sends mu to
y_0 = (emax - mu) / (emax - emin); every SP2 step maps all eigenvalues and y
by the same polynomial, so the states below mu (mapped above y) go to 1 and
those above to 0 as long as y stays away from 0 and 1. The branch is chosen
on y alone: X^2 if y > 1/2, else 2X - X^2, and y follows the same map (it
moves into [1/4, 3/4] and stays there). A bound interval that does not hold mu
strictly inside is widened to include mu -/+ 1. Convergence as in §IV.A: |Tr X^2 - Tr X| < tol.

numpy's matmul is the only library primitive (the product X @ X).
"""

from __future__ import annotations

import numpy as np

from .sp2 import gershgorin_bounds, x0_map


def threshold_graph(G, tau):
    """Adjacency matrix A_ij = 1 if |G_ij| >= tau and i != j (boolean)."""
    G = np.asarray(G, dtype=np.float64)
    A = np.abs(G) >= tau
    np.fill_diagonal(A, False)
    return A


def core_partition(n, nparts):
    """Regular segments of the index list 0..n-1: part k holds
    [floor(k n / m), floor((k + 1) n / m))."""
    if nparts < 1 or nparts > max(n, 1):
        raise ValueError("nparts must be in [1, n]")
    edges = [(k * n) // nparts for k in range(nparts + 1)]
    return [np.arange(edges[k], edges[k + 1]) for k in range(nparts)]


def core_halo(A, cores):
    """Each core extended by the nodes directly connected to it (sorted)."""
    parts = []
    for c in cores:
        mask = np.zeros(A.shape[0], dtype=bool)
        mask[c] = True
        mask |= A[c].any(axis=0)
        parts.append(np.flatnonzero(mask))
    return parts


def sp2_fixed_mu(H, mu, tol, maxiter=100, bounds=None):
    """theta(mu I - H) by SP2 with the branch taken on the mapped mu (see the
    module note). Returns dict(D, iters, converged, bits)."""
    H = np.asarray(H, dtype=np.float64)
    n = H.shape[0]
    emin, emax = gershgorin_bounds(H) if bounds is None else bounds
    if not emax > emin:
        emin, emax = emin - 1.0, emax + 1.0
    # mu must map strictly inside (0, 1): an interval that does not contain it
    # is widened to mu -/+ 1 (the answer is then 0 or I)
    if not emin < mu < emax:
        emin, emax = min(emin, mu - 1.0), max(emax, mu + 1.0)
    X = x0_map(H, emin, emax)
    y = (emax - mu) / (emax - emin)
    bits = []
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
        b = 0 if y > 0.5 else 1
        S = X @ X
        X = 2.0 * X - S if b else S
        y = 2.0 * y - y * y if b else y * y
        bits.append(b)
        k += 1
    return {"D": X, "iters": k, "converged": converged, "bits": bits}


def graph_density(H, G, tau, nparts, mu, tol, maxiter=100):
    """The graph-based density matrix P ~ theta(mu I - H) (§VIII.B).

    Returns (P, parts) with parts = [(core, core_halo), ...]."""
    H = np.asarray(H, dtype=np.float64)
    n = H.shape[0]
    A = threshold_graph(G, tau)
    cores = core_partition(n, nparts)
    halos = core_halo(A, cores)
    P = np.zeros((n, n))
    for c, ch in zip(cores, halos):
        h = H[np.ix_(ch, ch)]
        d = sp2_fixed_mu(h, mu, tol, maxiter)["D"]
        pos = np.searchsorted(ch, c)  # positions of the core inside the part
        P[np.ix_(ch, c)] = d[:, pos]
    return 0.5 * (P + P.T), list(zip(cores, halos))
