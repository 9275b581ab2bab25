"""Pins of the thresholded-SP2 oracle (§IV.A Listing 1 with its cutoff tau):
tau = 0 is plain SP2 exactly; every pruned iterate has no element inside
(0, tau); on the gapped dimerized chain (exponentially localized density
matrix, closed-form spectrum) the error against the exact projector shrinks
with tau and stays within a small multiple of it, while the density matrix
gets sparser; mutation tests plant plausible mistakes and check a pin fails."""

import numpy as np
import pytest

import oracle
from oracle import sparse as S
from workloads import chain_hamiltonian, cube_hamiltonian


def exact_projector(H, nocc):
    w, V = np.linalg.eigh(H)
    return V[:, :nocc] @ V[:, :nocc].T


def test_tau_zero_is_plain_sp2():
    H, nocc = cube_hamiltonian(30, 4)
    a = S.sp2_thresholded(H, nocc, 1e-10, 0.0)
    b = oracle.sp2_plain(H, nocc, 1e-10)
    assert a["iters"] == b["iters"] and a["bits"] == b["bits"]
    assert np.array_equal(a["D"], b["D"])


def no_element_below(X, tau):
    a = np.abs(X)
    return not bool(((a > 0) & (a < tau)).any())


def test_iterates_are_pruned():
    H, nocc = chain_hamiltonian(96)
    r = S.sp2_thresholded(H, nocc, 1e-9, 1e-4, keep_iterates=True)
    assert r["converged"]
    # X0 is not pruned (the chain's X0 has no small elements anyway); every later one is
    for X in r["iterates"][1:]:
        assert no_element_below(X, 1e-4)
        assert np.array_equal(X, X.T)
    assert r["nnz"][-1] < H.size


def test_error_and_sparsity_follow_tau_on_the_gapped_chain():
    H, nocc = chain_hamiltonian(256)
    P = exact_projector(H, nocc)
    errs, nnz = [], []
    for tau in (1e-3, 1e-5, 1e-7):
        r = S.sp2_thresholded(H, nocc, 1e-9, tau)
        assert r["converged"]
        errs.append(float(np.abs(r["D"] - P).max()))
        nnz.append(r["nnz"][-1])
        assert errs[-1] <= 20.0 * tau, (tau, errs[-1])
    assert errs[0] > errs[1] > errs[2]
    assert nnz[0] < nnz[1] < nnz[2] < H.size
    # the exact projector pruned at tau has about the same pattern
    Pp = S.prune(P, 1e-5)
    r = S.sp2_thresholded(H, nocc, 1e-9, 1e-5)
    assert abs(np.count_nonzero(r["D"]) - np.count_nonzero(Pp)) <= 0.05 * np.count_nonzero(Pp)


def test_trace_is_kept():
    H, nocc = chain_hamiltonian(128)
    r = S.sp2_thresholded(H, nocc, 1e-9, 1e-6)
    assert abs(np.trace(r["D"]) - nocc) <= 1e-5


def _mutants():
    def prune_before(H, nocc, tol, tau, rule=0, maxiter=100, bounds=None, keep_iterates=False):
        # prunes the operand instead of the product
        H = np.asarray(H, dtype=np.float64)
        n = H.shape[0]
        emin, emax = oracle.gershgorin_bounds(H)
        X = oracle.x0_map(H, emin, emax)
        its = [X]
        for k in range(maxiter):
            t1, t2 = float(np.trace(X)), float(np.sum(X * X))
            if abs(t2 - t1) < tol:
                break
            b = oracle.branch_bit(t1, t2, nocc, n, rule)
            Xp = S.prune(X, tau)
            X2 = Xp @ Xp
            X = 2.0 * X - X2 if b else X2
            its.append(X)
        return {"D": X, "iterates": its, "converged": True, "nnz": [np.count_nonzero(X)]}

    def no_prune_on_expand(H, nocc, tol, tau, rule=0, maxiter=100, bounds=None,
                           keep_iterates=False):
        H = np.asarray(H, dtype=np.float64)
        n = H.shape[0]
        emin, emax = oracle.gershgorin_bounds(H)
        X = oracle.x0_map(H, emin, emax)
        its = [X]
        for k in range(maxiter):
            t1, t2 = float(np.trace(X)), float(np.sum(X * X))
            if abs(t2 - t1) < tol:
                break
            b = oracle.branch_bit(t1, t2, nocc, n, rule)
            X2 = S.prune(X @ X, tau)
            X = 2.0 * X - X2 if b else X2
            its.append(X)
        return {"D": X, "iterates": its, "converged": True, "nnz": [np.count_nonzero(X)]}
    return {"prune_before": prune_before, "no_prune_on_expand": no_prune_on_expand}


@pytest.mark.parametrize("name", ["prune_before", "no_prune_on_expand"])
def test_mutations_are_caught(name, monkeypatch):
    monkeypatch.setattr(S, "sp2_thresholded", _mutants()[name])
    H, nocc = chain_hamiltonian(96)
    r = S.sp2_thresholded(H, nocc, 1e-9, 1e-4, keep_iterates=True)
    assert not all(no_element_below(X, 1e-4) for X in r["iterates"][1:]), name
