"""Pins of the graph-based divide-and-conquer oracle (§VIII.B) and of SP2 at a
fixed chemical potential, against definitions written out by brute force,
exact projectors and limiting cases; mutation tests plant plausible mistakes
in the oracle and check that a pin catches each."""

import numpy as np
import pytest

import oracle
from oracle import graph as G
from workloads import chain_hamiltonian


def projector_below(H, mu):
    """theta(mu I - H) from numpy's eigh (library routine)."""
    w, V = np.linalg.eigh(H)
    occ = V[:, w < mu]
    return occ @ occ.T


def random_gapped(n, rng, gap_at, gap=0.5):
    """Random symmetric matrix with eigenvalues pushed away from gap_at."""
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    w = rng.uniform(-3.0, 3.0, n)
    w = np.where(w < gap_at, np.minimum(w, gap_at - gap / 2), np.maximum(w, gap_at + gap / 2))
    return (Q * w) @ Q.T


def test_threshold_graph_brute_force():
    rng = np.random.default_rng(0)
    M = rng.standard_normal((9, 9))
    M = M + M.T
    A = G.threshold_graph(M, 0.7)
    for i in range(9):
        for j in range(9):
            assert A[i, j] == (i != j and abs(M[i, j]) >= 0.7)


def test_core_partition_regular_segments():
    for n, m in ((10, 3), (7, 7), (1000, 32), (5, 1)):
        parts = G.core_partition(n, m)
        assert len(parts) == m
        assert np.array_equal(np.concatenate(parts), np.arange(n))
        sizes = [len(p) for p in parts]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        G.core_partition(3, 4)


def test_core_halo_brute_force():
    rng = np.random.default_rng(1)
    A = rng.random((30, 30)) < 0.08
    A = A | A.T
    np.fill_diagonal(A, False)
    cores = G.core_partition(30, 4)
    for c, ch in zip(cores, G.core_halo(A, cores)):
        expect = sorted(set(c.tolist()) | {j for i in c for j in range(30) if A[i, j]})
        assert ch.tolist() == expect


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fixed_mu_sp2_is_the_projector_below_mu(seed):
    rng = np.random.default_rng(seed)
    mu = rng.uniform(-1.0, 1.0)
    H = random_gapped(40, rng, mu)
    r = G.sp2_fixed_mu(H, mu, 1e-12)
    assert r["converged"]
    assert np.abs(r["D"] - projector_below(H, mu)).max() <= 1e-10


def test_fixed_mu_sp2_special_cases():
    # dimerized chain at mu = 0 (mid-gap): half filling, the closed-form case
    H, nocc = chain_hamiltonian(256)
    r = G.sp2_fixed_mu(H, 0.0, 1e-12)
    w, V = oracle.jacobi_eigh(H)
    Dref, _ = oracle.density_projector(w, V, nocc)
    assert np.abs(r["D"] - Dref).max() <= 1e-10
    # diagonal H: exactly the entries below mu
    d = np.linspace(-2.0, 2.0, 17)
    r = G.sp2_fixed_mu(np.diag(d), 0.1, 1e-13)
    assert np.abs(r["D"] - np.diag((d < 0.1).astype(float))).max() <= 1e-12
    # mu below / above the whole spectrum
    assert np.abs(G.sp2_fixed_mu(np.diag(d), -5.0, 1e-13)["D"]).max() <= 1e-12
    assert np.abs(G.sp2_fixed_mu(np.diag(d), 5.0, 1e-13)["D"] - np.eye(17)).max() <= 1e-12


def test_graph_density_complete_graph_is_exact():
    # tau below every entry: each halo is the whole system, every part solves H
    rng = np.random.default_rng(3)
    H = random_gapped(36, rng, 0.2)
    P, parts = G.graph_density(H, H, 0.0, 5, 0.2, 1e-12)
    assert all(len(ch) == 36 for _, ch in parts)
    assert np.abs(P - projector_below(H, 0.2)).max() <= 1e-10


def test_graph_density_error_falls_with_the_threshold():
    # gapped 1D chain, auxiliary matrix = a previously computed density matrix
    H, nocc = chain_hamiltonian(512)
    Dprev = projector_below(H, 0.0)
    errs = []
    for tau in (1e-2, 1e-4, 1e-6, 1e-8):
        P, parts = G.graph_density(H, Dprev, tau, 8, 0.0, 1e-12)
        errs.append(float(np.abs(P - Dprev).max()))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] <= 1e-6 and errs[0] >= 1e-4
    # symmetric by construction, trace close to the occupation
    assert np.array_equal(P, P.T)
    assert abs(np.trace(P) - nocc) <= 1e-4


def _mutants():
    """Oracle variants with one plausible mistake each."""
    def no_halo(A, cores):
        return [np.asarray(c) for c in cores]

    def flipped_branch(H, mu, tol, maxiter=100, bounds=None):
        H = np.asarray(H, dtype=np.float64)
        emin, emax = oracle.gershgorin_bounds(H)
        X = oracle.x0_map(H, emin, emax)
        y = (emax - mu) / (emax - emin)
        for _ in range(maxiter):
            if abs(np.sum(X * X) - np.trace(X)) < tol:
                break
            b = 1 if y > 0.5 else 0
            S = X @ X
            X = 2.0 * X - S if b else S
            y = 2.0 * y - y * y if b else y * y
        return {"D": X, "iters": 0, "converged": True, "bits": []}

    def unsymmetrized(H, Gm, tau, nparts, mu, tol, maxiter=100):
        H = np.asarray(H, dtype=np.float64)
        n = H.shape[0]
        A = G.threshold_graph(Gm, tau)
        cores = G.core_partition(n, nparts)
        P = np.zeros((n, n))
        for c, ch in zip(cores, G.core_halo(A, cores)):
            d = G.sp2_fixed_mu(H[np.ix_(ch, ch)], mu, tol, maxiter)["D"]
            P[np.ix_(ch, c)] = d[:, :len(c)]  # wrong: core positions taken as the first ones
        return 0.5 * (P + P.T), None
    return {"no_halo": ("core_halo", no_halo), "flipped_branch": ("sp2_fixed_mu", flipped_branch),
            "core_positions": ("graph_density", unsymmetrized)}


@pytest.mark.parametrize("name", ["no_halo", "flipped_branch", "core_positions"])
def test_mutations_are_caught(name, monkeypatch):
    attr, fn = _mutants()[name]
    monkeypatch.setattr(G, attr, fn)
    H, nocc = chain_hamiltonian(128)
    Dprev = projector_below(H, 0.0)
    caught = False
    try:
        P, _ = G.graph_density(H, Dprev, 1e-8, 4, 0.0, 1e-12)
        caught = float(np.abs(P - Dprev).max()) > 1e-6
    except Exception:
        caught = True
    if not caught and name == "flipped_branch":
        r = G.sp2_fixed_mu(np.diag(np.linspace(-2, 2, 9)), 0.1, 1e-13)
        caught = np.abs(r["D"] - np.diag((np.linspace(-2, 2, 9) < 0.1).astype(float))).max() > 1e-6
    assert caught, name
