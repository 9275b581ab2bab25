"""Pins of the CPU oracle against what the mathematics fixes (no GPU).

Each pin is independent of the oracle's own code path: closed forms, the
Riesz contour-integral projector, a library eigensolver, analytic 2x2 results,
exact special cases and brute force on tiny matrices. The mutation tests at the
end plant plausible mistakes in the oracle and check that a pin catches each.
"""

import numpy as np
import pytest

import oracle
from oracle import sp2 as osp2
from workloads import chain_hamiltonian, cube_hamiltonian

T1, T2 = -1.0, -0.6


def chain_closed_form(n=512, t1=T1, t2=T2):
    """Dimerized chain with two sites per cell: eps_+-(k) = +-|t1 + t2 e^{ik}|."""
    k = 2.0 * np.pi * np.arange(n // 2) / (n // 2)
    e = np.sqrt(t1 * t1 + t2 * t2 + 2.0 * t1 * t2 * np.cos(k))
    return np.sort(np.concatenate([-e, e]))


def riesz_projector(H, mu, lo, delta):
    """(1/2 pi i) contour integral of (z - H)^{-1} over a circle enclosing the
    spectrum below mu (trapezoid rule, exponentially convergent).

    ``delta`` is the distance from the contour to the nearest eigenvalue; the
    trapezoid error decays like (1 - delta/r)^npts, so npts ~ 40 r / delta
    reaches round-off."""
    n = H.shape[0]
    c = 0.5 * (lo + mu)
    r = 0.5 * (mu - lo)
    npts = int(max(1024, 40.0 * r / delta))
    th = 2.0 * np.pi * (np.arange(npts) + 0.5) / npts
    z = c + r * np.exp(1j * th)
    dz = 1j * r * np.exp(1j * th) * (2.0 * np.pi / npts)
    I = np.eye(n)
    D = np.zeros((n, n), dtype=complex)
    for zq, wq in zip(z, dz):
        D += wq * np.linalg.solve(zq * I - H, I)
    return (D / (2j * np.pi)).real


def random_gapped(n, rng, nocc, min_gap=0.1):
    while True:
        A = rng.standard_normal((n, n))
        H = 0.5 * (A + A.T)
        w = np.linalg.eigvalsh(H)
        if 0 < nocc < n and w[nocc] - w[nocc - 1] >= min_gap:
            return H, w


# --------------------------------------------------------------------------
# Jacobi eigensolver
# --------------------------------------------------------------------------

def test_tournament_covers_all_pairs_once_per_sweep():
    # The C code's pairing, restated: every index pair meets once per sweep and
    # every step is a perfect matching.
    for m in (2, 4, 6, 8, 12):
        seen = set()
        for s in range(m - 1):
            used = set()
            for k in range(m // 2):
                a = 0 if k == 0 else 1 + ((k - 1 + s) % (m - 1))
                b = 1 + ((m - 1 - k - 1 + s) % (m - 1))
                used |= {a, b}
                seen.add((min(a, b), max(a, b)))
            assert len(used) == m
        assert len(seen) == m * (m - 1) // 2


def test_jacobi_chain_closed_form_spectrum():
    H, _ = chain_hamiltonian(512, T1, T2)
    w, V, info = oracle.jacobi_eigh(H, return_info=True)
    assert np.abs(w - chain_closed_form(512)).max() < 1e-12
    assert np.abs(V.T @ V - np.eye(512)).max() < 1e-12
    assert np.abs(H @ V - V * w).max() < 1e-12
    assert info["sweeps"] < 40


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 17, 64])
def test_jacobi_vs_library_eigh(n):
    rng = np.random.default_rng(100 + n)
    A = rng.standard_normal((n, n))
    H = A + A.T
    w, V = oracle.jacobi_eigh(H)
    we = np.linalg.eigvalsh(H)
    assert np.abs(w - we).max() < 1e-12 * max(1.0, np.abs(we).max())
    assert np.abs(V @ np.diag(w) @ V.T - H).max() < 1e-12 * max(1.0, np.abs(H).max())
    assert np.abs(V.T @ V - np.eye(n)).max() < 1e-13


def test_jacobi_cube_vs_library_projector():
    H, nocc = cube_hamiltonian(64, 7)  # n = 256
    w, V = oracle.jacobi_eigh(H)
    we, Ve = np.linalg.eigh(H)
    D, gap = oracle.density_projector(w, V, nocc)
    De, _ = oracle.density_projector(we, Ve, nocc)
    assert gap > 0
    assert np.abs(D - De).max() < 1e-11


# --------------------------------------------------------------------------
# Density projector (§III)
# --------------------------------------------------------------------------

def test_projector_chain_chiral_symmetry():
    H, nocc = chain_hamiltonian(512, T1, T2)
    w, V = oracle.jacobi_eigh(H)
    D, gap = oracle.density_projector(w, V, nocc)
    assert abs(gap - 2.0 * (abs(T1) - abs(T2))) < 1e-12  # band gap 0.8
    assert np.abs(np.diag(D) - 0.5).max() < 1e-12  # half filling, bipartite
    i, j = np.meshgrid(np.arange(512), np.arange(512), indexing="ij")
    same_sublattice = ((i - j) % 2 == 0) & (i != j)
    assert np.abs(D[same_sublattice]).max() < 1e-12


@pytest.mark.parametrize("n,nocc", [(2, 1), (3, 1), (4, 2), (5, 3), (6, 2), (8, 4), (8, 7)])
def test_projector_vs_riesz_contour(n, nocc):
    rng = np.random.default_rng(10 * n + nocc)
    H, wl = random_gapped(n, rng, nocc)
    mu = 0.5 * (wl[nocc - 1] + wl[nocc])
    Dr = riesz_projector(H, mu, wl[0] - 1.0, 0.5 * (wl[nocc] - wl[nocc - 1]))
    w, V = oracle.jacobi_eigh(H)
    D, _ = oracle.density_projector(w, V, nocc)
    assert np.abs(D - Dr).max() < 1e-11


def test_projector_2x2_analytic():
    for a, b, c in [(0.3, 0.7, -1.1), (2.0, -0.01, 1.0), (0.0, 1.0, 0.0)]:
        H = np.array([[a, b], [b, c]])
        r = np.sqrt(((a - c) / 2.0) ** 2 + b * b)
        Dex = 0.5 * (np.eye(2) - (H - 0.5 * (a + c) * np.eye(2)) / r)
        w, V = oracle.jacobi_eigh(H)
        D, _ = oracle.density_projector(w, V, 1)
        assert np.abs(D - Dex).max() < 1e-14
        out = oracle.sp2_plain(H, 1, 1e-14)
        assert out["converged"]
        assert np.abs(out["D"] - Dex).max() < 1e-12


# --------------------------------------------------------------------------
# Gershgorin bounds and X0 map
# --------------------------------------------------------------------------

def test_gershgorin_chain_exact_extremes():
    H, _ = chain_hamiltonian(512, T1, T2)
    emin, emax = oracle.gershgorin_bounds(H)
    assert emin == -1.6 and emax == 1.6
    w = chain_closed_form(512)
    assert abs(w[0] - emin) < 1e-14 and abs(w[-1] - emax) < 1e-14


def test_gershgorin_encloses_spectrum_and_is_brute_force_max():
    rng = np.random.default_rng(5)
    for n in (1, 2, 7, 33):
        A = rng.standard_normal((n, n))
        H = A + A.T
        emin, emax = oracle.gershgorin_bounds(H)
        w = np.linalg.eigvalsh(H)
        assert emin <= w[0] + 1e-12 and w[-1] <= emax + 1e-12
        # brute force over the discs
        lo = min(H[i, i] - sum(abs(H[i, j]) for j in range(n) if j != i) for i in range(n))
        hi = max(H[i, i] + sum(abs(H[i, j]) for j in range(n) if j != i) for i in range(n))
        assert abs(lo - emin) < 1e-12 and abs(hi - emax) < 1e-12


def test_x0_maps_spectrum_into_unit_interval_reversed():
    H, nocc = cube_hamiltonian(32, 3)
    emin, emax = oracle.gershgorin_bounds(H)
    X0 = oracle.x0_map(H, emin, emax)
    w = np.linalg.eigvalsh(H)
    x = np.linalg.eigvalsh(X0)
    assert x.min() >= -1e-12 and x.max() <= 1 + 1e-12
    # lowest energies map nearest 1: x_i = (emax - eps_i) / (emax - emin)
    assert np.abs(np.sort((emax - w) / (emax - emin)) - x).max() < 1e-12


# --------------------------------------------------------------------------
# SP2 (§IV.A)
# --------------------------------------------------------------------------

def test_sp2_chain_converges_to_projector():
    H, nocc = chain_hamiltonian(512, T1, T2)
    w, V = oracle.jacobi_eigh(H)
    Dref, _ = oracle.density_projector(w, V, nocc)
    for rule in (oracle.NEARER, oracle.PAPER):
        out = oracle.sp2_plain(H, nocc, 1e-12, rule=rule)
        assert out["converged"]
        assert out["iters"] == 16
        assert np.abs(out["D"] - Dref).max() < 1e-12
    near = oracle.sp2_plain(H, nocc, 1e-12, rule=oracle.NEARER)["bits"]
    paper = oracle.sp2_plain(H, nocc, 1e-12, rule=oracle.PAPER)["bits"]
    # Step 1 is an exact tie (Tr X0 = 256, Tr X0^2 = 196): the two rules choose
    # opposite branches there, and by the chain's particle-hole symmetry they
    # stay complementary.
    assert [1 - b for b in near] == paper


def test_sp2_diagonal_h_is_exact_occupation():
    rng = np.random.default_rng(11)
    for n, nocc in [(10, 3), (33, 16), (64, 1), (64, 63)]:
        d = rng.permutation(np.linspace(-3.0, 2.0, n))
        H = np.diag(d)
        out = oracle.sp2_plain(H, nocc, 1e-13)
        expect = np.zeros(n)
        expect[np.argsort(d)[:nocc]] = 1.0
        assert out["converged"]
        assert np.abs(out["D"] - np.diag(expect)).max() < 1e-12


@pytest.mark.parametrize("n,nocc", [(4, 2), (6, 1), (7, 4), (8, 4)])
def test_sp2_bruteforce_small_vs_riesz(n, nocc):
    rng = np.random.default_rng(1000 + 10 * n + nocc)
    H, wl = random_gapped(n, rng, nocc, min_gap=0.3)
    mu = 0.5 * (wl[nocc - 1] + wl[nocc])
    Dr = riesz_projector(H, mu, wl[0] - 1.0, 0.5 * (wl[nocc] - wl[nocc - 1]))
    for rule in (oracle.NEARER, oracle.PAPER):
        out = oracle.sp2_plain(H, nocc, 1e-13, rule=rule)
        assert out["converged"]
        assert np.abs(out["D"] - Dr).max() < 1e-10


def test_sp2_cube_vs_projector_and_invariants():
    H, nocc = cube_hamiltonian(64, 1)  # n = 256
    w, V = oracle.jacobi_eigh(H)
    Dref, gap = oracle.density_projector(w, V, nocc)
    out = oracle.sp2_plain(H, nocc, 1e-12)
    assert out["converged"]
    assert np.abs(out["D"] - Dref).max() < 1e-10
    inv = oracle.invariants(out["D"], H, nocc)
    assert inv["symmetry"] < 1e-13 and inv["idempotency"] < 1e-11
    assert inv["trace_err"] < 1e-10 and inv["commutator"] < 1e-10


def test_spectral_sp2_predicts_iterates():
    H, nocc = cube_hamiltonian(24, 2)  # n = 96
    w, V = oracle.jacobi_eigh(H)
    emin, emax = oracle.gershgorin_bounds(H)
    spec = oracle.spectral_sp2(w, nocc, 1e-12, emin, emax)
    full = oracle.sp2_plain(H, nocc, 1e-12)
    assert spec["iters"] == full["iters"]
    big = [k for k, m in enumerate(spec["margins"]) if abs(m) > 1e-6 * len(w)]
    assert [spec["bits"][k] for k in big] == [full["bits"][k] for k in big]
    # an intermediate iterate is V p_k(Lambda) V^T
    k = 10
    mid = oracle.sp2_plain(H, nocc, 0.0, stop_after=k)
    x = (emax - w) / (emax - emin)
    for b in mid["bits"]:
        x = 2 * x - x * x if b else x * x
    assert np.abs(mid["D"] - (V * x) @ V.T).max() < 1e-12


def test_branch_rules_definition():
    # nearer rule: trace of X^2 is t2, trace of 2X - X^2 is 2 t1 - t2
    assert oracle.branch_bit(10.0, 9.0, 5.0, 20) == 0  # |9-5|=4 < |11-5|=6
    assert oracle.branch_bit(4.0, 3.0, 5.0, 20) == 1  # |3-5|=2 > |5-5|=0
    assert oracle.branch_bit(6.0, 5.0, 6.0, 20) == 0  # tie 1 vs 1 -> X^2
    # paper rule: 2X - X^2 iff Tr X - Nocc <= 0
    assert oracle.branch_bit(5.0, 1.0, 5.0, 20, oracle.PAPER) == 1
    assert oracle.branch_bit(5.1, 1.0, 5.0, 20, oracle.PAPER) == 0


# --------------------------------------------------------------------------
# Mutation tests: plant a plausible mistake in the oracle, a pin must fail.
# --------------------------------------------------------------------------

def _chain_pin_fails():
    H, nocc = chain_hamiltonian(64, T1, T2)
    Dr = riesz_projector(H, 0.0, -2.0, 0.4)
    out = osp2.sp2_plain(H, nocc, 1e-12)
    return (not out["converged"]) or np.abs(out["D"] - Dr).max() > 1e-8


def _cube_pin_fails():
    H, nocc = cube_hamiltonian(8, 4)  # n = 32
    w = np.linalg.eigvalsh(H)
    mu = 0.5 * (w[nocc - 1] + w[nocc])
    Dr = riesz_projector(H, mu, w[0] - 1.0, 0.5 * (w[nocc] - w[nocc - 1]))
    out = osp2.sp2_plain(H, nocc, 1e-12)
    return (not out["converged"]) or np.abs(out["D"] - Dr).max() > 1e-8


def test_pins_pass_unmutated():
    assert not _chain_pin_fails()
    assert not _cube_pin_fails()


@pytest.mark.parametrize("mutant", ["x0_sign", "x0_scale", "gersh_noabs", "branch_swap",
                                    "trace_only_diag", "expand_coeff"])
def test_pins_catch_planted_mistakes(monkeypatch, mutant):
    good_x0, good_g, good_b = osp2.x0_map, osp2.gershgorin_bounds, osp2.branch_bit
    if mutant == "x0_sign":  # (H - emin)/(emax - emin): occupies the top states
        monkeypatch.setattr(osp2, "x0_map",
                            lambda H, a, b: (H - a * np.eye(H.shape[0])) / (b - a))
    elif mutant == "x0_scale":  # dropped the denominator
        monkeypatch.setattr(osp2, "x0_map", lambda H, a, b: (b * np.eye(H.shape[0]) - H))
    elif mutant == "gersh_noabs":  # radius without absolute values
        def g(H):
            d = np.diag(H)
            R = H.sum(axis=1) - d
            return float(np.min(d - R)), float(np.max(d + R))
        monkeypatch.setattr(osp2, "gershgorin_bounds", g)
    elif mutant == "branch_swap":
        monkeypatch.setattr(osp2, "branch_bit", lambda t1, t2, no, n, rule=0: 1 - good_b(t1, t2, no, n, rule))
    elif mutant == "trace_only_diag":  # Tr X^2 taken as sum of squared diagonal
        real_sum = np.sum

        def fake_sum(a, *k, **kw):
            if isinstance(a, np.ndarray) and a.ndim == 2 and a.shape[0] == a.shape[1] and not k and not kw:
                return real_sum(np.diag(a))
            return real_sum(a, *k, **kw)
        monkeypatch.setattr(osp2.np, "sum", fake_sum)
    elif mutant == "expand_coeff":  # X - X^2 instead of 2X - X^2
        orig = osp2.sp2_plain

        def mutated(H, nocc, tol, rule=0, maxiter=100, bounds=None, stop_after=None):
            n = H.shape[0]
            emin, emax = osp2.gershgorin_bounds(H)
            X = osp2.x0_map(H, emin, emax)
            it, conv = 0, False
            while it <= maxiter:
                t1, t2 = np.trace(X), np.sum(X * X)
                if abs(t2 - t1) < tol:
                    conv = True
                    break
                b = osp2.branch_bit(t1, t2, nocc, n, rule)
                S = X @ X
                X = X - S if b else S
                it += 1
            return {"D": X, "iters": it, "converged": conv, "bits": []}
        monkeypatch.setattr(osp2, "sp2_plain", mutated)
    assert _chain_pin_fails() or _cube_pin_fails()
    del good_x0, good_g


def test_golden_chain_fixture_matches_closed_form_facts():
    """The stored chain fixture agrees with facts fixed by the closed form:
    Tr X0 = N/2 (zero onsite), ||X0||_F^2 = N/4 + N (t1^2 + t2^2)/(emax - emin)^2."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "chain512_sp2.json")))
    assert g["emin"] == -1.6 and g["emax"] == 1.6
    assert abs(g["nearer"]["trace_x0"] - 256.0) < 1e-12
    assert abs(g["nearer"]["trace_x0_sq"] - (128.0 + 512 * (1.0 + 0.36) / 3.2 ** 2)) < 1e-11
    assert g["nearer"]["iters"] == g["paper"]["iters"] == 16
    assert g["paper"]["bits"] == "".join("1" if c == "0" else "0" for c in g["nearer"]["bits"])
    H, nocc = chain_hamiltonian(512, T1, T2)
    assert "".join(map(str, oracle.sp2_plain(H, nocc, 1e-12)["bits"])) == g["nearer"]["bits"]


def test_sp2_scalar_and_multiple_of_identity():
    # zero-width Gershgorin interval: the occupation is still exact
    for nocc in (0, 1):
        out = oracle.sp2_plain(np.array([[0.7]]), nocc, 1e-14)
        assert out["converged"] and abs(out["D"][0, 0] - nocc) < 1e-14
    out = oracle.sp2_plain(2.5 * np.eye(6), 6, 1e-14)
    assert np.abs(out["D"] - np.eye(6)).max() < 1e-14
