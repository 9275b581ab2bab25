"""Host logic of the Chebyshev solver (no GPU): the library's own schedule
(coefficients, division by T_k, stack slots, scales, launch grouping),
executed step by step in FP64 with numpy products, must give the oracle's
Paterson-Stockmeyer density matrix; every stored operand must fit the
fixed-point slice range (|value| <= 1) and no launch may read a slot that the
same launch writes."""

import numpy as np
import pytest

import oracle
from oracle import cheb as C
from workloads import chain_hamiltonian, cube_hamiltonian


@pytest.fixture(scope="module")
def pkg():
    from paper_2401_13772_gb300.build import build
    build()
    import paper_2401_13772_gb300 as p
    return p


def execute(plan, H, k, m):
    """Run the schedule: T_1 -> T-level launches -> S_j pass -> nested launches."""
    n = H.shape[0]
    I = np.eye(n)
    slots = {0: (H - plan["a"] * I) / plan["b"]}
    D = None
    peak = float(np.abs(slots[0]).max())

    def launch(group):
        nonlocal D, peak
        snap = dict(slots)
        written = set()
        for (a, b, e, c, _), (alpha, sab, beta, se, gamma, inv_sc) in group:
            assert a in snap and b in snap and a not in written and b not in written
            x = float(alpha) * float(sab) * (snap[a] @ snap[b]) + float(gamma) * I
            if e >= 0:
                assert e in snap and e not in written
                x = x + float(beta) * float(se) * snap[e]
            if c < 0:
                D = x
            else:
                assert c not in (a, b, e)
                slots[c] = x * float(inv_sc)
                written.add(c)
                peak = max(peak, float(np.abs(slots[c]).max()))
    pr, pa = plan["prods"], plan["params"]
    rows = list(zip(map(tuple, pr), map(tuple, pa)))
    t = plan["t_products"]
    for L in sorted({int(r[0][4]) for r in rows[:t]}):
        launch([r for r in rows[:t] if r[0][4] == L])
    # S_j = sum_i d_ij T_i, T_0 = I, T_i in slot i - 1
    d = plan["d"]
    for j in range(m):
        S = d[0, j] * I + sum(d[i, j] * slots[i - 1] for i in range(1, k))
        if m == 1:
            D = S
        else:
            slots[k + j] = S * plan["inv_s"][j]
            peak = max(peak, float(np.abs(slots[k + j]).max()))
    for L in sorted({int(r[0][4]) for r in rows[t:]}):
        launch([r for r in rows[t:] if r[0][4] == L])
    return D, peak


@pytest.mark.parametrize("k,m", [(16, 16), (8, 4), (5, 3), (1, 6), (7, 1), (1, 1), (2, 2),
                                 (64, 2), (4, 12)])
def test_schedule_reproduces_the_oracle(pkg, k, m):
    H, _ = cube_hamiltonian(24, 3)
    mu, beta = 0.3, 0.8
    ref = C.fermi_operator(H, mu, beta, k, m)
    plan = pkg.cheb_plan(k, m, mu, beta, ref["emin"], ref["emax"])
    assert plan["slots"] == k + m + 2
    k_top = k if m > 1 else k - 1
    assert len(plan["prods"]) == max(k_top - 1, 0) + (m - 1)
    assert abs(plan["a"] - ref["a"]) <= 1e-12 and abs(plan["b"] - ref["b"]) <= 1e-12
    # (d is not compared entry by entry: each division by T_k doubles the quotient,
    # so the last columns amplify the ~1e-13 differences between the two sides'
    # coefficient sums by 2^j and more; the polynomial, D, is what must agree)
    D, peak = execute(plan, H, k, m)
    # (the nested sums may exceed 1 by the growth factor; compare relative to it)
    growth = float(np.abs(ref["d"]).sum())
    assert np.abs(D - ref["D"]).max() <= 1e-11 * max(1.0, growth)
    assert peak <= 1.0 + 1e-9


def test_levels_are_doubling_and_independent(pkg):
    plan = pkg.cheb_plan(16, 4, 0.0, 1.0, -2.0, 2.0)
    pr = plan["prods"]
    t = plan["t_products"]
    assert t == 15 and plan["product_launches"] == 4 + 3
    # T_n (slot n - 1) of level (2^(l-1), 2^l] in launch l - 1
    for a, b, e, c, launch in pr[:t]:
        q = c + 1
        assert launch == int(np.ceil(np.log2(q))) - 1
        assert a == (q + 1) // 2 - 1 and b == q // 2 - 1
    # nested products: T_k times the previous result, D last
    assert all(row[0] == 15 for row in pr[t:]) and pr[-1][3] == -1


def test_plan_argument_errors(pkg):
    with pytest.raises(pkg.ProgressError):
        pkg.cheb_plan(0, 4, 0.0, 1.0, -1.0, 1.0)
    with pytest.raises(pkg.ProgressError):
        pkg.cheb_plan(4, 4, 0.0, 1.0, 1.0, -1.0)
    with pytest.raises(pkg.ProgressError):
        pkg.cheb_plan(4, 4, 0.0, -1.0, -1.0, 1.0)


def test_chain_low_temperature_schedule(pkg):
    # a gapped chain at mu mid-gap: the schedule reaches the projector
    H, nocc = chain_hamiltonian(64)
    emin, emax = oracle.gershgorin_bounds(H)
    plan = pkg.cheb_plan(32, 16, 0.0, 40.0, emin, emax)
    D, peak = execute(plan, H, 32, 16)
    w, V = np.linalg.eigh(H)
    P = V[:, :nocc] @ V[:, :nocc].T
    assert np.abs(D - P).max() <= 1e-6 and peak <= 1.0 + 1e-9


def test_chooser_prefers_stable_splits(pkg):
    emin, emax = -58.86, 59.68  # the 4096-orbital cube's Gershgorin interval
    r = pkg.cheb_choose_km(256, 0.5, 1.0, emin, emax)
    assert (r["k"], r["m"], r["products"]) == (16, 16, 30) and r["growth"] <= 8.0
    # a sharp Fermi function: the square split k = m = 32 grows to ~1e5; the
    # chooser keeps the growth bounded with a few more products
    sharp = pkg.cheb_plan(32, 32, 0.5, 4.0, emin, emax)
    assert float(np.abs(sharp["d"]).sum()) > 1e4
    r = pkg.cheb_choose_km(1024, 0.5, 4.0, emin, emax)
    assert r["k"] * r["m"] >= 1024 and r["growth"] <= 8.0 and r["k"] > r["m"]
    # every split whose plan has fewer products exceeds the growth bound
    for k in range(1, 65):
        m = -(-1024 // k)
        if m > 64:
            continue
        plan = pkg.cheb_plan(k, m, 0.5, 4.0, emin, emax)
        if len(plan["prods"]) < r["products"]:
            assert float(np.abs(plan["d"]).sum()) > 8.0
    assert len(pkg.cheb_plan(r["k"], r["m"], 0.5, 4.0, emin, emax)["prods"]) == r["products"]
    with pytest.raises(pkg.ProgressError):
        pkg.cheb_choose_km(1024, 0.5, 4.0, emin, emax, max_growth=1e-3)


def test_chosen_split_reproduces_the_oracle(pkg):
    H, _ = cube_hamiltonian(24, 3)
    ref0 = C.fermi_operator(H, 0.3, 2.0, 4, 4)  # only for the bounds
    r = pkg.cheb_choose_km(200, 0.3, 2.0, ref0["emin"], ref0["emax"])
    ref = C.fermi_operator(H, 0.3, 2.0, r["k"], r["m"])
    plan = pkg.cheb_plan(r["k"], r["m"], 0.3, 2.0, ref["emin"], ref["emax"])
    D, peak = execute(plan, H, r["k"], r["m"])
    assert np.abs(D - ref["D"]).max() <= 1e-11 * max(1.0, r["growth"]) and peak <= 1.0 + 1e-9
