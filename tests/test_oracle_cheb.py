"""Pins of the Chebyshev Fermi-operator oracle (§IV.B, Eqs. 5-11) against
closed forms (T_n(cos t) = cos(n t), the Bessel series of exp), library
routines (numpy's eigh, scipy's modified Bessel functions), the serial
recursion as an independent algorithm for the same polynomial, and limiting
cases; mutation tests plant plausible mistakes in the oracle and check that a
pin catches each."""

import numpy as np
import pytest

import oracle
from oracle import cheb as C
from workloads import chain_hamiltonian


def cheb_closed(n, x):
    """T_n(x) = cos(n arccos x) on [-1, 1]."""
    return np.cos(n * np.arccos(np.clip(x, -1.0, 1.0)))


def random_spectrum_matrix(n, rng, lo=-1.0, hi=1.0):
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    w = rng.uniform(lo, hi, n)
    return (Q * w) @ Q.T, w, Q


def test_coefficients_reproduce_polynomials():
    # the interpolant of a polynomial of degree <= L is the polynomial itself
    c = C.cheb_coefficients(lambda x: cheb_closed(5, x), 9)
    e = np.zeros(10)
    e[5] = 1.0
    assert np.abs(c - e).max() <= 1e-14
    c = C.cheb_coefficients(lambda x: x * x, 4)          # x^2 = (T_0 + T_2) / 2
    assert np.abs(c - [0.5, 0.0, 0.5, 0.0, 0.0]).max() <= 1e-15
    c = C.cheb_coefficients(lambda x: 3.0 + 0.0 * x, 3)
    assert np.abs(c - [3.0, 0.0, 0.0, 0.0]).max() <= 1e-15


def test_coefficients_of_exp_are_bessel_values():
    # e^{t x} = I_0(t) + 2 sum_n I_n(t) T_n(x)
    special = pytest.importorskip("scipy.special")
    t = 2.5
    c = C.cheb_coefficients(lambda x: np.exp(t * x), 30)
    ref = np.array([special.iv(n, t) * (1.0 if n == 0 else 2.0) for n in range(31)])
    assert np.abs(c - ref).max() <= 1e-14


@pytest.mark.parametrize("k,m", [(1, 1), (1, 6), (5, 1), (3, 4), (8, 8), (16, 4), (4, 16)])
def test_ps_coefficients_reproduce_the_series(k, m):
    # nested form of Eq. 7 evaluated with the closed-form T_n at scalar points
    rng = np.random.default_rng(k * 100 + m)
    c = rng.standard_normal(k * m) / (1.0 + np.arange(k * m))
    d = C.ps_coefficients(c, k, m)
    x = rng.uniform(-1.0, 1.0, 64)
    direct = sum(c[n] * cheb_closed(n, x) for n in range(k * m))
    S = [sum(d[i, j] * cheb_closed(i, x) for i in range(k)) for j in range(m)]
    P = S[m - 1]
    for j in range(m - 2, -1, -1):
        P = S[j] + cheb_closed(k, x) * P
    assert np.abs(P - direct).max() <= 1e-12 * max(1.0, np.abs(d).max())


def test_ps_coefficients_argument_check():
    with pytest.raises(ValueError):
        C.ps_coefficients(np.ones(7), 2, 4)


def test_chebyshev_polynomials_closed_form():
    rng = np.random.default_rng(4)
    A, w, Q = random_spectrum_matrix(24, rng)
    T = C.chebyshev_polynomials(A, 13)
    assert len(T) == 14
    for n, Tn in enumerate(T):
        ref = (Q * cheb_closed(n, w)) @ Q.T
        assert np.abs(Tn - ref).max() <= 1e-12, n


def test_ps_evaluate_equals_serial_recursion():
    rng = np.random.default_rng(5)
    A, _, _ = random_spectrum_matrix(30, rng)
    for k, m in ((4, 4), (6, 3), (1, 5), (7, 1)):
        c = rng.standard_normal(k * m) * 0.7 ** np.arange(k * m)
        d = C.ps_coefficients(c, k, m)
        assert np.abs(C.ps_evaluate(A, d) - C.serial_chebyshev(A, c)).max() <= 1e-12


def test_serial_recursion_closed_form():
    rng = np.random.default_rng(6)
    A, w, Q = random_spectrum_matrix(16, rng)
    c = rng.standard_normal(9)
    ref = (Q * sum(c[n] * cheb_closed(n, w) for n in range(9))) @ Q.T
    assert np.abs(C.serial_chebyshev(A, c) - ref).max() <= 1e-12


def test_fermi_operator_converges_to_fermi_dirac():
    # eigh-based f(H) = V f(w) V^T (§III, Eq. 2) at finite temperature
    rng = np.random.default_rng(7)
    H, w, Q = random_spectrum_matrix(40, rng, -3.0, 2.0)
    mu, beta = 0.3, 4.0
    ref = (Q * C.fermi(w, mu, beta)) @ Q.T
    errs = []
    for k, m in ((4, 4), (8, 4), (8, 8), (16, 8), (16, 16)):
        r = C.fermi_operator(H, mu, beta, k, m)
        errs.append(float(np.abs(r["D"] - ref).max()))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] <= 1e-10
    r = C.fermi_operator(H, mu, beta, 16, 16)
    assert abs(np.trace(r["D"]) - C.fermi(w, mu, beta).sum()) <= 1e-9


def test_fermi_operator_limits():
    rng = np.random.default_rng(8)
    H, w, Q = random_spectrum_matrix(20, rng, -1.0, 1.0)
    # beta = 0: f = 1/2 everywhere, D = I / 2 exactly
    r = C.fermi_operator(H, 0.0, 0.0, 4, 4)
    assert np.abs(r["D"] - 0.5 * np.eye(20)).max() <= 1e-14
    # mu far below / above the spectrum: D = 0 / I
    assert np.abs(C.fermi_operator(H, -50.0, 2.0, 16, 8)["D"]).max() <= 1e-10
    assert np.abs(C.fermi_operator(H, 50.0, 2.0, 16, 8)["D"] - np.eye(20)).max() <= 1e-10
    # n = 1: zero-width interval widened by 1, D = f(h)
    r = C.fermi_operator(np.array([[0.7]]), 0.2, 3.0, 8, 4)
    assert abs(r["D"][0, 0] - C.fermi(0.7, 0.2, 3.0)) <= 1e-13
    assert (r["emin"], r["emax"]) == (0.7, 0.7)


def test_low_temperature_reaches_the_projector():
    # gapped dimerized chain, mu mid-gap: as beta grows D -> theta(mu I - H)
    H, nocc = chain_hamiltonian(128)
    w, V = oracle.jacobi_eigh(H)
    P, _ = oracle.density_projector(w, V, nocc)
    r = C.fermi_operator(H, 0.0, 40.0, 32, 16)
    assert np.abs(r["D"] - P).max() <= 1e-6
    assert abs(np.trace(r["D"]) - nocc) <= 1e-6


def _mutants():
    """Oracle variants with one plausible mistake each."""
    def divide_factor(a, k):          # quotient coefficient without the factor 2
        a = np.array(a, dtype=np.float64)
        deg = len(a) - 1
        q = np.zeros(max(deg - k + 1, 1))
        for n in range(deg, k - 1, -1):
            v = a[n]
            a[n] = 0.0
            if n == k:
                q[0] += v
            else:
                q[n - k] += v
                a[abs(2 * k - n)] -= v
        r = np.zeros(k)
        r[:min(k, deg + 1)] = a[:min(k, deg + 1)]
        return r, q

    def doubling_sign(Ht, k):          # T_n = 2 T_a T_b + T_{a-b}
        T = [np.eye(Ht.shape[0]), np.asarray(Ht, dtype=np.float64).copy()]
        for n in range(2, k + 1):
            a, b = (n + 1) // 2, n // 2
            T.append(2.0 * (T[a] @ T[b]) + T[a - b])
        return T[:k + 1]

    def c0_not_halved(g, L, M=None):   # the n = 0 weight taken as 2 / M
        M = 2 * (L + 1) if M is None else M
        theta = np.pi * (np.arange(M) + 0.5) / M
        gx = g(np.cos(theta))
        return np.array([2.0 / M * float(np.sum(gx * np.cos(n * theta))) for n in range(L + 1)])
    return {"divide_factor": ("cheb_divide", divide_factor),
            "doubling_sign": ("chebyshev_polynomials", doubling_sign),
            "c0_not_halved": ("cheb_coefficients", c0_not_halved)}


@pytest.mark.parametrize("name", ["divide_factor", "doubling_sign", "c0_not_halved"])
def test_mutations_are_caught(name, monkeypatch):
    attr, fn = _mutants()[name]
    monkeypatch.setattr(C, attr, fn)
    rng = np.random.default_rng(9)
    H, w, Q = random_spectrum_matrix(24, rng, -2.0, 2.0)
    ref = (Q * C.fermi(w, 0.1, 3.0)) @ Q.T
    # unmutated, this case is within 2e-11 of the eigh-based result
    r = C.fermi_operator(H, 0.1, 3.0, 16, 8)
    assert np.abs(r["D"] - ref).max() > 1e-6, name


def test_mutation_case_is_accurate_unmutated():
    rng = np.random.default_rng(9)
    H, w, Q = random_spectrum_matrix(24, rng, -2.0, 2.0)
    ref = (Q * C.fermi(w, 0.1, 3.0)) @ Q.T
    assert np.abs(C.fermi_operator(H, 0.1, 3.0, 16, 8)["D"] - ref).max() <= 1e-10
