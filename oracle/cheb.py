"""Chebyshev Fermi-operator expansion -- TEST INFRASTRUCTURE ONLY.

Plain FP64 statement of §IV.B of arXiv 2401.13772 (Eqs. 5-10), step by step:

1. The Hamiltonian is mapped into [-1, 1] with the Gershgorin bounds of
   §VIII.A: Ht = (H - a I) / b, a = (emax + emin) / 2, b = (emax - emin) / 2.
                                                   ``scaled_hamiltonian``
2. The Fermi-Dirac function of §III, f(e) = 1 / (1 + exp(beta (e - mu))),
   becomes g(x) = f(b x + a) on [-1, 1], and g ~ sum_{n=0}^{L} c_n T_n(x)
   (Eq. 5). The coefficients are those of the interpolant at the M = 2 (L + 1)
   Chebyshev-Gauss nodes x_j = cos(theta_j), theta_j = pi (j + 1/2) / M:
   c_n = (2 - [n = 0]) / M * sum_j g(x_j) cos(n theta_j). (A reading: the
   paper calls c_n the Chebyshev expansion coefficients without fixing how
   they are computed, and applies no damping kernel.)     ``cheb_coefficients``
3. Serial evaluation (Eq. 6): T_0 = I, T_1 = Ht, T_{n+1} = 2 Ht T_n - T_{n-1},
   and the sum of c_n T_n.                                ``serial_chebyshev``
4. Paterson-Stockmeyer form (Eq. 7), L + 1 = k m:
   sum c_n T_n = S_0 + T_k (S_1 + T_k (S_2 + ... + T_k S_{m-1})), with
   S_j = sum_{i<k} d_{i,j} T_i (Eq. 9). The d_{i,j} follow from the product
   rule T_a T_b = (T_{a+b} + T_{|a-b|}) / 2 (Eq. 8), written as
   T_n = 2 T_k T_{n-k} - T_{|2k-n|}: dividing the series by T_k, highest
   degree first, leaves a remainder of degree < k (S_0) and a quotient
   series, which is divided again for S_1, and so on.     ``ps_coefficients``
5. T_2 ... T_k from the same rule (Eqs. 10-11): T_n = 2 T_a T_b - T_{a-b}
   with a = ceil(n/2), b = floor(n/2), so that every T_n of
   (2^(l-1), 2^l] needs only polynomials of lower levels (the products of one
   level are independent).                                ``chebyshev_polynomials``
6. The nested (Horner-like) evaluation of step 4.        ``ps_evaluate``

``fermi_operator`` runs steps 1, 2, 4, 5, 6: the density matrix at a known
chemical potential and inverse temperature.

numpy's matmul is the only library primitive (the matrix products).
"""

from __future__ import annotations

import numpy as np

from .sp2 import gershgorin_bounds


def fermi(e, mu, beta):
    """Fermi-Dirac occupation 1 / (1 + exp(beta (e - mu))) (§III), written as
    (1 - tanh(beta (e - mu) / 2)) / 2, which does not overflow."""
    return 0.5 * (1.0 - np.tanh(0.5 * beta * (np.asarray(e, dtype=np.float64) - mu)))


def scaled_hamiltonian(H, emin, emax):
    """Ht = (H - a I) / b with a = (emax + emin) / 2, b = (emax - emin) / 2.
    Returns (Ht, a, b). A zero-width interval is widened by 1 on each side."""
    H = np.asarray(H, dtype=np.float64)
    if not emax > emin:
        emin, emax = emin - 1.0, emax + 1.0
    a = 0.5 * (emax + emin)
    b = 0.5 * (emax - emin)
    return (H - a * np.eye(H.shape[0])) / b, a, b


def cheb_coefficients(g, L, M=None):
    """c_0..c_L of the Chebyshev interpolant of g at M Chebyshev-Gauss nodes."""
    if M is None:
        M = 2 * (L + 1)
    theta = np.pi * (np.arange(M) + 0.5) / M
    gx = np.asarray(g(np.cos(theta)), dtype=np.float64)
    c = np.empty(L + 1)
    for n in range(L + 1):
        c[n] = (2.0 if n else 1.0) / M * float(np.sum(gx * np.cos(n * theta)))
    return c


def cheb_divide(a, k):
    """Divide the Chebyshev series a (coefficients of T_0, T_1, ...) by T_k:
    a = r + T_k q with deg r < k. Returns (r, q)."""
    a = np.array(a, dtype=np.float64)
    deg = len(a) - 1
    q = np.zeros(max(deg - k + 1, 1))
    for n in range(deg, k - 1, -1):
        v = a[n]
        a[n] = 0.0
        if n == k:          # T_k = T_k T_0
            q[0] += v
        else:               # T_n = 2 T_k T_{n-k} - T_{|2k-n|}
            q[n - k] += 2.0 * v
            a[abs(2 * k - n)] -= v
    r = np.zeros(k)
    r[:min(k, deg + 1)] = a[:min(k, deg + 1)]
    return r, q


def ps_coefficients(c, k, m):
    """d (k x m): column j holds the coefficients of S_j in Eq. 7 (L + 1 = k m)."""
    c = np.asarray(c, dtype=np.float64)
    if len(c) != k * m:
        raise ValueError("need L + 1 = k m coefficients")
    d = np.zeros((k, m))
    rest = c
    for j in range(m - 1):
        r, rest = cheb_divide(rest, k)
        d[:, j] = r
    d[:len(rest), m - 1] = rest[:k]
    return d


def chebyshev_polynomials(Ht, k):
    """[T_0, ..., T_k] of the matrix Ht by T_n = 2 T_a T_b - T_{a-b},
    a = ceil(n/2), b = floor(n/2) (Eqs. 10-11)."""
    Ht = np.asarray(Ht, dtype=np.float64)
    T = [np.eye(Ht.shape[0]), Ht.copy()]
    for n in range(2, k + 1):
        a, b = (n + 1) // 2, n // 2
        T.append(2.0 * (T[a] @ T[b]) - T[a - b])
    return T[:k + 1]


def serial_chebyshev(Ht, c):
    """sum_n c_n T_n(Ht) with the three-term recursion of Eq. 6."""
    Ht = np.asarray(Ht, dtype=np.float64)
    Tm, T = np.eye(Ht.shape[0]), Ht.copy()
    F = c[0] * Tm
    if len(c) > 1:
        F = F + c[1] * T
    for n in range(1, len(c) - 1):
        Tm, T = T, 2.0 * (Ht @ T) - Tm
        F = F + c[n + 1] * T
    return F


def ps_evaluate(Ht, d):
    """S_0 + T_k (S_1 + T_k (... + T_k S_{m-1})) with S_j = sum_i d_ij T_i."""
    k, m = d.shape
    T = chebyshev_polynomials(Ht, k)
    S = [sum(d[i, j] * T[i] for i in range(k)) for j in range(m)]
    P = S[m - 1]
    for j in range(m - 2, -1, -1):
        P = S[j] + T[k] @ P
    return P


def fermi_operator(H, mu, beta, k, m, bounds=None):
    """Density matrix f(H) at chemical potential mu and inverse temperature
    beta by the Paterson-Stockmeyer Chebyshev expansion with L + 1 = k m.
    Returns dict(D, c, d, a, b, emin, emax)."""
    H = np.asarray(H, dtype=np.float64)
    emin, emax = gershgorin_bounds(H) if bounds is None else bounds
    Ht, a, b = scaled_hamiltonian(H, emin, emax)
    c = cheb_coefficients(lambda x: fermi(b * x + a, mu, beta), k * m - 1)
    d = ps_coefficients(c, k, m)
    return {"D": ps_evaluate(Ht, d), "c": c, "d": d, "a": a, "b": b,
            "emin": emin, "emax": emax}
