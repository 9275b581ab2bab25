"""Chebyshev Fermi-operator expansion (§IV.B, Paterson-Stockmeyer form) on the
GPU against the CPU oracle (oracle/cheb.py), element by element.

Tolerance, from the arithmetic: each product is FP32-class (16-bit operand
slices, FP32 accumulation; the tensor core's truncating accumulation leaves a
measured diagonal bias of about 6e-7 per square of a matrix with diagonal
entries near +-1, a few units of 2^-23). An absolute perturbation u of Ht moves
f(Ht) by at most max|f'| u = (beta b / 4) u in scaled units (b the half-width of
the bounds), and the nested sums can be larger than D by the growth factor
g = sum |d_ij|. So the error is of order g max(1, beta b / 4) 2^-23; measured
0.25-0.5 of that. The gate is 8 times the estimate for both slice formats (the
accumulation, not the slice rounding, sets the floor)."""

import numpy as np
import pytest

from oracle import cheb as C
from workloads import chain_hamiltonian, cube_hamiltonian

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    assert torch.cuda.is_available(), "GPU test run without a CUDA device"
    from paper_2401_13772_gb300.build import build
    build()
    import paper_2401_13772_gb300 as p
    p.load()
    return p


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def gate(ref, beta, prec):
    g = max(1.0, float(np.abs(ref["d"]).sum()))
    slope = max(1.0, beta * ref["b"] / 4.0)
    return 8.0 * 2.0 ** -23 * g * slope


# (the S_j pass takes its coefficient table in 16 x 16, 32 x 32 or 64 x 64 form)
# k <= 16 (and k >= 2) runs the TMA-staged sum pass, k = 1 and k > 16 the direct
# ones; (75, 2, 5) is the staged pass with a single T plane per box, (75, 7, 1)
# its FP64 output of D
CASES = [(75, 16, 16), (75, 8, 4), (75, 5, 3), (75, 1, 6), (75, 7, 1), (75, 1, 1), (32, 16, 16),
         (33, 4, 8), (33, 20, 20), (33, 40, 3), (33, 64, 2), (75, 2, 5)]


@pytest.mark.parametrize("prec", ["fp32_split", "fp32_split_bf16"])
@pytest.mark.parametrize("sites,k,m", CASES)
def test_cheb_matches_oracle(pkg, sites, k, m, prec):
    # n = 300 (3 x 3 tiles, ragged), 128 (one tile), 132 (one tile + 4)
    H, _ = cube_hamiltonian(sites, 7)
    mu, beta = 0.3, 0.8
    ref = C.fermi_operator(H, mu, beta, k, m)
    D, info = pkg.cheb_fermi(dev(H), mu, beta, k, m, prec=prec)
    Dh = D.cpu().numpy()
    err = float(np.abs(Dh - ref["D"]).max())
    assert err <= gate(ref, beta, prec), (err, gate(ref, beta, prec))
    assert np.array_equal(Dh, Dh.T)
    k_top = k if m > 1 else k - 1
    assert info["products"] == max(k_top - 1, 0) + (m - 1)
    assert abs(info["trace"] - np.trace(Dh)) <= 1e-9 * max(1.0, abs(np.trace(Dh)))
    assert (info["emin"], info["emax"]) == pytest.approx(
        (ref["emin"], ref["emax"]), rel=1e-12, abs=1e-12)


def test_cheb_converges_to_fermi_dirac(pkg):
    # enough terms that truncation is far below the slice rounding: the GPU
    # result is the eigendecomposition's f(H) to the rounding gate
    H, _ = cube_hamiltonian(75, 11)
    mu, beta = -0.5, 0.5
    w, V = np.linalg.eigh(H)
    exact = (V * C.fermi(w, mu, beta)) @ V.T
    ref = C.fermi_operator(H, mu, beta, 16, 16)
    assert float(np.abs(ref["D"] - exact).max()) <= 1e-9
    D, info = pkg.cheb_fermi(dev(H), mu, beta, 16, 16)
    assert float(np.abs(D.cpu().numpy() - exact).max()) <= gate(ref, beta, "fp32_split") + 1e-9
    assert abs(info["trace"] - C.fermi(w, mu, beta).sum()) <= 1e-3


def test_cheb_explicit_bounds_and_repeatability(pkg):
    H, _ = cube_hamiltonian(40, 2)
    emin, emax = -30.0, 25.0  # wider than Gershgorin: still encloses the spectrum
    ref = C.fermi_operator(H, 0.0, 1.0, 16, 8, bounds=(emin, emax))
    Hd = dev(H)
    D1, info = pkg.cheb_fermi(Hd, 0.0, 1.0, 16, 8, bounds=(emin, emax))
    D2, _ = pkg.cheb_fermi(Hd, 0.0, 1.0, 16, 8, bounds=(emin, emax))
    assert (info["emin"], info["emax"]) == (emin, emax)
    assert float(np.abs(D1.cpu().numpy() - ref["D"]).max()) <= gate(ref, 1.0, "fp32_split")
    assert bool((D1 == D2).all())  # no atomics in the sums: bit-identical


def test_cheb_degenerate_cases(pkg):
    # n = 1: zero-width interval widened by 1, D = f(h)
    D, info = pkg.cheb_fermi(dev(np.array([[0.7]])), 0.2, 3.0, 8, 4)
    assert abs(float(D.cpu().numpy()[0, 0]) - C.fermi(0.7, 0.2, 3.0)) <= 1e-5
    # beta = 0: D = I / 2
    H, _ = cube_hamiltonian(20, 1)
    D, _ = pkg.cheb_fermi(dev(H), 0.0, 0.0, 4, 4)
    assert float(np.abs(D.cpu().numpy() - 0.5 * np.eye(80)).max()) <= 1e-6
    # mu far above the spectrum: D = I
    D, _ = pkg.cheb_fermi(dev(H), 1e3, 2.0, 8, 8)
    assert float(np.abs(D.cpu().numpy() - np.eye(80)).max()) <= 1e-5


def test_cheb_low_temperature_chain_is_the_projector(pkg):
    # gapped chain at mu mid-gap and large beta: the density matrix is the
    # zero-temperature projector (the SP2 answer) to the truncation + gate
    H, nocc = chain_hamiltonian(384)
    w, V = np.linalg.eigh(H)
    P = V[:, :nocc] @ V[:, :nocc].T
    ref = C.fermi_operator(H, 0.0, 40.0, 32, 16)
    assert float(np.abs(ref["D"] - P).max()) <= 1e-6
    D, info = pkg.cheb_fermi(dev(H), 0.0, 40.0, 32, 16)
    assert float(np.abs(D.cpu().numpy() - ref["D"]).max()) <= gate(ref, 40.0, "fp32_split")
    assert abs(info["trace"] - nocc) <= 1e-3
