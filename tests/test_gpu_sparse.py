"""Thresholded SP2 (Listing 1's cutoff tau) on the GPU against the CPU oracle
(oracle/sparse.py).

Tolerance: the products are FP32-class split products (about 2^-22 relative
per entry), and an element within that of tau may be pruned on one side and
kept on the other, a difference of at most tau in that element; SP2 contracts
perturbations near convergence (its maps have zero slope at 0 and 1), so the
gate is 4 tau + 2e-5 (the dense FP32-split gate of the chain)."""

import numpy as np
import pytest

from oracle import sparse as S
from workloads import chain_hamiltonian

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


def gate(tau):
    return 4.0 * tau + 2e-5


@pytest.mark.parametrize("prec", ["fp32_split", "fp32_split_bf16"])
@pytest.mark.parametrize("n,tau", [(256, 1e-6), (1000, 1e-6), (2048, 1e-5), (1000, 1e-3)])
def test_thresholded_chain_matches_oracle(pkg, n, tau, prec):
    H, nocc = chain_hamiltonian(n)
    ref = S.sp2_thresholded(H, nocc, 1e-9, tau)
    D, info = pkg.sp2_dense_ex(dev(H), nocc, 1e-9, prec=prec, tau=tau)
    Dh = D.cpu().numpy()
    err = float(np.abs(Dh - ref["D"]).max())
    assert err <= gate(tau), (err, gate(tau))
    # (the all-split mode stops once the idempotency error sits on its FP32 floor
    # for two steps, which can be several products after the FP64 oracle's tol)
    assert info["converged"] and info["iters"] >= ref["iters"] - 1
    # pruned: no element strictly inside (0, tau) beyond FP32 rounding of the cut
    a = np.abs(Dh)
    assert not ((a > 0) & (a < 0.999 * tau)).any()
    # sparsity close to the oracle's, and the tile counter saw fewer tiles than dense
    nnz, nnz_ref = np.count_nonzero(Dh), np.count_nonzero(ref["D"])
    assert abs(nnz - nnz_ref) <= 0.02 * nnz_ref + 4 * n
    T = (n + 127) // 128
    dense_kblocks = info["iters"] * T * (T + 1) // 2 * (T * 2)
    assert 0 < info["kblocks"] <= dense_kblocks
    if n >= 1000 and tau <= 1e-5:
        assert info["kblocks"] < 0.8 * dense_kblocks


def test_decoupled_blocks_stay_zero(pkg):
    # two chains in one matrix: the off-diagonal block never gets a non-zero,
    # its tiles are never streamed and never written after the first product
    A, na = chain_hamiltonian(512)
    B, nb = chain_hamiltonian(640, -0.9, -0.5)
    H = np.zeros((1152, 1152))
    H[:512, :512] = A
    H[512:, 512:] = B
    nocc = na + nb
    ref = S.sp2_thresholded(H, nocc, 1e-9, 1e-6)
    D, info = pkg.sp2_dense_ex(dev(H), nocc, 1e-9, prec="fp32_split", tau=1e-6)
    Dh = D.cpu().numpy()
    assert float(np.abs(Dh - ref["D"]).max()) <= gate(1e-6)
    assert not Dh[:512, 512:].any() and not Dh[512:, :512].any()


def test_tau_zero_is_the_dense_split_path(pkg):
    import torch
    H, nocc = chain_hamiltonian(512)
    Hd = dev(H)
    D0, i0 = pkg.sp2_dense_ex(Hd, nocc, 1e-9, prec="fp32_split")
    D1, i1 = pkg.sp2_dense_ex(Hd, nocc, 1e-9, prec="fp32_split", tau=0.0)
    assert bool(torch.equal(D0, D1)) and i1["kblocks"] == 0 and i0["iters"] == i1["iters"]


def test_thresholded_then_dense_reuses_the_workspace(pkg):
    # switching tau on and off on one stream rebuilds the loop graph each time
    H, nocc = chain_hamiltonian(384)
    Hd = dev(H)
    ref_sparse = S.sp2_thresholded(H, nocc, 1e-9, 1e-5)["D"]
    for _ in range(2):
        Ds, _ = pkg.sp2_dense_ex(Hd, nocc, 1e-9, prec="fp32_split", tau=1e-5)
        Dd, _ = pkg.sp2_dense_ex(Hd, nocc, 1e-9, prec="fp32_split")
        assert float(np.abs(Ds.cpu().numpy() - ref_sparse).max()) <= gate(1e-5)
        assert np.count_nonzero(Dd.cpu().numpy()) > np.count_nonzero(Ds.cpu().numpy())
