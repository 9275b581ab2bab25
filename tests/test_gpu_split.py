"""Split-precision (tcgen05) SP2 products through the C ABI against the CPU oracle.

Tolerances follow from the arithmetic: an FP16x2 operand carries 22
significant bits (2^-22 relative), BF16x3 carries 24, and the products
accumulate in FP32. For symmetric X with spectrum in [0, 1] every row has
norm <= 1, so one product X*X is off by at most ~2^-21 + FP32 accumulation
(< 5e-6 absolute, the single-product gate). Whole solves in split precision
inherit the accuracy of FP32 SP2 (gap-limited); the MIXED modes end with FP64
refinement and must meet max|D - D_ref| <= 1e-5 and |Tr D - Nocc| <= 1e-8.
"""

import numpy as np
import pytest

import oracle
from workloads import chain_hamiltonian, cube_hamiltonian

pytestmark = pytest.mark.gpu

TOL_PRODUCT = 5e-6
TOL_MIXED = 1e-5
TOL_TRACE = 1e-8


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


def host(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("prec,split_tile", [("fp32_split", 2), ("fp32_split", 1),
                                              ("mixed_bf16", 0)])
@pytest.mark.parametrize("sites", [32, 75, 160])
def test_single_split_product_matches_fp64(pkg, prec, split_tile, sites):
    # n = 128 (one tile), 300 (ragged, 3x3 tiles of 128 x 128, an odd number of
    # 128-column blocks for the 128 x 256 tiles), 640 (5x5 tiles)
    H, nocc = cube_hamiltonian(sites, 21)
    kw = {"prec": prec, "maxiter": 1, "split_tile": split_tile}
    if prec.startswith("mixed"):
        kw["fp64_prefix"] = 0
    D, info = pkg.sp2_dense_ex(dev(H), nocc, 0.0, raise_on_status=False, **kw)
    assert info["status"] == "ENOCONV" and info["iters"] == 1
    ref = oracle.sp2_plain(H, nocc, 0.0, stop_after=1)
    assert info["bits"] == ref["bits"]
    err = np.abs(host(D) - ref["D"]).max()
    assert err <= TOL_PRODUCT, err


def test_split_iterates_track_fp64(pkg):
    H, nocc = cube_hamiltonian(64, 8)  # n = 256
    for k in (2, 5, 10):
        D, info = pkg.sp2_dense_ex(dev(H), nocc, 0.0, prec="fp32_split", maxiter=k,
                                   raise_on_status=False)
        ref = oracle.sp2_plain(H, nocc, 0.0, stop_after=k)
        assert info["iters"] == k
        assert info["bits"] == ref["bits"]
        assert np.abs(host(D) - ref["D"]).max() <= TOL_PRODUCT * 4 * k


def test_chain_all_split_converges(pkg):
    H, nocc = chain_hamiltonian(512)
    w, V = oracle.jacobi_eigh(H)
    Dref, _ = oracle.density_projector(w, V, nocc)
    D, info = pkg.sp2_dense_ex(dev(H), nocc, 1e-12, prec="fp32_split")
    assert info["status"] == "OK" and info["converged"]
    # chain: large gap 0.8, low precision is not amplified
    assert np.abs(host(D) - Dref).max() <= 1e-5


@pytest.mark.parametrize("prec", ["mixed_fp16", "mixed_bf16"])
@pytest.mark.parametrize("sites,seed", [(75, 3), (250, 4)])
def test_mixed_solve_meets_gate(pkg, prec, sites, seed):
    H, nocc = cube_hamiltonian(sites, seed)
    w, V = oracle.jacobi_eigh(H)
    Dref, gap = oracle.density_projector(w, V, nocc)
    D, info = pkg.sp2_dense_ex(dev(H), nocc, 1e-10, prec=prec, fp64_prefix=12)
    assert info["status"] == "OK" and info["converged"], info
    assert info["phase_iters"][0] >= 1 and info["phase_iters"][1] >= 1 and info["phase_iters"][2] >= 1
    Dn = host(D)
    assert np.abs(Dn - Dref).max() <= TOL_MIXED
    assert abs(np.trace(Dn) - nocc) <= TOL_TRACE


def test_split_degenerate_and_status(pkg):
    H, nocc = cube_hamiltonian(16, 9)  # n = 64
    n = H.shape[0]
    D, info = pkg.sp2_dense_ex(dev(H), 0, 1e-10, prec="mixed_fp16")
    assert info["converged"] and np.abs(host(D)).max() <= 1e-8
    D, info = pkg.sp2_dense_ex(dev(H), n, 1e-10, prec="mixed_fp16")
    assert info["converged"] and np.abs(host(D) - np.eye(n)).max() <= 1e-8
    Hn = H.copy()
    Hn[1, 2] = Hn[2, 1] = np.inf
    D, info = pkg.sp2_dense_ex(dev(Hn), nocc, 1e-10, prec="fp32_split", raise_on_status=False)
    assert info["status"] == "EBOUNDS"
    D, info = pkg.sp2_dense_ex(dev(H), nocc, 1e-10, prec="mixed_bf16")
    assert info["converged"]


@pytest.mark.parametrize("prec", ["fp32_split", "mixed_fp16"])
@pytest.mark.parametrize("sites", [75, 250, 512, 700])
def test_wide_and_square_tiles_agree_bit_for_bit(pkg, prec, sites):
    """The FP16 split product on 128 x 256 tiles issues, per element, the same
    tensor-core products in the same order as the 128 x 128 kernel (leading
    group in 256-k chunks, corrections over the whole K), so whole solves give
    the same D and the same branch sequence. n = 300, 1000, 2048, 2800: ld =
    384, 1024, 2048, 2816, i.e. 3, 8, 16, 22 blocks of 128 (odd counts leave a
    half-empty last column pair); the mixed solves also write FP64 X' from the
    split epilogue before the refinement. Only the traces that each kernel sums
    for the branch test may differ, in the order of their partial sums."""
    H, nocc = cube_hamiltonian(sites, 33)
    Hd = dev(H)
    kw = dict(prec=prec, fp64_prefix=8)
    Dw, iw = pkg.sp2_dense_ex(Hd, nocc, 1e-9, split_tile=2, **kw)
    Ds, is_ = pkg.sp2_dense_ex(Hd, nocc, 1e-9, split_tile=1, **kw)
    assert iw["bits"] == is_["bits"] and iw["phase_iters"] == is_["phase_iters"]
    # the traces of the last product are partial sums in each kernel's own order
    assert abs(iw["trace"] - is_["trace"]) <= 1e-9 * nocc
    a, b = host(Dw), host(Ds)
    assert np.isfinite(a).all()
    assert np.array_equal(a, b), float(np.abs(a - b).max())


def test_split_tile_option_is_checked(pkg):
    H, nocc = cube_hamiltonian(32, 5)
    with pytest.raises(pkg.ProgressError):
        pkg.sp2_dense_ex(dev(H), nocc, 1e-9, prec="fp32_split", split_tile=3)
