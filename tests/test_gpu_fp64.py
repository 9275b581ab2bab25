"""FP64 SP2 on the GPU through the C ABI, element by element against the CPU oracle."""

import json
import os

import numpy as np
import pytest

import oracle
from workloads import chain_hamiltonian, cube_hamiltonian

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10  # max |D - D_ref| gate of the FP64 path


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


def test_gershgorin_matches_oracle(pkg):
    for H in (chain_hamiltonian(512)[0], cube_hamiltonian(70, 1)[0], np.array([[3.5]])):
        b = host(pkg.gershgorin_bounds(dev(H)))
        emin, emax = oracle.gershgorin_bounds(H)
        assert abs(b[0] - emin) <= 1e-12 * max(1.0, abs(emin))
        assert abs(b[1] - emax) <= 1e-12 * max(1.0, abs(emax))


def test_gershgorin_row_sums_are_exactly_rounded(pkg):
    # the row sums R_i = sum_{j != i} |H_ij| are accumulated exactly (fixed point)
    # and rounded once: against exact rational arithmetic on entries spread over
    # 60 orders of magnitude, with zeros and subnormal entries
    from fractions import Fraction
    rng = np.random.default_rng(3)
    for n in (1, 7, 64, 333):
        A = rng.standard_normal((n, n)) * np.exp(rng.uniform(-70, 70, (n, n)))
        A[rng.uniform(size=(n, n)) < 0.3] = 0.0
        if n > 1:
            A[0, 1] = 5e-320  # subnormal
        H = np.triu(A) + np.triu(A, 1).T
        b = host(pkg.gershgorin_bounds(dev(H)))
        lo = hi = None
        for i in range(n):
            R = sum((Fraction(abs(float(H[i, j]))) for j in range(n) if j != i), Fraction(0))
            d = Fraction(float(H[i, i]))
            lo = d - R if lo is None else min(lo, d - R)
            hi = d + R if hi is None else max(hi, d + R)
        scale = max(abs(float(lo)), abs(float(hi)), 1e-300)
        assert abs(b[0] - float(lo)) <= 4e-16 * scale, (n, b[0], float(lo))
        assert abs(b[1] - float(hi)) <= 4e-16 * scale, (n, b[1], float(hi))
    # a non-finite entry gives non-finite bounds (the solve then reports EBOUNDS)
    H = cube_hamiltonian(16, 1)[0]
    H[3, 5] = H[5, 3] = np.inf
    b = host(pkg.gershgorin_bounds(dev(H)))
    assert not np.isfinite(b).all()


@pytest.mark.parametrize("n", [301, 300])
def test_odd_order_and_unaligned_input(pkg, n):
    # an odd order (rows not on 16-byte boundaries) and an H whose first entry
    # sits 8 bytes past a 16-byte boundary: the O(n^2) kernels take their
    # scalar paths; bounds and solves must not change
    import torch
    rng = np.random.default_rng(n)
    nocc = n // 2
    w = np.concatenate([rng.uniform(-3.0, -0.5, nocc), rng.uniform(0.5, 3.0, n - nocc)])
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    H = (Q * w) @ Q.T
    H = (H + H.T) / 2
    Dref = Q[:, :nocc] @ Q[:, :nocc].T
    buf = torch.zeros(n * n + 1, dtype=torch.float64, device="cuda:0")
    Hv = buf[1:].view(n, n)
    Hv.copy_(torch.from_numpy(H))
    assert Hv.data_ptr() % 16 == 8
    b = host(pkg.gershgorin_bounds(Hv))
    emin, emax = oracle.gershgorin_bounds(H)
    assert abs(b[0] - emin) <= 1e-12 * abs(emin) and abs(b[1] - emax) <= 1e-12 * abs(emax)
    D, info = pkg.sp2_dense_ex(Hv, nocc, 1e-12)
    assert info["status"] == "OK" and np.abs(host(D) - Dref).max() <= TOL_FP64
    D, info = pkg.sp2_dense_ex(Hv, nocc, 1e-10, prec="mixed_fp16", fp64_prefix=8)
    assert info["status"] == "OK" and np.abs(host(D) - Dref).max() <= 1e-5


def test_chain_512_matches_projector_and_golden_bits(pkg):
    H, nocc = chain_hamiltonian(512, -1.0, -0.6)
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "chain512_sp2.json")))
    w, V = oracle.jacobi_eigh(H)
    Dref, _ = oracle.density_projector(w, V, nocc)
    for rule in ("nearer", "paper"):
        for loop_mode in (0, 1):
            D, info = pkg.sp2_dense_ex(dev(H), nocc, 1e-12, rule=rule, loop_mode=loop_mode)
            assert info["status"] == "OK" and info["converged"]
            assert info["iters"] == g[rule]["iters"]
            assert "".join(map(str, info["bits"])) == g[rule]["bits"]
            assert info["emin"] == -1.6 and info["emax"] == 1.6
            assert np.abs(host(D) - Dref).max() <= TOL_FP64


@pytest.mark.parametrize("sites,seed", [(32, 1), (75, 2), (128, 3), (250, 4)])
def test_cube_ragged_sizes_match_projector(pkg, sites, seed):
    # n = 128, 300, 512, 1000: one tile, several tiles with a ragged tail
    H, nocc = cube_hamiltonian(sites, seed)
    w, V = oracle.jacobi_eigh(H)
    Dref, gap = oracle.density_projector(w, V, nocc)
    D, info = pkg.sp2_dense_ex(dev(H), nocc, 1e-12)
    assert info["status"] == "OK" and info["converged"], info
    assert np.abs(host(D) - Dref).max() <= TOL_FP64
    ref = oracle.sp2_plain(H, nocc, 1e-12)
    assert abs(info["iters"] - ref["iters"]) <= 1


def test_intermediate_iterates_match_plain_sp2(pkg):
    # maxiter = k stops with ENOCONV and leaves X_k in D
    H, nocc = cube_hamiltonian(75, 5)  # n = 300
    for k in (1, 2, 7, 20):
        D, info = pkg.sp2_dense_ex(dev(H), nocc, 0.0, maxiter=k, raise_on_status=False)
        assert info["status"] == "ENOCONV" and info["iters"] == k
        ref = oracle.sp2_plain(H, nocc, 0.0, stop_after=k)
        assert info["bits"] == ref["bits"]
        assert np.abs(host(D) - ref["D"]).max() <= 1e-12
        assert abs(info["trace"] - ref["t1"][-1]) <= 1e-9


def test_degenerate_cases(pkg):
    import torch
    H, _ = cube_hamiltonian(16, 9)  # n = 64
    n = H.shape[0]
    D, info = pkg.sp2_dense_ex(dev(H), 0, 1e-12)
    assert info["converged"] and np.abs(host(D)).max() <= 1e-12
    D, info = pkg.sp2_dense_ex(dev(H), n, 1e-12)
    assert info["converged"] and np.abs(host(D) - np.eye(n)).max() <= 1e-12
    # 1 x 1
    D, info = pkg.sp2_dense_ex(dev(np.array([[0.7]])), 1, 1e-12)
    assert abs(host(D)[0, 0] - 1.0) <= 1e-12
    D, info = pkg.sp2_dense_ex(dev(np.array([[0.7]])), 0, 1e-12)
    assert abs(host(D)[0, 0]) <= 1e-12
    # diagonal H: exact occupation of the nocc lowest levels
    d = np.random.default_rng(3).permutation(np.linspace(-2.0, 3.0, 200))
    D, info = pkg.sp2_dense_ex(dev(np.diag(d)), 77, 1e-13)
    expect = np.zeros(200)
    expect[np.argsort(d)[:77]] = 1.0
    assert np.abs(host(D) - np.diag(expect)).max() <= 1e-12
    # n = 0
    z = torch.empty((0, 0), dtype=torch.float64, device="cuda:0")
    D, info = pkg.sp2_dense_ex(z, 0, 1e-12)
    assert info["converged"]


def test_bad_bounds_and_nonfinite_input_report_status(pkg):
    H, nocc = cube_hamiltonian(32, 2)
    emin, emax = oracle.gershgorin_bounds(H)
    w = np.linalg.eigvalsh(H)
    # bounds that cut the spectrum: the iterate leaves [0, 1]
    D, info = pkg.sp2_dense_ex(dev(H), nocc, 1e-12, emin=w[3], emax=w[-3],
                               raise_on_status=False)
    assert info["status"] in ("EBOUNDS", "ENOCONV")
    Hn = H.copy()
    Hn[3, 5] = Hn[5, 3] = np.nan
    D, info = pkg.sp2_dense_ex(dev(Hn), nocc, 1e-12, raise_on_status=False)
    assert info["status"] == "EBOUNDS"
    # the library stays usable afterwards
    D, info = pkg.sp2_dense_ex(dev(H), nocc, 1e-12)
    assert info["converged"]
    # tighter (exact) bounds are accepted and converge to the same D
    D1, i1 = pkg.sp2_dense_ex(dev(H), nocc, 1e-12, emin=w[0], emax=w[-1])
    D2, i2 = pkg.sp2_dense_ex(dev(H), nocc, 1e-12)
    assert np.abs(host(D1) - host(D2)).max() <= 1e-10
    assert i1["iters"] <= i2["iters"]


def test_async_entry_point_and_query(pkg):
    import torch
    H, nocc = cube_hamiltonian(64, 11)
    Hd = dev(H)
    D = pkg.sp2_dense(Hd, nocc, 1e-12)
    from paper_2401_13772_gb300 import _lib
    import ctypes
    info = _lib.Info()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert pkg.load().progress_sp2_query(s, ctypes.byref(info)) == _lib.OK
    assert info.converged == 1
    ref = oracle.sp2_plain(H, nocc, 1e-12)
    assert np.abs(host(D) - ref["D"]).max() <= TOL_FP64
    # in place (dD == dH) is allowed in the _ex entry point
    Hd2 = dev(H)
    out, _ = pkg.sp2_dense_ex(Hd2, nocc, 1e-12, D=Hd2)
    assert np.abs(host(out) - ref["D"]).max() <= TOL_FP64


def test_streams_are_independent(pkg):
    import torch
    H1, n1 = cube_hamiltonian(40, 1)
    H2, n2 = chain_hamiltonian(256)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    A1, A2 = dev(H1), dev(H2)
    torch.cuda.synchronize()
    with torch.cuda.stream(s1):
        D1 = pkg.sp2_dense(A1, n1, 1e-12, stream=s1)
    with torch.cuda.stream(s2):
        D2 = pkg.sp2_dense(A2, n2, 1e-12, stream=s2)
    torch.cuda.synchronize()
    assert np.abs(host(D1) - oracle.sp2_plain(H1, n1, 1e-12)["D"]).max() <= TOL_FP64
    assert np.abs(host(D2) - oracle.sp2_plain(H2, n2, 1e-12)["D"]).max() <= TOL_FP64
    pkg.release(s1)
    pkg.release(s2)


def test_df64_products_match_plain_sp2(pkg):
    """Double-float products (pairs of FP32, ~2^-47 relative) track the FP64
    iterates to ~1e-12 and the whole solve meets the FP64 gate."""
    H, nocc = cube_hamiltonian(75, 5)  # n = 300, ragged
    for k in (1, 5):
        D, info = pkg.sp2_dense_ex(dev(H), nocc, 0.0, prec="df64", maxiter=k,
                                   raise_on_status=False)
        ref = oracle.sp2_plain(H, nocc, 0.0, stop_after=k)
        assert info["bits"] == ref["bits"]
        assert np.abs(host(D) - ref["D"]).max() <= 1e-11
    for sites, seed in ((75, 2), (250, 4)):
        H, nocc = cube_hamiltonian(sites, seed)
        w, V = oracle.jacobi_eigh(H)
        Dref, _ = oracle.density_projector(w, V, nocc)
        D, info = pkg.sp2_dense_ex(dev(H), nocc, 1e-10, prec="df64")
        assert info["status"] == "OK" and info["converged"]
        assert np.abs(host(D) - Dref).max() <= TOL_FP64


@pytest.mark.parametrize("prefix_full,tol", [(1, 1e-10), (0, 1e-9)])
def test_digit_products_match_plain_sp2(pkg, prefix_full, tol):
    """FP64-accurate products as exact BF16 digit products on the tensor cores
    (fp64_impl 3): with a prefix longer than the run, every product is one of
    them; the iterates track the FP64 oracle's. All 15 digit products
    (prefix_full 1): digits carry 2^-44 absolute, the products ~2^-40, gate
    1e-10. The prefix's short form (13 products) drops x0 x4^T + x4 x0^T, at
    most 2 sqrt(K) 2^-36 per entry and product (5e-10 at K = 300), of random
    sign (~1e-11 typical): gate 1e-9. A wrong digit product is off by 1e-6 or
    more."""
    for sites, seed in ((75, 5), (32, 3)):  # n = 300 (ragged, 3 row blocks), 128 (one tile)
        H, nocc = cube_hamiltonian(sites, seed)
        for k in (1, 2, 6, 14):
            D, info = pkg.sp2_dense_ex(dev(H), nocc, 0.0, prec="mixed_fp16", fp64_impl=3,
                                       fp64_prefix=60, maxiter=k, raise_on_status=False,
                                       prefix_full=prefix_full)
            ref = oracle.sp2_plain(H, nocc, 0.0, stop_after=k)
            assert info["iters"] == k and info["bits"] == ref["bits"]
            assert np.abs(host(D) - ref["D"]).max() <= tol, (sites, k)
            assert abs(info["trace"] - ref["t1"][-1]) <= 1e-8


def test_digit_product_mixed_solve_meets_mixed_gate(pkg):
    """n = 1000 (8 chunks of 128 k for the exact G2 drain): the whole mixed
    solve with digit-product prefix (short form, and all 15 products) and
    refinement."""
    H, nocc = cube_hamiltonian(250, 4)
    w, V = oracle.jacobi_eigh(H)
    Dref, _ = oracle.density_projector(w, V, nocc)
    for fmt, prefix_full in (("mixed_fp16", 0), ("mixed_bf16", 0), ("mixed_fp16", 1)):
        D, info = pkg.sp2_dense_ex(dev(H), nocc, 1e-10, prec=fmt, fp64_impl=3, fp64_prefix=8,
                                   prefix_full=prefix_full)
        assert info["status"] == "OK" and info["converged"], info
        Dn = host(D)
        assert np.abs(Dn - Dref).max() <= 1e-5
        assert abs(np.trace(Dn) - nocc) <= 1e-8
        assert info["phase_iters"][0] == 8 and info["phase_iters"][2] >= 1


def test_mixed_with_native_and_double_float_fp64_phases(pkg):
    H, nocc = cube_hamiltonian(250, 4)
    w, V = oracle.jacobi_eigh(H)
    Dref, _ = oracle.density_projector(w, V, nocc)
    for impl in (0, 1, 2):  # default (digit products here), native FP64, double-float
        D, info = pkg.sp2_dense_ex(dev(H), nocc, 1e-10, prec="mixed_fp16", fp64_impl=impl)
        assert info["status"] == "OK" and info["converged"]
        Dn = host(D)
        assert np.abs(Dn - Dref).max() <= 1e-5
        assert abs(np.trace(Dn) - nocc) <= 1e-8
