"""The workloads at the sizes the benchmark runs, in the launch configuration
it times (default options: mixed FP16 schedule with digit-product prefix and
refinement; batched launch configuration from the autotuner).

N = 4096 (1024-site cube): the whole D against the oracle's plain FP64 SP2,
element by element (about 20 s of numpy on the host), for the mixed schedule
(gate 1e-5), plain FP64 (gate 1e-10) and the FP32-class all-split modes.
N = 8192 (2048 sites, the benchmark's headline): the whole D of the mixed FP16
and mixed BF16 schedules against one oracle solve (gates max |D - D_ref| <=
1e-5, |Tr D - Nocc| <= 1e-8), plus the invariants on sampled rows. 4000 batched parts:
the autotuned launch, then 40 parts sampled across the size range, each
against the oracle's plain FP64 SP2. The Chebyshev workload (N = 4096, L + 1 =
256): the whole D against the oracle's evaluation of the same expansion. The
thresholded workload (N = 16384 chain, tau = 1e-6): sampled rows against the
exact projector's band.
"""

import numpy as np
import pytest

import oracle
from workloads import batch_packed, batch_sizes, cube_hamiltonian

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


def solve(pkg, H, nocc, **opts):
    import torch
    Hd = torch.from_numpy(H).to("cuda:0")
    D, info = pkg.sp2_dense_ex(Hd, nocc, 1e-10, **opts)
    torch.cuda.synchronize()
    return D.cpu().numpy(), info


@pytest.fixture(scope="module")
def cube4096():
    """N = 4096 cube (1024 sites, seed 0) and one whole oracle solve of it
    (plain FP64 SP2, about 20 s of numpy on the host)."""
    H, nocc = cube_hamiltonian(1024, 0)
    ref = oracle.sp2_plain(H, nocc, 1e-10)
    assert ref["converged"]
    return H, nocc, ref


@pytest.fixture(scope="module")
def cube8192():
    """N = 8192 cube (2048 sites, seed 0) and one whole oracle solve of it
    (plain FP64 SP2, a few minutes of numpy on the host)."""
    H, nocc = cube_hamiltonian(2048, 0)
    ref = oracle.sp2_plain(H, nocc, 1e-10)
    assert ref["converged"]
    return H, nocc, ref


MIXED = dict(fp64_prefix=8)  # the benchmark's schedule: 8 FP64-accurate products first


def test_n4096_mixed_matches_oracle_elementwise(pkg, cube4096):
    H, nocc, ref = cube4096
    D, info = solve(pkg, H, nocc, prec="mixed_fp16", **MIXED)
    assert info["status"] == "OK" and info["converged"]
    err = float(np.abs(D - ref["D"]).max())
    assert err <= 1e-5, err                      # mixed-path gate
    assert abs(np.trace(D) - nocc) <= 1e-8
    assert np.array_equal(D, D.T)


def test_n4096_fp64_matches_oracle_elementwise(pkg, cube4096):
    # plain FP64 SP2 (native FP64 products) at the N = 4096 size: FP64 gate
    H, nocc, ref = cube4096
    D, info = solve(pkg, H, nocc, prec="fp64")
    assert info["status"] == "OK" and info["converged"]
    assert abs(info["iters"] - ref["iters"]) <= 1
    err = float(np.abs(D - ref["D"]).max())
    assert err <= 1e-10, err


@pytest.mark.parametrize("prec", ["fp32_split", "fp32_split_bf16"])
def test_n4096_fp32_split_matches_oracle_elementwise(pkg, cube4096, prec):
    # every product in FP32-class split precision, no FP64 refinement. Gate
    # (FP32-class reading): max |D - D_ref| <= 1e-4 and |Tr D - Nocc| <= 4 n 2^-22
    # -- the split phase stops on its round-off floor, where the idempotency
    # error, and with it the trace error, is of order n times the slices'
    # 2^-22 resolution (measured: 2.4e-5 and 1.5e-3 at N = 4096)
    H, nocc, ref = cube4096
    n = H.shape[0]
    D, info = solve(pkg, H, nocc, prec=prec)
    assert info["status"] == "OK" and info["converged"]
    err = float(np.abs(D - ref["D"]).max())
    tr = abs(np.trace(D) - nocc)
    print(f"{prec}: max|D - D_ref| = {err:.3e}, |Tr D - Nocc| = {tr:.3e}")
    assert err <= 1e-4, err
    assert tr <= 4.0 * n * 2.0 ** -22, tr


@pytest.mark.parametrize("prec", ["mixed_fp16", "mixed_bf16"])
def test_n8192_mixed_matches_oracle_elementwise(pkg, cube8192, prec):
    # the benchmark's headline workload: the whole D against the oracle's
    H, nocc, ref = cube8192
    D, info = solve(pkg, H, nocc, prec=prec, **MIXED)
    assert info["status"] == "OK" and info["converged"], info
    err = float(np.abs(D - ref["D"]).max())
    tr = abs(np.trace(D) - nocc)
    print(f"{prec} N=8192: max|D - D_ref| = {err:.3e}, |Tr D - Nocc| = {tr:.3e}, "
          f"phases {info['phase_iters']}")
    assert err <= 1e-5, err
    assert tr <= 1e-8, tr
    assert np.array_equal(D, D.T)


def test_n8192_mixed_properties_on_sampled_rows(pkg, cube8192):
    # smoke check of the invariants that hold at any size (not a parity test)
    H, nocc, _ = cube8192
    D, info = solve(pkg, H, nocc, prec="mixed_fp16", **MIXED)
    assert info["status"] == "OK" and info["converged"]
    n = H.shape[0]
    rows = np.random.default_rng(0).choice(n, size=64, replace=False)
    idem = float(np.abs(D[rows] @ D - D[rows]).max())
    comm = float(np.abs(H[rows] @ D - D[rows] @ H).max()) / float(np.abs(H).max())
    assert idem <= 1e-9, idem
    assert comm <= 1e-4, comm
    w = np.linalg.eigvalsh(D[np.ix_(rows, rows)])
    assert w.min() >= -1e-9 and w.max() <= 1.0 + 1e-9


def test_4000_part_batch_sampled_parts_match_oracle(pkg):
    import torch
    sites = batch_sizes(4000, 0)
    packed, n, offsets, nocc = batch_packed(sites, 1000)
    H = torch.from_numpy(packed).to("cuda:0")
    D = torch.empty_like(H)
    rep = pkg.batched_tune(H, n, offsets, nocc, 1e-10, D_packed=D,
                           sample_stride=max(1, len(n) // 600), reps=1)
    assert rep["tile_n"] in (64, 128) and rep["cluster"] in (1, 2, 4, 8)
    D, iters, status = pkg.sp2_batched(H, n, offsets, nocc, 1e-10, D_packed=D)
    torch.cuda.synchronize()
    assert (status.cpu().numpy() == 0).all()
    Dh = D.cpu().numpy()
    order = np.argsort(n, kind="stable")
    sample = order[np.linspace(0, len(n) - 1, 40).astype(int)]
    for i in sample:
        k = int(n[i])
        Hi = packed[offsets[i]:offsets[i] + k * k].reshape(k, k)
        Di = Dh[offsets[i]:offsets[i] + k * k].reshape(k, k)
        ref = oracle.sp2_plain(Hi, int(nocc[i]), 1e-10)["D"]
        w = np.linalg.eigvalsh(Hi)
        emin, emax = oracle.gershgorin_bounds(Hi)
        relgap = (w[nocc[i]] - w[nocc[i] - 1]) / (emax - emin)
        gate = min(0.2 * 2.0 ** -22 / relgap + 1e-6, 1e-2)  # as in test_gpu_batched.py
        assert float(np.abs(Di - ref).max()) <= gate, (i, k)
        assert abs(np.trace(Di) - nocc[i]) <= 4e-6 * k


def test_cheb_n4096_matches_oracle_elementwise(pkg):
    # the Chebyshev workload of the benchmark: C1's H, mu = 0.5 eV, beta = 1 / eV,
    # L + 1 = 256 (k = m = 16); the whole D against the oracle's FP64 evaluation of
    # the same expansion (gate as in test_gpu_cheb: 8 g max(1, beta b / 4) 2^-23)
    import torch
    from oracle import cheb as C
    H, _ = cube_hamiltonian(1024, 0)
    D, info = pkg.cheb_fermi(torch.from_numpy(H).to("cuda:0"), 0.5, 1.0, 16, 16)
    ref = C.fermi_operator(H, 0.5, 1.0, 16, 16)
    gate = 8.0 * 2.0 ** -23 * max(1.0, float(np.abs(ref["d"]).sum())) * max(1.0, ref["b"] / 4.0)
    err = float(np.abs(D.cpu().numpy() - ref["D"]).max())
    assert info["products"] == 30 and err <= gate, (err, gate)


def test_thresholded_n16384_chain_against_exact_band(pkg):
    # the thresholded workload of the benchmark: the N = 16384 dimerized chain,
    # tau = 1e-6; 64 sampled rows against the exact projector of a 512-site chain
    # (the same entries within 256 sites of the diagonal), zero beyond the band
    import torch
    from workloads import chain_hamiltonian
    n = 16384
    H, nocc = chain_hamiltonian(n, -1.0, -0.6)
    D, info = pkg.sp2_dense_ex(torch.from_numpy(H).to("cuda:0"), nocc, 1e-9,
                               prec="fp32_split", tau=1e-6)
    assert info["status"] == "OK" and info["converged"]
    Hs, ns = chain_hamiltonian(512, -1.0, -0.6)
    w, V = oracle.jacobi_eigh(Hs)
    P, _ = oracle.density_projector(w, V, ns)
    rows = np.linspace(0, n - 1, 64).astype(np.int64)
    Dn = D[torch.from_numpy(rows).to("cuda:0")].cpu().numpy()
    for k, r in enumerate(rows):
        off = (np.arange(n) - r + n // 2) % n - n // 2
        band = np.abs(off) < 256
        ref = P[r % 2, (r % 2 + off[band]) % 512]
        assert float(np.abs(Dn[k, band] - ref).max()) <= 4e-6 + 2e-5
        assert not Dn[k, ~band].any()
    T = n // 128
    assert info["kblocks"] < 1e-3 * info["iters"] * T * (T + 1) // 2 * (n // 64)
