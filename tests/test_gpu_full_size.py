"""The workloads at the sizes the benchmark runs, in the launch configuration
it times (default options: mixed FP16 schedule with digit-product prefix and
refinement; batched launch configuration from the autotuner).

N = 4096 (1024-site cube): the whole D against the oracle's plain FP64 SP2,
element by element (about 20 s of numpy on the host). N = 8192 (2048 sites):
properties that hold at any size, on sampled rows -- symmetry, Tr D = Nocc,
D^2 = D and [H, D] = 0 -- with the exact gate on Tr D. 4000 batched parts:
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


def bench_solve(pkg, sites):
    import torch
    H, nocc = cube_hamiltonian(sites, 0)
    Hd = torch.from_numpy(H).to("cuda:0")
    D, info = pkg.sp2_dense_ex(Hd, nocc, 1e-10, prec="mixed_fp16", fp64_prefix=8)
    torch.cuda.synchronize()
    return H, nocc, D.cpu().numpy(), info


def test_n4096_mixed_matches_oracle_elementwise(pkg):
    H, nocc, D, info = bench_solve(pkg, 1024)
    assert info["status"] == "OK" and info["converged"]
    ref = oracle.sp2_plain(H, nocc, 1e-10)
    assert ref["converged"]
    err = float(np.abs(D - ref["D"]).max())
    assert err <= 1e-5, err                      # mixed-path gate
    assert abs(np.trace(D) - nocc) <= 1e-8
    assert np.array_equal(D, D.T)


def test_n8192_mixed_properties_on_sampled_rows(pkg):
    H, nocc, D, info = bench_solve(pkg, 2048)
    assert info["status"] == "OK" and info["converged"]
    n = H.shape[0]
    assert np.array_equal(D, D.T)
    assert abs(np.trace(D) - nocc) <= 1e-8
    rows = np.random.default_rng(0).choice(n, size=64, replace=False)
    idem = float(np.abs(D[rows] @ D - D[rows]).max())
    comm = float(np.abs(H[rows] @ D - D[rows] @ H).max()) / float(np.abs(H).max())
    assert idem <= 1e-9, idem
    assert comm <= 1e-4, comm
    # the spectrum of the sampled principal block stays inside [0, 1]
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
        gate = 0.2 * 2.0 ** -22 / relgap + 1e-6   # as in test_gpu_batched.py
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
