"""Fixed-chemical-potential SP2 in the batched kernel and the graph-based
divide-and-conquer density matrix (§VIII.B) on the GPU, against the CPU
oracle (oracle/graph.py)."""

import numpy as np
import pytest

import oracle
from oracle import graph as OG
from workloads import batch_instance, chain_hamiltonian, cube_hamiltonian

pytestmark = pytest.mark.gpu
U = 2.0 ** -22  # unit round-off class of the split products


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


def test_batched_fixed_mu_matches_oracle(pkg):
    import torch
    mats, mus, refs, gates = [], [], [], []
    for i, sites in enumerate((16, 33, 60, 97)):
        H, nocc = batch_instance(900 + i, sites)
        w = np.linalg.eigvalsh(H)
        k = nocc - 3 * i  # fillings below half as well
        mu = 0.5 * (w[k - 1] + w[k])
        emin, emax = oracle.gershgorin_bounds(H)
        mats.append(H)
        mus.append(mu)
        refs.append(OG.sp2_fixed_mu(H, mu, 1e-10)["D"])
        gates.append(0.2 * U * (emax - emin) / (w[k] - w[k - 1]) + 1e-6)
    # mu outside the spectrum on one more instance: D = 0
    H0, _ = batch_instance(950, 20)
    mats.append(H0)
    mus.append(-1e3)
    refs.append(np.zeros_like(H0))
    gates.append(1e-6)
    packed, n, offsets = pkg.pack_batch(mats)
    D, iters, status = pkg.sp2_batched(dev(packed), n, offsets, np.zeros(len(n)), 1e-10,
                                       mu=mus)
    torch.cuda.synchronize()
    Dh = D.cpu().numpy()
    assert (status.cpu().numpy() == 0).all()
    for Hm, o, r, g in zip(mats, offsets, refs, gates):
        k = Hm.shape[0]
        assert float(np.abs(Dh[o:o + k * k].reshape(k, k) - r).max()) <= g


def test_graph_complete_graph_is_the_projector(pkg):
    H, nocc = cube_hamiltonian(64, 7)  # n = 256
    w = np.linalg.eigvalsh(H)
    mu = 0.5 * (w[nocc - 1] + w[nocc])
    D, info = pkg.sp2_graph(dev(H), dev(H), 0.0, 4, mu, 1e-10)
    assert info["nparts"] == 4 and info["max_part"] == 256 and info["failed_parts"] == 0
    ref = OG.sp2_fixed_mu(H, mu, 1e-10)["D"]
    emin, emax = oracle.gershgorin_bounds(H)
    gate = 0.2 * U * (emax - emin) / (w[nocc] - w[nocc - 1]) + 1e-6
    Dn = D.cpu().numpy()
    assert np.array_equal(Dn, Dn.T)
    assert float(np.abs(Dn - ref).max()) <= gate


@pytest.mark.parametrize("tau", [1e-3, 1e-5])
def test_graph_chain_matches_oracle(pkg, tau):
    # gapped chain, auxiliary matrix = a previously computed density matrix
    H, nocc = chain_hamiltonian(1024)
    w, V = np.linalg.eigh(H)
    Dprev = V[:, :nocc] @ V[:, :nocc].T
    D, info = pkg.sp2_graph(dev(H), dev(Dprev), tau, 8, 0.0, 1e-10)
    P, parts = OG.graph_density(H, Dprev, tau, 8, 0.0, 1e-10)
    assert info["max_part"] == max(len(ch) for _, ch in parts)
    assert abs(info["mean_part"] - np.mean([len(ch) for _, ch in parts])) < 1e-9
    Dn = D.cpu().numpy()
    # the same graph approximation; the GPU adds split round-off (relative gap 0.25)
    assert float(np.abs(Dn - P).max()) <= 1e-5
    # and the approximation error itself shrinks with tau
    err = float(np.abs(Dn - Dprev).max())
    assert err <= (2e-2 if tau == 1e-3 else 2e-4), err
