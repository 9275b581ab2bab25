"""Synthetic tight-binding Hamiltonians (real symmetric, dense, FP64, row-major).

Two families stand in for the paper's workloads, whose data files are not
public (the solvated-peptide DFTB benchmark of §II and the "soft matter
synthetic Hamiltonians" of §VI are not available):

* ``chain_hamiltonian`` -- a dimerized periodic 1D chain with alternating
  hoppings t1, t2 and zero onsite energy. Its spectrum is known in closed form,
  which makes it the exact pin for every solver.
* ``cube_hamiltonian`` -- sites uniform-random in a periodic cube at 0.1
  sites/A^3, 4 orbitals per site, onsite +1/-1 alternating by site index, and a
  random exponentially decaying hopping -2.0*exp(-r/1.5 A)*u, u ~ U(0.5, 1),
  between orbitals of distinct sites closer than 6 A (minimum-image distance).
  Orbitals on the same site are not coupled. With a few hundred non-zeros per
  row before fill-in it has the sparsity structure of the paper's
  tight-binding systems (Table I: the density matrix is dense for N ~ 10^3
  and sparse beyond).

Random numbers come from numpy's PCG64 (``numpy.random.default_rng(seed)``).
Draw order (fixed, part of the recipe): the 3*S site coordinates first, then
one U(0.5, 1) number per coupled orbital pair, site pairs in lexicographic
(i < j) order, orbital pairs (a, b) a-major within a site pair.
"""

from __future__ import annotations

import numpy as np

CUBE_DENSITY = 0.1  # sites per cubic Angstrom
CUBE_CUTOFF = 6.0  # Angstrom
CUBE_DECAY = 1.5  # Angstrom
CUBE_HOP = -2.0  # eV
CUBE_ONSITE = 1.0  # eV, +1 on even sites, -1 on odd sites
ORBITALS_PER_SITE = 4


def chain_hamiltonian(n: int = 512, t1: float = -1.0, t2: float = -0.6):
    """Dimerized periodic chain: H[i, i+1 mod n] = t1 for even i, t2 for odd i.

    Returns (H, nocc) with nocc = n // 2 (half filling). ``n`` must be even so
    that the periodic dimerization closes.
    """
    if n < 2 or n % 2:
        raise ValueError("chain length must be even and >= 2")
    H = np.zeros((n, n), dtype=np.float64)
    i = np.arange(n)
    j = (i + 1) % n
    t = np.where(i % 2 == 0, t1, t2)
    H[i, j] = t
    H[j, i] = t
    return H, n // 2


def cube_geometry(sites: int, seed: int, density: float = CUBE_DENSITY):
    """Site positions, box length and the random generator positioned after them."""
    rng = np.random.default_rng(seed)
    L = (sites / density) ** (1.0 / 3.0)
    pos = rng.uniform(0.0, L, size=(sites, 3))
    return pos, L, rng


def cube_hamiltonian(sites: int, seed: int, density: float = CUBE_DENSITY,
                     cutoff: float = CUBE_CUTOFF):
    """Random-cube tight-binding Hamiltonian with n = 4*sites orbitals.

    Returns (H, nocc) with nocc = n // 2.
    """
    if sites < 1:
        raise ValueError("sites must be >= 1")
    pos, L, rng = cube_geometry(sites, seed, density)
    m = ORBITALS_PER_SITE
    n = m * sites
    H = np.zeros((n, n), dtype=np.float64)
    onsite = np.where(np.arange(sites) % 2 == 0, CUBE_ONSITE, -CUBE_ONSITE)
    H[np.arange(n), np.arange(n)] = np.repeat(onsite, m)
    if sites < 2:
        return H, n // 2
    iu, ju = np.triu_indices(sites, 1)
    d = pos[ju] - pos[iu]
    d -= L * np.round(d / L)  # minimum image
    r = np.sqrt(np.einsum("ij,ij->i", d, d))
    keep = r < cutoff
    iu, ju, r = iu[keep], ju[keep], r[keep]
    u = rng.uniform(0.5, 1.0, size=(iu.size, m, m))
    hop = CUBE_HOP * np.exp(-r / CUBE_DECAY)[:, None, None] * u
    a = np.arange(m)
    rows = (m * iu)[:, None, None] + a[None, :, None]
    cols = (m * ju)[:, None, None] + a[None, None, :]
    rows = np.broadcast_to(rows, hop.shape)
    cols = np.broadcast_to(cols, hop.shape)
    H[rows, cols] = hop
    H[cols, rows] = hop
    return H, n // 2


def batch_sizes(count: int = 4000, seed: int = 0, lo_sites: int = 16,
                hi_sites: int = 192):
    """Site counts of the batched workload: U{lo..hi} sites, n = 4*sites."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo_sites, hi_sites + 1, size=count)


def batch_instance(index: int, sites: int, base_seed: int = 1000):
    """Instance ``index`` of a batch: a cube Hamiltonian with seed base+index."""
    return cube_hamiltonian(int(sites), base_seed + int(index))


def _fill_batch(args):
    """Worker: write instances [lo, hi) of a batch into a file-backed buffer."""
    path, total, sites, offsets, lo, hi, base_seed, index = args
    buf = np.memmap(path, dtype=np.float64, mode="r+", shape=(total,))
    for i in range(lo, hi):
        H, _ = cube_hamiltonian(int(sites[i]), base_seed + int(index[i]))
        n = H.shape[0]
        buf[offsets[i]:offsets[i] + n * n] = H.ravel()
    buf.flush()
    del buf
    return hi - lo


def batch_packed(sites, base_seed=1000, workers=None, index=None):
    """All instances of a batch packed row-major into one FP64 vector.

    Instance i is cube_hamiltonian(sites[i], base_seed + index[i]) (index
    defaults to 0, 1, ...: a rank's shard keeps the seeds of the whole
    batch); returns (packed, n, offsets, nocc). Generation runs in `workers`
    processes (spawned, so it is safe before or after CUDA initialisation)
    writing into a temporary file-backed buffer."""
    import multiprocessing as mp
    import os
    import tempfile
    sites = np.asarray(sites, dtype=np.int64)
    index = np.arange(len(sites)) if index is None else np.asarray(index, dtype=np.int64)
    if len(index) != len(sites):
        raise ValueError("index must have one entry per instance")
    n = (ORBITALS_PER_SITE * sites).astype(np.int32)
    sizes = n.astype(np.int64) ** 2
    offsets = np.zeros(len(n), dtype=np.int64)
    if len(n) > 1:
        offsets[1:] = np.cumsum(sizes)[:-1]
    total = int(sizes.sum())
    if workers is None:
        workers = min(16, os.cpu_count() or 1)
    fd, path = tempfile.mkstemp(suffix=".f64")
    os.close(fd)
    try:
        np.memmap(path, dtype=np.float64, mode="w+", shape=(max(total, 1),)).flush()
        chunks = np.linspace(0, len(n), max(1, workers * 4) + 1).astype(int)
        jobs = [(path, total, sites, offsets, int(a), int(b), base_seed, index)
                for a, b in zip(chunks[:-1], chunks[1:]) if b > a]
        if workers > 1 and len(jobs) > 1:
            with mp.get_context("spawn").Pool(workers) as pool:
                pool.map(_fill_batch, jobs)
        else:
            for j in jobs:
                _fill_batch(j)
        packed = np.array(np.memmap(path, dtype=np.float64, mode="r", shape=(total,)))
    finally:
        os.unlink(path)
    return packed, n, offsets, (n // 2).astype(np.int32)
