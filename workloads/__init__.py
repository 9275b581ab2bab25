"""Seeded synthetic Hamiltonian generators shared by the CUDA path's tests,
the benchmark and the CPU oracle's tests.

This module holds no arithmetic of the SP2 method (no bounds, no spectral map,
no purification): it only builds symmetric matrices H and the occupation
number, with the shapes and structure of the workloads the paper measures
(tight-binding Hamiltonians, §II and §VI; thousands of dense parts of a
graph-partitioned system, §VIII.B).
"""

from .hamiltonians import (  # noqa: F401
    chain_hamiltonian,
    cube_hamiltonian,
    cube_geometry,
    batch_sizes,
    batch_instance,
    batch_packed,
    CUBE_DENSITY,
    CUBE_CUTOFF,
)
