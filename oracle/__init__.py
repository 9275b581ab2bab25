"""CPU oracle for the SP2 density-matrix solver -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct FP64 implementations of what the GPU path
computes, written from the paper (arXiv 2401.13772):

* ``eig.jacobi_eigh`` -- cyclic Jacobi eigendecomposition in plain C (§III,
  step 1 of the density-matrix procedure).
* ``sp2.density_projector`` -- D = V f V^T with the zero-temperature
  occupations (§III, Eq. 2, in the insulating limit the paragraph after it
  describes): the exact answer SP2 converges to.
* ``sp2.gershgorin_bounds``, ``sp2.x0_map``, ``sp2.sp2_plain`` -- the SP2
  recursion of §IV.A step by step (bounds, the shifted/rescaled D_0, the
  X^2 / 2X - X^2 branches chosen by the trace, idempotency convergence), with
  numpy's matmul as the only library primitive.
* ``sp2.spectral_sp2`` -- the same recursion applied to the eigenvalues
  alone (every iterate is a polynomial in H, so traces, branch choices and the
  iteration count are fixed by the spectrum).
* ``mlp`` -- forward/backward of the small MLP used by the learned-sequence
  path, written as plain numpy algebra, for gradient checks.
* ``graph`` -- the graph-based divide-and-conquer density matrix of §VIII.B
  (threshold graph, core and core-halo partitions, submatrices, SP2 at a
  fixed chemical potential, core columns mapped back).
* ``sparse`` -- thresholded SP2 (Listing 1's cutoff tau: each product and each
  2X - X^2 update drops the elements below tau).
* ``cheb`` -- the Chebyshev Fermi-operator expansion of §IV.B at a known
  chemical potential and temperature: coefficients, the serial recursion, and
  the Paterson-Stockmeyer nested form with its T_k-division coefficients.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package. It shares no code with the CUDA path and the
CUDA path never imports it.
"""

from .sp2 import (  # noqa: F401
    gershgorin_bounds,
    x0_map,
    branch_bit,
    sp2_plain,
    spectral_sp2,
    density_projector,
    invariants,
    NEARER,
    PAPER,
)
from .eig import jacobi_eigh, build_oracle  # noqa: F401
from .graph import (  # noqa: F401
    threshold_graph,
    core_partition,
    core_halo,
    sp2_fixed_mu,
    graph_density,
)
from .cheb import (  # noqa: F401
    fermi,
    scaled_hamiltonian,
    cheb_coefficients,
    ps_coefficients,
    chebyshev_polynomials,
    serial_chebyshev,
    ps_evaluate,
    fermi_operator,
)
from .sparse import prune, sp2_thresholded  # noqa: F401
