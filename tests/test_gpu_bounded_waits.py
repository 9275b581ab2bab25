"""The bounded device-side waits of the tensor-core product kernels.

Every mbarrier wait of the split and digit-product kernels gives up after a
time limit, records PROGRESS_ETIMEOUT, lets the copies already in flight land,
frees its tensor memory and returns, so the context stays usable. Here the
option `stall_test` makes the first CTA of the first tensor-core product wait
on a barrier that nothing arrives on, with the limit lowered to 2 ms through
`wait_limit_us`: the solve must end with ETIMEOUT, and the next solves on the
same stream (which allocate tensor memory again on every SM) must run and
match the oracle.
"""

import numpy as np
import pytest

import oracle
from workloads import cube_hamiltonian

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


@pytest.mark.parametrize("loop_mode", [0, 1])
@pytest.mark.parametrize("prec,gate,split_tile", [("fp32_split", 1e-4, 2), ("fp32_split", 1e-4, 1),
                                                  ("mixed_fp16", 1e-5, 0)])
def test_wait_that_runs_out_reports_etimeout_then_solves_again(pkg, prec, gate, split_tile,
                                                               loop_mode):
    """FP32_SPLIT stalls in the split product (128 x 256 tiles for split_tile 2,
    128 x 128 for 1, the default); MIXED_FP16 in the first digit product of its
    prefix."""
    import torch
    H, nocc = cube_hamiltonian(64, 7)  # n = 256: 3 (128 x 128) or 2 (128 x 256) tiles
    Hd = torch.from_numpy(H).to("cuda:0")
    w, V = oracle.jacobi_eigh(H)
    Dref, _ = oracle.density_projector(w, V, nocc)
    opts = dict(prec=prec, fp64_prefix=8, loop_mode=loop_mode, split_tile=split_tile)
    D, info = pkg.sp2_dense_ex(Hd, nocc, 1e-10, wait_limit_us=2000, stall_test=1,
                               raise_on_status=False, **opts)
    assert info["status"] == "ETIMEOUT", info
    assert not info["converged"]
    # the context is usable and tensor memory was given back: two normal
    # solves on the same stream
    for _ in range(2):
        D, info = pkg.sp2_dense_ex(Hd, nocc, 1e-10, **opts)
        assert info["status"] == "OK" and info["converged"], info
        err = float(np.abs(D.cpu().numpy() - Dref).max())
        assert err <= gate, err


def test_stall_test_needs_tensor_core_products(pkg):
    import torch
    H, nocc = cube_hamiltonian(32, 7)
    Hd = torch.from_numpy(H).to("cuda:0")
    with pytest.raises(pkg.ProgressError):
        pkg.sp2_dense_ex(Hd, nocc, 1e-10, prec="fp64", stall_test=1)
    with pytest.raises(pkg.ProgressError):
        pkg.sp2_dense_ex(Hd, nocc, 1e-10, prec="fp32_split", wait_limit_us=-1)
