"""The allocation-free FP64 entry point, through the C ABI, against the
regular one. It serves callers that cannot allocate device memory (a device
already owned by the application's own memory pool, a time-stepping loop that
must not pay allocation latency): its work space is a fixed device array
inside the library, so two calls in a row must not leak state from one into
the other."""

import ctypes

import numpy as np
import pytest

from workloads import chain_hamiltonian, cube_hamiltonian

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10  # the FP64 path's parity tolerance


def test_noalloc_matches_regular_entry_point_twice():
    import torch
    assert torch.cuda.is_available(), "GPU test run without a CUDA device"
    from paper_2401_13772_gb300.build import build
    build()
    import paper_2401_13772_gb300 as pkg
    from paper_2401_13772_gb300 import _lib
    lib = pkg.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [cube_hamiltonian(75, 12), chain_hamiltonian(256)]  # n = 300, then n = 256
    for H, nocc in cases:
        Hd = torch.from_numpy(H).to("cuda:0")
        D_ref = torch.empty_like(Hd)
        D_new = torch.full_like(Hd, float("nan"))
        assert lib.progress_sp2_dense(ctypes.c_void_p(Hd.data_ptr()), H.shape[0], nocc, 1e-12,
                                      ctypes.c_void_p(D_ref.data_ptr()), stream) == _lib.OK
        assert lib.progress_sp2_dense_noalloc(ctypes.c_void_p(Hd.data_ptr()), H.shape[0], nocc,
                                              1e-12, ctypes.c_void_p(D_new.data_ptr()),
                                              stream) == _lib.OK
        torch.cuda.synchronize()
        a, b = D_ref.cpu().numpy(), D_new.cpu().numpy()
        assert np.isfinite(b).all()
        assert np.abs(a - b).max() <= TOL_FP64
    # sizes beyond the fixed work space are rejected with a clear error
    big = torch.zeros((2048, 2048), dtype=torch.float64, device="cuda:0")
    out = torch.empty_like(big)
    assert lib.progress_sp2_dense_noalloc(ctypes.c_void_p(big.data_ptr()), 2048, 1024, 1e-12,
                                          ctypes.c_void_p(out.data_ptr()), stream) == _lib.EINVAL
    assert b"1024" in lib.progress_last_error()
