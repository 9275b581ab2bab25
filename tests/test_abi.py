"""The C-ABI library builds, loads and exports every symbol the headers declare
(no GPU needed: no compute call is made)."""

import ctypes
import glob
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2401_13772_gb300.build import build
    build()
    import paper_2401_13772_gb300 as pkg
    return pkg.load()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(progress_\w+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_headers_declare_the_boundary():
    names = declared_functions()
    for required in ("progress_gershgorin_bounds", "progress_sp2_dense", "progress_sp2_dense_ex"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2401_13772_gb300 import _lib
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"{name} has no ctypes signature"


def test_struct_sizes_match_header_layout():
    from paper_2401_13772_gb300 import _lib
    # progress_opts_t: 4 int32, 2 double, 2 int32, 2 pointers, then fp64_impl, tau,
    # wait_limit_us, stall_test, split_tile, prefix_full (4 bytes each)
    assert ctypes.sizeof(_lib.Opts) == 4 * 4 + 2 * 8 + 2 * 4 + 2 * 8 + 6 * 4
    assert _lib.Opts.emin.offset == 16 and _lib.Opts.loop_mode.offset == 32
    assert _lib.Opts.loop_events.offset == 40
    assert _lib.Opts.fp64_impl.offset == 56 and _lib.Opts.tau.offset == 60
    assert _lib.Opts.split_tile.offset == 72
    # progress_info_t: 6 int32, 4 double, 4 uint64, uint64 kblocks
    assert ctypes.sizeof(_lib.Info) == 6 * 4 + 4 * 8 + 4 * 8 + 8
    assert _lib.Info.emin.offset == 24 and _lib.Info.bits.offset == 56
    assert _lib.Info.kblocks.offset == 88
    # progress_batch_ex_t: 8 pointer/double slots, 4 int32 (configuration), 2 pointers
    assert ctypes.sizeof(_lib.BatchEx) == 8 * 8 + 4 * 4 + 2 * 8
    assert _lib.BatchEx.tile_n.offset == 64 and _lib.BatchEx.d_cycles.offset == 80
    assert _lib.BatchEx.d_mu.offset == 88
    # progress_graph_info_t
    assert ctypes.sizeof(_lib.GraphInfo) == 2 * 4 + 8 + 2 * 4 + 8
    # progress_batch_tune_t: 4 int32, int32 cand[16][3], float ms[16]
    assert ctypes.sizeof(_lib.BatchTune) == 4 * 4 + 16 * 3 * 4 + 16 * 4
    assert _lib.BatchTune.ms.offset == 16 + 16 * 3 * 4
    # progress_cheb_info_t: 5 double, 2 int32
    assert ctypes.sizeof(_lib.ChebInfo) == 5 * 8 + 2 * 4
    assert _lib.ChebInfo.products.offset == 40


def test_cheb_argument_errors(lib):
    from paper_2401_13772_gb300 import _lib
    P = ctypes.c_void_p
    ci = _lib.ChebInfo()
    args = dict(n=64, mu=0.0, beta=1.0, k=8, m=8, prec=_lib.FP32_SPLIT)

    def call(dH=P(16), dD=P(32), **kw):
        a = dict(args, **kw)
        return lib.progress_cheb_fermi(dH, a["n"], a["mu"], a["beta"], a["k"], a["m"],
                                       a["prec"], None, dD, ctypes.byref(ci), None)
    assert call(n=0) == _lib.EINVAL
    assert call(k=0) == _lib.EINVAL and call(m=65) == _lib.EINVAL
    assert b"k and m" in lib.progress_last_error()
    assert call(beta=-1.0) == _lib.EINVAL
    assert call(mu=float("nan")) == _lib.EINVAL
    assert call(prec=_lib.MIXED_FP16) == _lib.EINVAL
    assert b"prec" in lib.progress_last_error()
    assert call(dD=P(16)) == _lib.EINVAL
    assert call(dH=None) == _lib.EINVAL


def test_batched_argument_errors(lib):
    from paper_2401_13772_gb300 import _lib
    P = ctypes.c_void_p
    n = (ctypes.c_int32 * 2)(64, 5000)
    off = (ctypes.c_int64 * 2)(0, 4096)
    nocc = (ctypes.c_int32 * 2)(32, 10)
    assert lib.progress_sp2_batched(2, n, off, nocc, P(16), 1e-9, P(32), None, None, None,
                                    None) == _lib.EINVAL
    assert b"n_i" in lib.progress_last_error()
    tune = _lib.BatchTune()
    assert lib.progress_sp2_batched_tune(2, n, off, nocc, P(16), 1e-9, P(32), None, 0, 3,
                                         ctypes.byref(tune), None) == _lib.EINVAL
    assert lib.progress_sp2_batched_tune(2, n, off, nocc, P(16), 1e-9, P(32), None, 1, 3,
                                         ctypes.byref(tune), None) == _lib.EINVAL
    # the fixed-mu rule needs the per-instance chemical potentials
    o = _lib.Opts()
    lib.progress_opts_default(ctypes.byref(o))
    o.prec, o.rule = _lib.FP32_SPLIT, _lib.RULE_MU
    n[1] = 64
    assert lib.progress_sp2_batched(2, n, off, nocc, P(16), 1e-9, P(32), None, None,
                                    ctypes.byref(o), None) == _lib.EINVAL
    assert b"d_mu" in lib.progress_last_error()
    # graph solver argument checks
    gi = _lib.GraphInfo()
    assert lib.progress_sp2_graph(P(16), P(16), 100, 1e-3, 0, 0.0, 1e-9, P(32), None,
                                  ctypes.byref(gi), None) == _lib.EINVAL
    assert lib.progress_sp2_graph(P(16), P(16), 100, -1.0, 4, 0.0, 1e-9, P(32), None,
                                  ctypes.byref(gi), None) == _lib.EINVAL
    assert lib.progress_sp2_graph(P(16), P(16), 100, 1e-3, 4, 0.0, 1e-9, P(16), None,
                                  ctypes.byref(gi), None) == _lib.EINVAL


def test_defaults_and_version(lib):
    from paper_2401_13772_gb300 import _lib
    o = _lib.Opts()
    lib.progress_opts_default(ctypes.byref(o))
    assert o.prec == _lib.FP64 and o.rule == _lib.RULE_NEARER
    assert o.maxiter == 100 and o.fp64_prefix == 12
    assert math.isnan(o.emin) and math.isnan(o.emax)
    assert lib.progress_version() == b"0.1.0"


def test_argument_errors_before_any_device_work(lib):
    from paper_2401_13772_gb300 import _lib
    P = ctypes.c_void_p
    # nocc out of range, negative n, negative tol: rejected before touching CUDA
    assert lib.progress_sp2_dense(P(16), 8, 9, 1e-9, P(32), None) == _lib.EINVAL
    assert lib.progress_sp2_dense(P(16), -1, 0, 1e-9, P(32), None) == _lib.EINVAL
    assert lib.progress_sp2_dense(P(16), 8, 4, -1.0, P(32), None) == _lib.EINVAL
    assert lib.progress_sp2_dense(P(16), 8, 4, 1e-9, P(16), None) == _lib.EINVAL  # D aliases H
    lib.progress_sp2_dense(P(16), 8, 9, 1e-9, P(32), None)
    assert b"nocc" in lib.progress_last_error()
    o = _lib.Opts()
    lib.progress_opts_default(ctypes.byref(o))
    o.maxiter = 1000
    assert lib.progress_sp2_dense_ex(P(16), 8, 4, 1e-9, P(32), ctypes.byref(o), None, None) == _lib.EINVAL
    o.maxiter = 10
    o.emin, o.emax = 1.0, 0.0
    assert lib.progress_sp2_dense_ex(P(16), 8, 4, 1e-9, P(32), ctypes.byref(o), None, None) == _lib.EINVAL
    # thresholded SP2: tau >= 0, and tau > 0 only with the split precisions
    o.emin, o.emax = float("nan"), float("nan")
    o.tau = -1.0
    assert lib.progress_sp2_dense_ex(P(16), 8, 4, 1e-9, P(32), ctypes.byref(o), None, None) == _lib.EINVAL
    o.tau = 1e-6
    o.prec = _lib.FP64
    assert lib.progress_sp2_dense_ex(P(16), 8, 4, 1e-9, P(32), ctypes.byref(o), None, None) == _lib.EINVAL
    assert b"tau" in lib.progress_last_error()
    o.prec, o.slice_fixed = _lib.FP32_SPLIT, 1
    assert lib.progress_sp2_dense_ex(P(16), 8, 4, 1e-9, P(32), ctypes.byref(o), None, None) == _lib.EINVAL
    assert lib.progress_gershgorin_bounds(P(16), 0, P(32), P(40), None) == _lib.EINVAL
    assert lib.progress_gershgorin_bounds(P(16), 4, P(32), None, None) == _lib.EINVAL
    assert b"n < 1" in lib.progress_last_error()
    # n = 0 is a no-op
    info = _lib.Info()
    assert lib.progress_sp2_dense_ex(None, 0, 0, 1e-9, None, None, ctypes.byref(info), None) == _lib.OK
    assert info.converged == 1


def test_product_path_has_no_cpu_fallback():
    """The package never imports the oracle and fails loudly without the library."""
    pkg_dir = os.path.join(ROOT, "paper_2401_13772_gb300")
    for f in glob.glob(os.path.join(pkg_dir, "*.py")):
        src = open(f).read()
        assert "import oracle" not in src and "from oracle" not in src, f
    from paper_2401_13772_gb300 import _lib
    old = os.environ.get("PROGRESS_SP2_LIB")
    saved = _lib._lib
    try:
        os.environ["PROGRESS_SP2_LIB"] = "/nonexistent/libprogress_sp2.so"
        _lib._lib = None
        with pytest.raises(RuntimeError, match="missing"):
            _lib.load()
    finally:
        _lib._lib = saved
        if old is None:
            os.environ.pop("PROGRESS_SP2_LIB", None)
        else:
            os.environ["PROGRESS_SP2_LIB"] = old
