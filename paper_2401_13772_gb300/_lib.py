"""ctypes declarations of the C ABI in include/progress_sp2.h.

Argument marshalling only: every step of the solver runs in the CUDA library.
Loading fails loudly when the library has not been built.
"""

from __future__ import annotations

import ctypes
import os
import threading

from .build import LIB_PATH

OK, EINVAL, ENOCONV, EBOUNDS, ECUDA, ENOMEM, ETIMEOUT, EUNSUPPORTED = range(8)
STATUS_NAMES = {OK: "OK", EINVAL: "EINVAL", ENOCONV: "ENOCONV", EBOUNDS: "EBOUNDS",
                ECUDA: "ECUDA", ENOMEM: "ENOMEM", ETIMEOUT: "ETIMEOUT",
                EUNSUPPORTED: "EUNSUPPORTED"}

FP64, FP32_SPLIT, MIXED_FP16, MIXED_BF16, FP32_SPLIT_BF16, DF64 = range(6)
RULE_NEARER, RULE_PAPER, RULE_MU = 0, 1, 2


class Opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int32), ("rule", ctypes.c_int32),
                ("fp64_prefix", ctypes.c_int32), ("maxiter", ctypes.c_int32),
                ("emin", ctypes.c_double), ("emax", ctypes.c_double),
                ("loop_mode", ctypes.c_int32), ("slice_fixed", ctypes.c_int32),
                ("loop_events", ctypes.c_void_p * 2), ("fp64_impl", ctypes.c_int32),
                ("tau", ctypes.c_float), ("wait_limit_us", ctypes.c_int32),
                ("stall_test", ctypes.c_int32), ("split_tile", ctypes.c_int32),
                ("prefix_full", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("phase_iters", ctypes.c_int32 * 3),
                ("emin", ctypes.c_double), ("emax", ctypes.c_double),
                ("trace", ctypes.c_double), ("idempotency", ctypes.c_double),
                ("bits", ctypes.c_uint64 * 4), ("kblocks", ctypes.c_uint64)]

    def to_dict(self):
        bits = [(self.bits[k // 64] >> (k % 64)) & 1 for k in range(self.iters)]
        return {"status": STATUS_NAMES.get(self.status, str(self.status)),
                "iters": self.iters, "converged": bool(self.converged),
                "floor_stop": self.converged == 2,
                "phase_iters": list(self.phase_iters), "emin": self.emin,
                "emax": self.emax, "trace": self.trace,
                "idempotency": self.idempotency, "bits": bits, "kblocks": self.kblocks}


class BatchEx(ctypes.Structure):
    _fields_ = [("d_bounds", ctypes.c_void_p), ("d_pred_bits", ctypes.c_void_p),
                ("d_pred_len", ctypes.c_void_p), ("judge_delta", ctypes.c_double),
                ("d_bits_out", ctypes.c_void_p), ("d_bounds_out", ctypes.c_void_p),
                ("d_fallback", ctypes.c_void_p), ("d_products", ctypes.c_void_p),
                ("tile_n", ctypes.c_int32), ("cluster", ctypes.c_int32),
                ("share", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("d_cycles", ctypes.c_void_p), ("d_mu", ctypes.c_void_p)]


class GraphInfo(ctypes.Structure):
    _fields_ = [("nparts", ctypes.c_int32), ("max_part", ctypes.c_int32),
                ("mean_part", ctypes.c_double), ("max_iters", ctypes.c_int32),
                ("failed_parts", ctypes.c_int32), ("sub_elements", ctypes.c_int64)]

    def to_dict(self):
        return {"nparts": self.nparts, "max_part": self.max_part, "mean_part": self.mean_part,
                "max_iters": self.max_iters, "failed_parts": self.failed_parts,
                "sub_elements": self.sub_elements}


class ChebInfo(ctypes.Structure):
    _fields_ = [("emin", ctypes.c_double), ("emax", ctypes.c_double),
                ("trace", ctypes.c_double), ("growth", ctypes.c_double),
                ("coef_last", ctypes.c_double), ("products", ctypes.c_int32),
                ("launches", ctypes.c_int32)]

    def to_dict(self):
        return {"emin": self.emin, "emax": self.emax, "trace": self.trace,
                "growth": self.growth, "coef_last": self.coef_last,
                "products": self.products, "launches": self.launches}


class BatchTune(ctypes.Structure):
    _fields_ = [("tile_n", ctypes.c_int32), ("cluster", ctypes.c_int32),
                ("share", ctypes.c_int32), ("ncand", ctypes.c_int32),
                ("cand", (ctypes.c_int32 * 3) * 16), ("ms", ctypes.c_float * 16)]

    def to_dict(self):
        return {"tile_n": self.tile_n, "cluster": self.cluster, "share": self.share,
                "candidates": [{"tile_n": self.cand[i][0], "cluster": self.cand[i][1],
                                "share": self.cand[i][2], "ms": float(self.ms[i])}
                               for i in range(self.ncand)]}


# symbol -> (restype, argtypes); every function declared in include/progress_sp2.h
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double
SIGNATURES = {
    "progress_opts_default": (None, [ctypes.POINTER(Opts)]),
    "progress_gershgorin_bounds": (ctypes.c_int, [_P, _I64, _P, _P, _P]),
    "progress_sp2_dense": (ctypes.c_int, [_P, _I64, _I64, _D, _P, _P]),
    "progress_sp2_dense_ex": (ctypes.c_int, [_P, _I64, _I64, _D, _P, ctypes.POINTER(Opts),
                                             ctypes.POINTER(Info), _P]),
    "progress_sp2_dense_noalloc": (ctypes.c_int, [_P, _I64, _I64, _D, _P, _P]),
    "progress_sp2_batched": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P, _P, _D, _P, _P, _P,
                                            ctypes.POINTER(Opts), _P]),
    "progress_sp2_batched_ex": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P, _P, _D, _P, _P, _P,
                                               ctypes.POINTER(Opts), ctypes.POINTER(BatchEx), _P]),
    "progress_sp2_batched_tune": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P, _P, _D, _P,
                                                 ctypes.POINTER(Opts), ctypes.c_int32,
                                                 ctypes.c_int32, ctypes.POINTER(BatchTune), _P]),
    "progress_sp2_graph": (ctypes.c_int, [_P, _P, _I64, _D, ctypes.c_int32, _D, _D, _P,
                                          ctypes.POINTER(Opts), ctypes.POINTER(GraphInfo), _P]),
    "progress_cheb_fermi": (ctypes.c_int, [_P, _I64, _D, _D, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int32, _P, _P, ctypes.POINTER(ChebInfo),
                                           _P]),
    "progress_cheb_slot": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _P, _P]),
    "progress_cheb_choose": (ctypes.c_int, [ctypes.c_int32, _D, _D, _D, _D, _D, _P, _P, _P,
                                            _P]),
    "progress_cheb_plan": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _D, _D, _D, _D,
                                          ctypes.c_int32, _P, _P, _P, _P, _P, _P]),
    "progress_features": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P, _P, _P]),
    "progress_learned_inputs": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _P, _P, _D,
                                               ctypes.c_float, _P, _P, _P, _P]),
    "progress_learned_targets": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _P,
                                                ctypes.c_int32, _P, _P, _P, _P, _P, _P]),
    "progress_learned_labels": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P, _P, _P, _D, _P, _P,
                                               _P, _P]),
    "progress_learned_margin": (ctypes.c_int, [ctypes.c_int32, _P, ctypes.c_int32, _P,
                                               ctypes.c_int32, _D, _D, _P]),
    "progress_trace_hd": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P, _P, _P, _P]),
    "progress_mlp_param_count": (ctypes.c_int32, [ctypes.c_int32] * 3),
    "progress_mlp_scratch_floats": (ctypes.c_int64, [ctypes.c_int32] * 4),
    "progress_mlp_to_fp16": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
    "progress_mlp_forward": (ctypes.c_int, [ctypes.c_int32] * 3 + [_P, ctypes.c_int32, _P, _P,
                                                                   _P, _P]),
    "progress_mlp_train_step": (ctypes.c_int, [ctypes.c_int32] * 3 + [_P, _P, _P, _P,
                                                                      ctypes.c_int32,
                                                                      ctypes.c_float,
                                                                      ctypes.c_int32, _P, _P, _P,
                                                                      _P, _P, _P]),
    "progress_sp2_query": (ctypes.c_int, [_P, ctypes.POINTER(Info)]),
    "progress_sp2_history": (ctypes.c_int32, [_P, _P, _P, ctypes.c_int32]),
    "progress_release": (ctypes.c_int, [_P]),
    "progress_release_all": (ctypes.c_int, []),
    "progress_last_error": (ctypes.c_char_p, []),
    "progress_version": (ctypes.c_char_p, []),
}

_lock = threading.Lock()
_lib = None


class ProgressError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def lib_path() -> str:
    return os.environ.get("PROGRESS_SP2_LIB", LIB_PATH)


def load():
    """Load the CUDA library (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing: run "
                               "paper_2401_13772_gb300.build.build() (needs nvcc)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def check(status: int):
    if status != OK:
        msg = load().progress_last_error().decode(errors="replace")
        raise ProgressError(status, msg)
