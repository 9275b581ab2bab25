"""GB300 (sm_103a) SP2 density-matrix solver: Python binding of the C ABI.

The solver computes the zero-temperature density matrix D of a real symmetric
Hamiltonian H with the SP2 recursive purification of arXiv 2401.13772 §IV.A:
Gershgorin bounds (§VIII.A), X0 = (emax I - H)/(emax - emin), then
X <- X^2 or 2X - X^2 chosen by the trace until X is idempotent.

Every function here only marshals torch CUDA tensors (device memory and the
current stream) into the C ABI declared in include/progress_sp2.h; all
arithmetic runs in the library's CUDA kernels. There is no CPU fallback: the
calls raise when the library is missing or the tensors are not on a GPU.
"""

from __future__ import annotations

import ctypes
import math

from . import _lib
from ._lib import (  # noqa: F401
    FP64, FP32_SPLIT, MIXED_FP16, MIXED_BF16, FP32_SPLIT_BF16, DF64, RULE_NEARER, RULE_PAPER,
    RULE_MU,
    Info, Opts, ProgressError, load, check,
)

__all__ = ["gershgorin_bounds", "sp2_dense", "sp2_dense_ex", "release", "load",
           "FP64", "FP32_SPLIT", "MIXED_FP16", "MIXED_BF16", "RULE_NEARER", "RULE_PAPER",
           "PREC_NAMES", "ProgressError"]

PREC_NAMES = {"fp64": FP64, "fp32_split": FP32_SPLIT, "mixed_fp16": MIXED_FP16,
              "mixed_bf16": MIXED_BF16, "fp32_split_bf16": FP32_SPLIT_BF16, "df64": DF64}
RULE_NAMES = {"nearer": RULE_NEARER, "paper": RULE_PAPER, "mu": RULE_MU}


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check_matrix(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64:
        raise TypeError(f"{name} must be float64")
    if t.dim() != 2 or t.shape[0] != t.shape[1]:
        raise ValueError(f"{name} must be square")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous (row-major)")


def gershgorin_bounds(H, out=None, stream=None):
    """Device tensor [emin, emax] of Gershgorin bounds of H (§VIII.A)."""
    import torch
    _check_matrix(H, "H")
    if out is None:
        out = torch.empty(2, dtype=torch.float64, device=H.device)
    with torch.cuda.device(H.device):
        check(load().progress_gershgorin_bounds(ctypes.c_void_p(H.data_ptr()), H.shape[0],
                                                ctypes.c_void_p(out.data_ptr()),
                                                ctypes.c_void_p(out.data_ptr() + 8),
                                                _stream_ptr(stream)))
    return out


def make_opts(prec="fp64", rule="nearer", fp64_prefix=12, maxiter=100, emin=None, emax=None,
              loop_mode=0, loop_events=None, slice_fixed=0, fp64_impl=0, tau=0.0,
              wait_limit_us=0, stall_test=0, split_tile=0, prefix_full=0):
    o = Opts()
    load().progress_opts_default(ctypes.byref(o))
    o.prec = PREC_NAMES[prec] if isinstance(prec, str) else int(prec)
    o.rule = RULE_NAMES[rule] if isinstance(rule, str) else int(rule)
    o.fp64_prefix = int(fp64_prefix)
    o.maxiter = int(maxiter)
    o.emin = math.nan if emin is None else float(emin)
    o.emax = math.nan if emax is None else float(emax)
    o.loop_mode = int(loop_mode)
    o.slice_fixed = int(slice_fixed)
    o.fp64_impl = int(fp64_impl)
    o.tau = float(tau)
    o.wait_limit_us = int(wait_limit_us)
    o.stall_test = int(stall_test)
    o.split_tile = int(split_tile)
    o.prefix_full = int(prefix_full)
    if loop_events is not None:
        # torch.cuda.Event pair, already created (recorded once)
        o.loop_events[0] = loop_events[0].cuda_event
        o.loop_events[1] = loop_events[1].cuda_event
    return o


def sp2_dense(H, nocc, tol, D=None, stream=None):
    """Asynchronous FP64 SP2 solve with default options; returns D."""
    import torch
    _check_matrix(H, "H")
    if D is None:
        D = torch.empty_like(H)
    _check_matrix(D, "D")
    with torch.cuda.device(H.device):
        check(load().progress_sp2_dense(ctypes.c_void_p(H.data_ptr()), H.shape[0], int(nocc),
                                        float(tol), ctypes.c_void_p(D.data_ptr()),
                                        _stream_ptr(stream)))
    return D


def sp2_dense_ex(H, nocc, tol, D=None, info=True, stream=None, raise_on_status=True, **opts):
    """SP2 solve with options (prec, rule, fp64_prefix, maxiter, emin, emax,
    loop_mode, loop_events, slice_fixed, fp64_impl, tau, wait_limit_us,
    stall_test, split_tile, prefix_full). With info=True it synchronizes and returns (D, info dict)."""
    import torch
    _check_matrix(H, "H")
    if D is None:
        D = torch.empty_like(H)
    _check_matrix(D, "D")
    o = make_opts(**opts)
    inf = _lib.Info() if info else None
    with torch.cuda.device(H.device):
        st = load().progress_sp2_dense_ex(ctypes.c_void_p(H.data_ptr()), H.shape[0], int(nocc),
                                          float(tol), ctypes.c_void_p(D.data_ptr()),
                                          ctypes.byref(o),
                                          ctypes.byref(inf) if info else None,
                                          _stream_ptr(stream))
    if st != _lib.OK and (raise_on_status or
                          st not in (_lib.ENOCONV, _lib.EBOUNDS, _lib.ETIMEOUT)):
        check(st)
    if info:
        return D, inf.to_dict()
    return D


def pack_batch(mats):
    """Pack a list of square numpy matrices into one FP64 vector.
    Returns (packed, n, offsets) with offsets in elements."""
    import numpy as np
    n = np.array([m.shape[0] for m in mats], dtype=np.int32)
    sizes = n.astype(np.int64) ** 2
    offsets = np.zeros(len(mats), dtype=np.int64)
    if len(mats) > 1:
        offsets[1:] = np.cumsum(sizes)[:-1]
    packed = np.empty(int(sizes.sum()), dtype=np.float64)
    for m, o, sz in zip(mats, offsets, sizes):
        packed[o:o + sz] = np.ascontiguousarray(m, dtype=np.float64).ravel()
    return packed, n, offsets


def _batch_arrays(n, offsets, nocc):
    import numpy as np
    return (np.ascontiguousarray(n, dtype=np.int32), np.ascontiguousarray(offsets, dtype=np.int64),
            np.ascontiguousarray(nocc, dtype=np.int32))


def _check_packed(H_packed):
    import torch
    if not (isinstance(H_packed, torch.Tensor) and H_packed.is_cuda and
            H_packed.dtype == torch.float64 and H_packed.dim() == 1 and H_packed.is_contiguous()):
        raise TypeError("H_packed must be a contiguous 1-D float64 CUDA tensor")


def sp2_batched(H_packed, n, offsets, nocc, tol, D_packed=None, rule="nearer", maxiter=100,
                stream=None, prec="fp32_split", config=None, cycles=False, mu=None):
    """Batched split-precision SP2 over packed device inputs.

    H_packed: 1-D float64 CUDA tensor; n, offsets, nocc: host int sequences.
    config: None (the autotuned configuration for this batch signature, else
    the library default) or (tile_n, cluster, share).
    Returns (D_packed, iters, status) with iters/status as int32 CUDA tensors,
    plus a per-instance int64 tensor of SM clock cycles when cycles=True.
    mu: per-instance chemical potentials -> D_i = theta(mu_i I - H_i) (the
    fixed-mu rule; nocc is then ignored).
    """
    import numpy as np
    import torch
    _check_packed(H_packed)
    n, offsets, nocc = _batch_arrays(n, offsets, nocc)
    b = len(n)
    if D_packed is None:
        D_packed = torch.empty_like(H_packed)
    iters = torch.zeros(b, dtype=torch.int32, device=H_packed.device)
    status = torch.zeros(b, dtype=torch.int32, device=H_packed.device)
    mu_d = None
    if mu is not None:
        rule = "mu"
        mu_d = torch.as_tensor(np.asarray(mu, dtype=np.float64), device=H_packed.device)
    o = make_opts(prec=prec, rule=rule, maxiter=maxiter)
    cyc = None
    with torch.cuda.device(H_packed.device):
        args = (b, ctypes.c_void_p(n.ctypes.data), ctypes.c_void_p(offsets.ctypes.data),
                ctypes.c_void_p(nocc.ctypes.data), ctypes.c_void_p(H_packed.data_ptr()),
                float(tol), ctypes.c_void_p(D_packed.data_ptr()),
                ctypes.c_void_p(iters.data_ptr()), ctypes.c_void_p(status.data_ptr()),
                ctypes.byref(o))
        if config is None and not cycles and mu_d is None:
            check(load().progress_sp2_batched(*args, _stream_ptr(stream)))
        else:
            ex = _lib.BatchEx()
            if mu_d is not None:
                ex.d_mu = mu_d.data_ptr()
            if config is not None:
                ex.tile_n, ex.cluster, ex.share = (int(v) for v in config)
            if cycles:
                cyc = torch.zeros(b, dtype=torch.int64, device=H_packed.device)
                ex.d_cycles = cyc.data_ptr()
            check(load().progress_sp2_batched_ex(*args, ctypes.byref(ex), _stream_ptr(stream)))
    if cycles:
        return D_packed, iters, status, cyc
    return D_packed, iters, status


def batched_tune(H_packed, n, offsets, nocc, tol, D_packed=None, rule="nearer", maxiter=100,
                 stream=None, prec="fp32_split", sample_stride=1, reps=3):
    """Run the batched launch-configuration autotuner on this batch (writes D
    for the sampled instances) and return its report: the chosen tile_n,
    cluster, share and each candidate's time per launch. Later sp2_batched
    calls with the same batch signature use the chosen configuration."""
    import torch
    _check_packed(H_packed)
    n, offsets, nocc = _batch_arrays(n, offsets, nocc)
    if D_packed is None:
        D_packed = torch.empty_like(H_packed)
    o = make_opts(prec=prec, rule=rule, maxiter=maxiter)
    out = _lib.BatchTune()
    with torch.cuda.device(H_packed.device):
        check(load().progress_sp2_batched_tune(
            len(n), ctypes.c_void_p(n.ctypes.data), ctypes.c_void_p(offsets.ctypes.data),
            ctypes.c_void_p(nocc.ctypes.data), ctypes.c_void_p(H_packed.data_ptr()), float(tol),
            ctypes.c_void_p(D_packed.data_ptr()), ctypes.byref(o), int(sample_stride), int(reps),
            ctypes.byref(out), _stream_ptr(stream)))
    return out.to_dict()


def sp2_graph(H, G, tau, nparts, mu, tol, D=None, prec="fp32_split", maxiter=100, stream=None):
    """Graph-based divide-and-conquer density matrix theta(mu I - H) (§VIII.B):
    adjacency |G_ij| >= tau of the auxiliary matrix G, nparts regular-segment
    cores extended by their neighbours, the dense parts solved in one batched
    SP2 launch at the chemical potential mu, core columns mapped back.
    H, G: square float64 CUDA tensors. Returns (D, info dict)."""
    import torch
    for M in (H, G):
        if not (isinstance(M, torch.Tensor) and M.is_cuda and M.dtype == torch.float64 and
                M.dim() == 2 and M.shape[0] == M.shape[1] and M.is_contiguous()):
            raise TypeError("H and G must be square contiguous float64 CUDA tensors")
    n = H.shape[0]
    if D is None:
        D = torch.empty_like(H)
    o = make_opts(prec=prec, maxiter=maxiter)
    info = _lib.GraphInfo()
    with torch.cuda.device(H.device):
        check(load().progress_sp2_graph(
            ctypes.c_void_p(H.data_ptr()), ctypes.c_void_p(G.data_ptr()), n, float(tau),
            int(nparts), float(mu), float(tol), ctypes.c_void_p(D.data_ptr()), ctypes.byref(o),
            ctypes.byref(info), _stream_ptr(stream)))
    return D, info.to_dict()


def cheb_fermi(H, mu, beta, k, m, prec="fp32_split", bounds=None, D=None, stream=None):
    """Finite-temperature density matrix f(H), f(e) = 1 / (1 + exp(beta (e - mu))),
    by the Chebyshev expansion of §IV.B in the Paterson-Stockmeyer form with
    L + 1 = k m terms ((k - 1) + (m - 1) matrix products on the tensor cores).
    prec: "fp32_split" (fp16 hi+lo slices) or "fp32_split_bf16" (bf16 hi+mid+lo).
    bounds: (emin, emax) enclosing the spectrum, or None for Gershgorin.
    H: square float64 CUDA tensor. Returns (D, info dict)."""
    import torch
    if not (isinstance(H, torch.Tensor) and H.is_cuda and H.dtype == torch.float64 and
            H.dim() == 2 and H.shape[0] == H.shape[1] and H.is_contiguous()):
        raise TypeError("H must be a square contiguous float64 CUDA tensor")
    codes = {"fp32_split": FP32_SPLIT, "fp32_split_bf16": FP32_SPLIT_BF16}
    if prec not in codes:
        raise ValueError(f"prec must be one of {sorted(codes)}")
    n = H.shape[0]
    if D is None:
        D = torch.empty_like(H)
    hb = None
    if bounds is not None:
        hb = (ctypes.c_double * 2)(float(bounds[0]), float(bounds[1]))
    info = _lib.ChebInfo()
    with torch.cuda.device(H.device):
        check(load().progress_cheb_fermi(
            ctypes.c_void_p(H.data_ptr()), n, float(mu), float(beta), int(k), int(m),
            int(codes[prec]), ctypes.cast(hb, ctypes.c_void_p) if hb is not None else None,
            ctypes.c_void_p(D.data_ptr()), ctypes.byref(info), _stream_ptr(stream)))
    return D, info.to_dict()


def cheb_slot(n, slot, prec="fp32_split", scale=1.0, stream=None):
    """Value (float64 numpy, n x n) of one stack slot of the last cheb_fermi solve
    on the stream, decoded from its slices and multiplied by scale."""
    import numpy as np
    ld = (n + 127) // 128 * 128
    ns = 2 if prec == "fp32_split" else 3
    planes = []
    for j in range(ns):
        buf = np.empty((ld, ld), dtype=np.uint16)
        check(load().progress_cheb_slot(int(slot), j, ctypes.c_void_p(buf.ctypes.data),
                                        _stream_ptr(stream)))
        planes.append(buf)
    if ns == 2:
        v = (planes[0].view(np.float16).astype(np.float64) +
             planes[1].view(np.float16).astype(np.float64) / 2048.0)
    else:
        def bf(u):
            return (u.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
        v = bf(planes[0]) + bf(planes[1]) + bf(planes[2])
    return scale * v[:n, :n]


def cheb_plan(k, m, mu, beta, emin, emax):
    """The product schedule cheb_fermi runs for the bounds (emin, emax), computed by
    the library on the host (no GPU). Returns a dict of numpy arrays: prods [P, 5]
    (a, b, e, c, launch), params [P, 6] (alpha, sab, beta, se, gamma, inv_sc),
    d [k, m], inv_s [m], a, b, product_launches, slots, t_products."""
    import numpy as np
    cap = max(1, (k - 1) + (m - 1))
    prods = np.zeros((cap, 5), dtype=np.int32)
    params = np.zeros((cap, 6), dtype=np.float32)
    d = np.zeros(k * m)
    inv_s = np.zeros(m)
    ab = np.zeros(2)
    counts = np.zeros(4, dtype=np.int32)
    check(load().progress_cheb_plan(int(k), int(m), float(mu), float(beta), float(emin),
                                    float(emax), cap, *(ctypes.c_void_p(x.ctypes.data) for x in
                                                        (prods, params, d, inv_s, ab, counts))))
    np_ = int(counts[0])
    return {"prods": prods[:np_], "params": params[:np_], "d": d.reshape(k, m), "inv_s": inv_s,
            "a": float(ab[0]), "b": float(ab[1]), "product_launches": int(counts[1]),
            "slots": int(counts[2]), "t_products": int(counts[3])}


def cheb_choose_km(terms, mu, beta, emin, emax, max_growth=8.0):
    """Pick (k, m) for cheb_fermi with k m >= terms (progress_cheb_choose, host
    only): the fewest matrix products of the library's own plan among the
    splits whose nested sums stay within max_growth (the plan's growth =
    sum |d_ij|; a large growth amplifies the products' rounding, e.g. k = m =
    32 at beta b = 236 gives 3e5). Ties go to fewer terms. Raises ProgressError
    (EINVAL) if no split qualifies."""
    k, m, p = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
    g = ctypes.c_double(0.0)
    check(load().progress_cheb_choose(int(terms), float(mu), float(beta), float(emin),
                                      float(emax), float(max_growth), ctypes.byref(k),
                                      ctypes.byref(m), ctypes.byref(p), ctypes.byref(g)))
    return {"k": k.value, "m": m.value, "products": p.value, "terms": k.value * m.value,
            "growth": g.value}


def query(stream=None):
    """Synchronize the stream and return the info dict of the last solve queued on it."""
    inf = _lib.Info()
    st = load().progress_sp2_query(_stream_ptr(stream), ctypes.byref(inf))
    if st not in (_lib.OK, _lib.ENOCONV, _lib.EBOUNDS, _lib.ETIMEOUT):
        check(st)
    return inf.to_dict()


def history(stream=None, cap=256):
    """(idem, margin) numpy arrays of the last solve on the stream: idem[k] =
    |Tr X_k^2 - Tr X_k|, margin[k] = signed branch-rule margin of product k."""
    import numpy as np
    idem = np.zeros(cap)
    margin = np.zeros(cap)
    cnt = load().progress_sp2_history(_stream_ptr(stream), ctypes.c_void_p(idem.ctypes.data),
                                      ctypes.c_void_p(margin.ctypes.data), cap)
    if cnt < 0:
        check(_lib.ECUDA)
    return idem[:cnt], margin[:max(cnt - 1, 0)]


def release(stream=None):
    """Free the library's cached workspace of the stream."""
    check(load().progress_release(_stream_ptr(stream)))
