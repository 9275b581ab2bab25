"""Learned spectral bounds and SP2 branch sequences.

A small perceptron maps cheap features of H (Gershgorin bounds, traces, a
histogram of the diagonal) to (a) tighter spectral bounds for the X0 map of
§IV.A -- the Gershgorin estimate of §VIII.A is loose, and a looser map leaves
a smaller relative gap and costs iterations -- and (b) the branch sequence of
the SP2 loop. Labels come from SP2 runs of the library itself:

* eps_1 = Tr(H D_1) with D_1 the SP2 projector of H for nocc = 1, and eps_N
  = Tr(H D'_1) with D'_1 the projector of -H for nocc = 1 (batched FP32-split
  solves); for a near-degenerate edge this is within the degeneracy;
* the branch bits of an SP2 run whose X0 uses those bounds widened by the
  safety margin the predictions will be widened by.

Training and inference run the library's own kernels (forward, loss,
backward, Adam; FP16 weights at inference). At solve time the trace-driven
rule judges every predicted branch; a disagreement beyond the judge margin,
or a run that leaves [0, 1], sends that instance back to the plain path
(Gershgorin bounds, trace rule). This module only marshals torch tensors.
"""

from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from . import _stream_ptr, check, load, make_opts, pack_batch

N_FEAT = 37
N_BOUNDS = 2


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def to_device_batch(mats, device="cuda:0"):
    """Pack numpy matrices; returns a dict with the packed device tensor and layout."""
    import torch
    packed, n, offsets = pack_batch(mats)
    return {"H": torch.from_numpy(packed).to(device), "n": n, "offsets": offsets,
            "d_n": torch.from_numpy(n).to(device), "d_off": torch.from_numpy(offsets).to(device)}


def features(batch):
    """[B, 37] float32 CUDA tensor of predictor inputs."""
    import torch
    B = len(batch["n"])
    f = torch.empty((B, N_FEAT), dtype=torch.float32, device=batch["H"].device)
    check(load().progress_features(B, _p(batch["d_n"]), _p(batch["d_off"]), _p(batch["H"]),
                                   _p(f), _stream_ptr()))
    return f


def trace_hd(batch, D):
    import torch
    B = len(batch["n"])
    out = torch.empty(B, dtype=torch.float64, device=D.device)
    check(load().progress_trace_hd(B, _p(batch["d_n"]), _p(batch["d_off"]), _p(batch["H"]),
                                   _p(D), _p(out), _stream_ptr()))
    return out


def batched_solve(batch, nocc, tol=1e-10, bounds=None, pred_bits=None, pred_len=None,
                  judge_delta=0.0, maxiter=100, prec="fp32_split_bf16"):
    """Batched split-precision SP2 with optional learned inputs (bf16 slices by
    default: their exponent range keeps runs with nocc << n intact).

    Returns a dict of CUDA tensors: D (packed), iters, status, bits [B,4]
    (uint64 stored as int64), bounds [B,2], fallback."""
    import torch
    dev = batch["H"].device
    B = len(batch["n"])
    nocc = np.ascontiguousarray(nocc, dtype=np.int32)
    D = torch.empty_like(batch["H"])
    iters = torch.zeros(B, dtype=torch.int32, device=dev)
    status = torch.zeros(B, dtype=torch.int32, device=dev)
    bits = torch.zeros((B, 4), dtype=torch.int64, device=dev)
    bnd = torch.zeros((B, 2), dtype=torch.float64, device=dev)
    fb = torch.zeros(B, dtype=torch.int32, device=dev)
    prod = torch.zeros(B, dtype=torch.int32, device=dev)
    ex = _lib.BatchEx()
    ex.d_bounds = bounds.data_ptr() if bounds is not None else None
    ex.d_pred_bits = pred_bits.data_ptr() if pred_bits is not None else None
    ex.d_pred_len = pred_len.data_ptr() if pred_len is not None else None
    ex.judge_delta = float(judge_delta)
    ex.d_bits_out = bits.data_ptr()
    ex.d_bounds_out = bnd.data_ptr()
    ex.d_fallback = fb.data_ptr()
    ex.d_products = prod.data_ptr()
    o = make_opts(prec=prec, maxiter=maxiter)
    n = np.ascontiguousarray(batch["n"], dtype=np.int32)
    off = np.ascontiguousarray(batch["offsets"], dtype=np.int64)
    check(load().progress_sp2_batched_ex(
        B, ctypes.c_void_p(n.ctypes.data), ctypes.c_void_p(off.ctypes.data),
        ctypes.c_void_p(nocc.ctypes.data), _p(batch["H"]), float(tol), _p(D), _p(iters),
        _p(status), ctypes.byref(o), ctypes.byref(ex), _stream_ptr()))
    return {"D": D, "iters": iters, "status": status, "bits": bits, "bounds": bnd,
            "fallback": fb, "products": prod}


def extremal_eigenvalues(batch, tol=1e-10):
    """(eps_1, eps_N, emin_G, emax_G) per instance from SP2 runs of the library.

    eps_1 = Tr(H D) with D the SP2 projector of H for nocc = 1 (its lowest
    state); eps_N the same for -H, negated. A Rayleigh quotient of a projector
    is second-order accurate in the projector's error."""
    n = np.asarray(batch["n"])
    r1 = batched_solve(batch, np.ones_like(n), tol)
    e1 = trace_hd(batch, r1["D"])
    neg = dict(batch)
    neg["H"] = -batch["H"]
    rN = batched_solve(neg, np.ones_like(n), tol)
    eN = trace_hd(batch, rN["D"])
    return e1, eN, r1["bounds"][:, 0].clone(), r1["bounds"][:, 1].clone()


def bits_tensor_to_array(bits, length):
    """[B,4] int64 (uint64 words) -> [B, length] float32 0/1."""
    import torch
    w = bits.to(torch.int64)
    out = torch.zeros((bits.shape[0], length), dtype=torch.float32, device=bits.device)
    for k in range(length):
        out[:, k] = ((w[:, k // 64] >> (k % 64)) & 1).to(torch.float32)
    return out


def array_to_bits_tensor(arr):
    """[B, L] 0/1 -> [B,4] int64 words."""
    import torch
    B, L = arr.shape
    words = torch.zeros((B, 4), dtype=torch.int64, device=arr.device)
    for k in range(min(L, 256)):
        words[:, k // 64] |= (arr[:, k] > 0.5).to(torch.int64) << (k % 64)
    return words


class Predictor:
    """37 -> hidden -> hidden -> 2 + kmax perceptron trained with the library kernels."""

    def __init__(self, hidden=128, kmax=80, seed=0, device="cuda:0"):
        import torch
        self.nin, self.nh, self.nout = N_FEAT, hidden, N_BOUNDS + kmax
        self.kmax = kmax
        cnt = load().progress_mlp_param_count(self.nin, self.nh, self.nout)
        if cnt <= 0:
            raise ValueError("bad perceptron dimensions")
        rng = np.random.default_rng(seed)
        p = np.zeros(cnt, dtype=np.float32)
        o = 0
        for fan_in, fan_out in ((self.nin, self.nh), (self.nh, self.nh), (self.nh, self.nout)):
            p[o:o + fan_in * fan_out] = rng.standard_normal(fan_in * fan_out) * np.sqrt(2.0 / fan_in)
            o += fan_in * fan_out + fan_out
        self.device = device
        self.params = torch.from_numpy(p).to(device)
        self.grad = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = 0
        self.params_h = torch.empty(cnt, dtype=torch.int16, device=device)

    def _scratch(self, batch):
        import torch
        n = load().progress_mlp_scratch_floats(self.nin, self.nh, self.nout, batch)
        return torch.empty(int(n), dtype=torch.float32, device=self.device)

    def train_step(self, X, T, M, lr):
        """One Adam step on a mini-batch; returns the loss tensor (1 float)."""
        import torch
        B = X.shape[0]
        loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        self.step += 1
        check(load().progress_mlp_train_step(
            self.nin, self.nh, self.nout, _p(self.params), _p(self.grad), _p(self.m), _p(self.v),
            self.step, float(lr), B, _p(X), _p(T), _p(M), _p(self._scratch(B)), _p(loss),
            _stream_ptr()))
        return loss

    def gradient(self, X, T, M):
        """Loss gradient at the current parameters (no update)."""
        import torch
        B = X.shape[0]
        loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        check(load().progress_mlp_train_step(
            self.nin, self.nh, self.nout, _p(self.params), _p(self.grad), None, None, 0, 0.0, B,
            _p(X), _p(T), _p(M), _p(self._scratch(B)), _p(loss), _stream_ptr()))
        return self.grad.clone(), loss

    def fit(self, X, T, M, epochs=200, batch=256, lr=2e-3, seed=0):
        import torch
        N = X.shape[0]
        g = torch.Generator(device="cpu").manual_seed(seed)
        losses = []
        for _ in range(epochs):
            perm = torch.randperm(N, generator=g).to(X.device)
            tot = 0.0
            for s in range(0, N, batch):
                idx = perm[s:s + batch]
                if idx.numel() < 2:
                    continue
                l = self.train_step(X[idx].contiguous(), T[idx].contiguous(),
                                    M[idx].contiguous(), lr)
                tot += float(l) * idx.numel()
            losses.append(tot / N)
        return losses

    def predict(self, X):
        """[B, 2 + kmax] outputs with the FP16 inference weights."""
        import torch
        B = X.shape[0]
        check(load().progress_mlp_to_fp16(_p(self.params), self.params.numel(),
                                          _p(self.params_h), _stream_ptr()))
        Y = torch.empty((B, self.nout), dtype=torch.float32, device=self.device)
        check(load().progress_mlp_forward(self.nin, self.nh, self.nout, _p(self.params_h), B,
                                          _p(X), _p(Y), _p(self._scratch(B)), _stream_ptr()))
        return Y


def bound_fractions(eps1, epsN, emin, emax):
    """u_min = (eps_1 - emin)/w, u_max = (emax - eps_N)/w with w = emax - emin."""
    import torch
    w = emax - emin
    return (torch.clamp((eps1 - emin) / w, min=0.0), torch.clamp((emax - epsN) / w, min=0.0))


def predicted_bounds(Y, emin, emax, margin):
    """[B, 2] bounds from predicted fractions, each widened by margin * w and
    never outside the Gershgorin enclosure."""
    import torch
    w = emax - emin
    u0 = torch.clamp(Y[:, 0].double() - margin, min=0.0)
    u1 = torch.clamp(Y[:, 1].double() - margin, min=0.0)
    lo = emin + w * u0
    hi = emax - w * u1
    ok = hi > lo
    lo = torch.where(ok, lo, emin)
    hi = torch.where(ok, hi, emax)
    return torch.stack([lo, hi], dim=1).contiguous()


def calibrate_margin(Y, T, quantile=0.97, floor=0.02):
    """Margin (fraction of the Gershgorin width) that covers the predicted
    bounds' overshoot on held-out instances: the `quantile` of
    max(y_j - t_j) over both bounds, never below `floor`. A run whose bounds
    cut the spectrum is rejected by the judge and restarts on the plain path,
    so the quantile sets the expected fallback rate of that cause."""
    import torch
    over = torch.clamp(Y[:, :2].double() - T[:, :2].double(), min=0.0).max(dim=1).values
    if over.numel() == 0:
        return float(floor)
    return max(float(floor), float(torch.quantile(over, quantile).item()))


def make_targets(u_min, u_max, bits, iters, kmax):
    """Targets and masks: the two bound fractions, then the branch bits of the
    labelled SP2 run (masked beyond its product count)."""
    import torch
    B = u_min.shape[0]
    dev = u_min.device
    T = torch.zeros((B, N_BOUNDS + kmax), dtype=torch.float32, device=dev)
    M = torch.zeros_like(T)
    T[:, 0] = u_min.float()
    T[:, 1] = u_max.float()
    M[:, :N_BOUNDS] = 1.0
    T[:, N_BOUNDS:] = bits_tensor_to_array(bits, kmax)
    ks = torch.arange(kmax, device=dev)
    M[:, N_BOUNDS:] = (ks[None, :] < iters[:, None].to(torch.int64)).float()
    return T, M


def label_batch(batch, nocc, margin, kmax, tol=1e-10):
    """Features and bound targets of one packed batch (SP2-derived labels);
    the branch targets are filled by ``branch_labels`` once bounds can be
    predicted."""
    feat = features(batch)
    e1, eN, emin, emax = extremal_eigenvalues(batch, tol)
    u_min, u_max = bound_fractions(e1, eN, emin, emax)
    import torch
    iters0 = torch.zeros_like(u_min, dtype=torch.int32)
    bits0 = torch.zeros((u_min.shape[0], 4), dtype=torch.int64, device=u_min.device)
    T, M = make_targets(u_min, u_max, bits0, iters0, kmax)
    return {"X": feat, "T": T, "M": M, "emin": emin, "emax": emax, "eps1": e1, "epsN": eN}


def branch_labels(pred, batch, nocc, lab, margin, tol=1e-10):
    """Branch targets consistent with inference: the bits of an SP2 run whose
    X0 uses the bounds ``pred`` predicts (widened by margin), and bound
    targets replaced by ``pred``'s own outputs so that further training keeps
    those bounds while it learns the branches."""
    Y = pred.predict(lab["X"])
    bounds = predicted_bounds(Y, lab["emin"], lab["emax"], margin)
    run = batched_solve(batch, nocc, tol, bounds=bounds)
    ok = run["fallback"] == 0
    kmax = lab["T"].shape[1] - N_BOUNDS
    T, M = make_targets(Y[:, 0].double(), Y[:, 1].double(), run["bits"], run["iters"], kmax)
    M[~ok, N_BOUNDS:] = 0.0  # a run that failed gives no branch labels
    return T, M


def confident_prefix(logits, tau):
    """Per row, the number of leading branch logits with |logit| >= tau: only
    that prefix of the sequence is predicted; later branches are left to the
    trace rule (no prediction to judge)."""
    import torch
    conf = (logits.abs() >= tau).to(torch.int32)
    # length of the leading run of ones
    run = torch.cumprod(conf, dim=1)
    return run.sum(dim=1).to(torch.int32).contiguous()


def solve_learned(pred, batch, nocc, emin, emax, margin, judge_delta, tau=2.0, tol=1e-10):
    """Batched solve with predicted bounds and the confident prefix of the
    predicted branch sequence, judged by the trace rule."""
    X = features(batch)
    Y = pred.predict(X)
    bounds = predicted_bounds(Y, emin, emax, margin)
    logits = Y[:, N_BOUNDS:]
    bits = array_to_bits_tensor((logits > 0).float())
    plen = confident_prefix(logits, tau)
    out = batched_solve(batch, nocc, tol, bounds=bounds, pred_bits=bits, pred_len=plen,
                        judge_delta=judge_delta)
    out["pred_len"] = plen
    return out
