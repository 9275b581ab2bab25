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
backward, Adam; FP16 weights at inference); the labels, training targets,
predicted bounds, branch bits and their confident prefix come from the
library's progress_learned_* calls. At solve time the trace-driven rule
judges every predicted branch; a disagreement beyond the judge margin, or a
run that leaves [0, 1], sends that instance back to the plain path
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


def labels(batch, tol=1e-10):
    """Bound labels from SP2 runs of the library (progress_learned_labels):
    u [B, 2] float32 bound fractions (u_min, u_max of the Gershgorin width),
    gersh [B, 2] float64 Gershgorin enclosure, eps [2, B] float64 (eps_1, eps_N)."""
    import torch
    dev = batch["H"].device
    B = len(batch["n"])
    u = torch.empty((B, 2), dtype=torch.float32, device=dev)
    gersh = torch.empty((B, 2), dtype=torch.float64, device=dev)
    eps = torch.empty((2, B), dtype=torch.float64, device=dev)
    n = np.ascontiguousarray(batch["n"], dtype=np.int32)
    off = np.ascontiguousarray(batch["offsets"], dtype=np.int64)
    check(load().progress_learned_labels(
        B, ctypes.c_void_p(n.ctypes.data), ctypes.c_void_p(off.ctypes.data), _p(batch["d_n"]),
        _p(batch["d_off"]), _p(batch["H"]), float(tol), _p(u), _p(gersh), _p(eps),
        _stream_ptr()))
    return {"u": u, "gersh": gersh, "eps": eps}


def targets(ub, kmax, bits=None, iters=None, reject=None):
    """Training targets and masks [B, 2 + kmax] (progress_learned_targets): the
    bound targets from the first two columns of ub ([B, >= 2] float32), then
    the branch bits of a labelled run (bits [B, 4] words), masked beyond its
    product count (iters) and for rejected runs (reject != 0)."""
    import torch
    B, ld = ub.shape
    T = torch.empty((B, N_BOUNDS + kmax), dtype=torch.float32, device=ub.device)
    M = torch.empty_like(T)
    check(load().progress_learned_targets(
        B, int(kmax), _p(ub), ld, None if bits is None else _p(bits),
        None if iters is None else _p(iters), None if reject is None else _p(reject), _p(T),
        _p(M), _stream_ptr()))
    return T, M


def solve_inputs(Y, gersh, margin, logit_tau=None):
    """Solve inputs from the predictor's outputs Y [B, 2 + kmax]
    (progress_learned_inputs): bounds [B, 2], the predicted fractions widened by
    margin and kept inside the Gershgorin enclosure gersh [B, 2]; with
    logit_tau, also the branch bits [B, 4] (1 iff logit > 0) and the length of
    the confident prefix [B] (leading logits with |logit| >= logit_tau)."""
    import torch
    B, nout = Y.shape
    bounds = torch.empty((B, 2), dtype=torch.float64, device=Y.device)
    bits = plen = None
    if logit_tau is not None:
        bits = torch.empty((B, 4), dtype=torch.int64, device=Y.device)
        plen = torch.empty(B, dtype=torch.int32, device=Y.device)
    check(load().progress_learned_inputs(
        B, nout, _p(Y), _p(gersh), float(margin),
        float(logit_tau) if logit_tau is not None else 0.0, _p(bounds),
        None if bits is None else _p(bits), None if plen is None else _p(plen),
        _stream_ptr()))
    return bounds, bits, plen


def predicted_bounds(Y, gersh, margin):
    """[B, 2] bounds from predicted fractions, each widened by margin * w and
    never outside the Gershgorin enclosure gersh [B, 2]."""
    return solve_inputs(Y, gersh, margin)[0]


def calibrate_margin(Y, T, quantile=0.97, floor=0.02):
    """Margin (fraction of the Gershgorin width) that covers the predicted
    bounds' overshoot on held-out instances (progress_learned_margin, on the
    bound columns copied to the host)."""
    y = np.ascontiguousarray(Y[:, :2].cpu().numpy(), dtype=np.float32)
    t = np.ascontiguousarray(T[:, :2].cpu().numpy(), dtype=np.float32)
    out = ctypes.c_double(0.0)
    check(load().progress_learned_margin(y.shape[0], ctypes.c_void_p(y.ctypes.data), 2,
                                         ctypes.c_void_p(t.ctypes.data), 2, float(quantile),
                                         float(floor), ctypes.byref(out)))
    return out.value


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


def label_batch(batch, nocc, margin, kmax, tol=1e-10):
    """Features and bound targets of one packed batch (SP2-derived labels);
    the branch targets are filled by ``branch_labels`` once bounds can be
    predicted."""
    feat = features(batch)
    lab = labels(batch, tol)
    T, M = targets(lab["u"], kmax)
    return {"X": feat, "T": T, "M": M, "gersh": lab["gersh"], "eps": lab["eps"]}


def branch_labels(pred, batch, nocc, lab, margin, tol=1e-10):
    """Branch targets consistent with inference: the bits of an SP2 run whose
    X0 uses the bounds ``pred`` predicts (widened by margin), and bound
    targets replaced by ``pred``'s own outputs so that further training keeps
    those bounds while it learns the branches."""
    Y = pred.predict(lab["X"])
    run = batched_solve(batch, nocc, tol, bounds=predicted_bounds(Y, lab["gersh"], margin))
    kmax = lab["T"].shape[1] - N_BOUNDS
    return targets(Y, kmax, bits=run["bits"], iters=run["iters"], reject=run["fallback"])


def solve_learned(pred, batch, nocc, gersh, margin, judge_delta, tau=None, tol=1e-10):
    """Batched solve with predicted bounds, judged by the trace rule. With tau
    (e.g. 2.0) the confident prefix of the predicted branch sequence (leading
    logits with |logit| >= tau) is predicted as well; the default predicts the
    bounds only, which measured faster (predicted branches gain nothing once
    the loop runs on the device without host syncs, and their rejections cost
    products)."""
    Y = pred.predict(features(batch))
    bounds, bits, plen = solve_inputs(Y, gersh, margin, logit_tau=tau)
    out = batched_solve(batch, nocc, tol, bounds=bounds, pred_bits=bits, pred_len=plen,
                        judge_delta=judge_delta)
    out["pred_len"] = plen
    return out
