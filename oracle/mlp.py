"""Plain FP64 statements of the learned-sequence part -- TEST INFRASTRUCTURE ONLY.

The learned part predicts, from cheap features of H, tighter spectral bounds
for the X0 map of §IV.A (the paper's eps_1, eps_N, estimated by Gershgorin
circles in §VIII.A) and the SP2 branch sequence. Everything here is written
from its definition, in numpy, for the GPU kernels to be checked against:

* ``features``: 37 numbers per Hamiltonian -- Gershgorin emin, emax, Tr H,
  ||H||_F, a 32-bin histogram of diag(H) over [emin, emax], and n -- in the
  dimensionless form the network reads (see ``features``).
* ``mlp_forward`` / ``mlp_backward``: a 3-layer perceptron
  in -> hidden (ReLU) -> hidden (ReLU) -> out, with the loss
  L = mean over samples of [ sum over the 2 bound outputs of
        c(pred, target) (pred - target)^2,  c = C_OVER if pred > target else 1
      + sum over bit outputs k with mask 1 of BCE-with-logits(logit_k, bit_k) / max(1, #mask) ]
  The bound targets are the fractions u_min = (eps_1 - emin)/(emax - emin) and
  u_max = (emax - eps_N)/(emax - emin); predicting more than the target would
  cut the spectrum, hence the heavier weight C_OVER on that side.
* ``adam_step``: Adam (Kingma & Ba 2015) with bias correction.

Parameters are one flat vector: W1 (hidden x in), b1, W2 (hidden x hidden),
b2, W3 (out x hidden), b3, each row-major.
"""

from __future__ import annotations

import numpy as np

N_FEAT = 37
N_BOUNDS = 2
HIST_BINS = 32
C_OVER = 10.0


def features(H):
    """The 37 input features of one Hamiltonian (§VIII.A bounds, traces)."""
    H = np.asarray(H, dtype=np.float64)
    n = H.shape[0]
    d = np.diag(H)
    R = np.abs(H).sum(axis=1) - np.abs(d)
    emin, emax = float(np.min(d - R)), float(np.max(d + R))
    w = emax - emin
    if not w > 0:
        emin, emax, w = emin - 1.0, emax + 1.0, 2.0
    tr = float(d.sum())
    fro = float(np.sqrt(np.sum(H * H)))
    hist = np.zeros(HIST_BINS)
    idx = np.floor((d - emin) / w * HIST_BINS).astype(np.int64)
    idx = np.clip(idx, 0, HIST_BINS - 1)
    np.add.at(hist, idx, 1.0)
    f = np.empty(N_FEAT)
    f[0] = emin / w
    f[1] = emax / w
    f[2] = tr / (n * w)
    f[3] = fro / (np.sqrt(n) * w)
    f[4:4 + HIST_BINS] = hist / n
    f[36] = n / 2048.0
    return f


def param_count(n_in, n_hidden, n_out):
    return n_hidden * n_in + n_hidden + n_hidden * n_hidden + n_hidden + n_out * n_hidden + n_out


def unpack(p, n_in, n_hidden, n_out):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + n_hidden * n_in].reshape(n_hidden, n_in); o += n_hidden * n_in
    b1 = p[o:o + n_hidden]; o += n_hidden
    W2 = p[o:o + n_hidden * n_hidden].reshape(n_hidden, n_hidden); o += n_hidden * n_hidden
    b2 = p[o:o + n_hidden]; o += n_hidden
    W3 = p[o:o + n_out * n_hidden].reshape(n_out, n_hidden); o += n_out * n_hidden
    b3 = p[o:o + n_out]; o += n_out
    return W1, b1, W2, b2, W3, b3


def mlp_forward(p, X, n_in, n_hidden, n_out):
    """Returns (Y, cache): Y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 per row of X."""
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, n_hidden, n_out)
    X = np.asarray(X, dtype=np.float64)
    Z1 = X @ W1.T + b1
    A1 = np.maximum(Z1, 0.0)
    Z2 = A1 @ W2.T + b2
    A2 = np.maximum(Z2, 0.0)
    Y = A2 @ W3.T + b3
    return Y, (X, Z1, A1, Z2, A2)


def loss_and_grad_out(Y, T, M):
    """Loss (scalar) and dL/dY for outputs Y, targets T, masks M (same shape)."""
    B = Y.shape[0]
    G = np.zeros_like(Y)
    loss = 0.0
    # bounds: asymmetric squared error
    e = Y[:, :N_BOUNDS] - T[:, :N_BOUNDS]
    c = np.where(e > 0.0, C_OVER, 1.0)
    loss += float(np.sum(c * e * e)) / B
    G[:, :N_BOUNDS] = 2.0 * c * e / B
    # bits: masked BCE with logits, averaged over each sample's valid bits
    z = Y[:, N_BOUNDS:]
    t = T[:, N_BOUNDS:]
    m = M[:, N_BOUNDS:]
    cnt = np.maximum(m.sum(axis=1, keepdims=True), 1.0)
    bce = np.maximum(z, 0.0) - z * t + np.log1p(np.exp(-np.abs(z)))
    loss += float(np.sum(m * bce / cnt)) / B
    sig = 1.0 / (1.0 + np.exp(-z))
    G[:, N_BOUNDS:] = m * (sig - t) / cnt / B
    return loss, G


def mlp_backward(p, cache, G, n_in, n_hidden, n_out):
    """Gradient of the loss with respect to the flat parameter vector."""
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, n_hidden, n_out)
    X, Z1, A1, Z2, A2 = cache
    dW3 = G.T @ A2
    db3 = G.sum(axis=0)
    dA2 = G @ W3
    dZ2 = dA2 * (Z2 > 0.0)
    dW2 = dZ2.T @ A1
    db2 = dZ2.sum(axis=0)
    dA1 = dZ2 @ W2
    dZ1 = dA1 * (Z1 > 0.0)
    dW1 = dZ1.T @ X
    db1 = dZ1.sum(axis=0)
    return np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])


def loss_and_grad(p, X, T, M, n_in, n_hidden, n_out):
    Y, cache = mlp_forward(p, X, n_in, n_hidden, n_out)
    loss, G = loss_and_grad_out(Y, T, M)
    return loss, mlp_backward(p, cache, G, n_in, n_hidden, n_out)


def adam_step(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
