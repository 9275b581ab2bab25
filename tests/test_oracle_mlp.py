"""Pins of the learned-part oracle: features from their definitions, gradients
against central finite differences, Adam against its closed first step."""

import numpy as np

from oracle import mlp
from oracle import sp2 as osp2
from workloads import chain_hamiltonian, cube_hamiltonian

NI, NH, NO = mlp.N_FEAT, 16, mlp.N_BOUNDS + 6


def test_features_by_hand():
    H, _ = chain_hamiltonian(64, -1.0, -0.6)
    f = mlp.features(H)
    assert f.shape == (37,)
    # Gershgorin of the chain is exactly +-1.6 (width 3.2); zero onsite
    assert abs(f[0] + 0.5) < 1e-15 and abs(f[1] - 0.5) < 1e-15
    assert f[2] == 0.0
    # ||H||_F^2 = 64 * (1 + 0.36): per-row rms hopping over the width
    assert abs(f[3] - np.sqrt(64 * 1.36) / (8.0 * 3.2)) < 1e-14
    # all diagonal entries (0) fall in the middle bin: (0 + 1.6)/3.2 * 32 = 16
    assert f[4 + 16] == 1.0 and f[4:36].sum() == 1.0
    assert f[36] == 64 / 2048.0


def test_features_cube_consistent_with_bounds():
    H, _ = cube_hamiltonian(40, 2)
    f = mlp.features(H)
    emin, emax = osp2.gershgorin_bounds(H)
    w = emax - emin
    assert abs(f[0] * w - emin) < 1e-12 and abs(f[1] * w - emax) < 1e-12
    assert abs(f[4:36].sum() - 1.0) < 1e-15
    # onsite +-1 alternate: two histogram bins hold half the diagonal each
    nz = np.sort(f[4:36][f[4:36] > 0])
    assert np.allclose(nz, [0.5, 0.5])


def _data(seed, B=7):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(mlp.param_count(NI, NH, NO)) * 0.3
    X = rng.standard_normal((B, NI))
    T = np.concatenate([rng.uniform(0, 1, (B, 2)), (rng.uniform(size=(B, NO - 2)) > 0.5)], 1)
    M = np.concatenate([np.ones((B, 2)), (rng.uniform(size=(B, NO - 2)) > 0.3)], 1).astype(float)
    return p, X, T.astype(float), M


def test_gradient_matches_finite_differences():
    p, X, T, M = _data(1)
    loss, g = mlp.loss_and_grad(p, X, T, M, NI, NH, NO)
    rng = np.random.default_rng(3)
    idx = rng.choice(p.size, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        lp, _ = mlp.loss_and_grad(p + e, X, T, M, NI, NH, NO)
        lm, _ = mlp.loss_and_grad(p - e, X, T, M, NI, NH, NO)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_loss_pieces_by_definition():
    # one sample, bounds over- and under-shooting, one masked bit
    Y = np.array([[0.7, 0.1, 2.0, -1.0]])
    T = np.array([[0.5, 0.3, 1.0, 1.0]])
    M = np.array([[1.0, 1.0, 1.0, 0.0]])
    loss, G = mlp.loss_and_grad_out(Y, T, M)
    bce = np.log1p(np.exp(-2.0))  # z = 2, t = 1
    assert abs(loss - (10.0 * 0.04 + 0.04 + bce)) < 1e-14
    assert G[0, 3] == 0.0
    assert abs(G[0, 0] - 2 * 10.0 * 0.2) < 1e-14 and abs(G[0, 1] - 2 * (-0.2)) < 1e-14


def test_adam_first_step_is_signed_lr():
    p = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -4.0, 0.0])
    p1, m, v = mlp.adam_step(p, g, np.zeros(3), np.zeros(3), 1, 0.01)
    # bias-corrected first step: m_hat = g, v_hat = g^2 -> lr * g/(|g| + eps)
    assert np.allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8))


def test_training_reduces_loss():
    p, X, T, M = _data(5, B=32)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    l0, _ = mlp.loss_and_grad(p, X, T, M, NI, NH, NO)
    for s in range(1, 201):
        _, g = mlp.loss_and_grad(p, X, T, M, NI, NH, NO)
        p, m, v = mlp.adam_step(p, g, m, v, s, 1e-2)
    l1, _ = mlp.loss_and_grad(p, X, T, M, NI, NH, NO)
    assert l1 < 0.5 * l0
