"""Learned-sequence part on the GPU: features, perceptron gradients and Adam
against the CPU oracle, the judge/fallback of predicted branches, and the
gain of a trained predictor over the plain method."""

import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from workloads import batch_instance, cube_hamiltonian

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available(), "GPU test run without a CUDA device"
    from paper_2401_13772_gb300.build import build
    build()
    import paper_2401_13772_gb300 as p
    p.load()
    from paper_2401_13772_gb300 import learned
    return learned


def test_features_match_oracle(L):
    mats = [cube_hamiltonian(s, 40 + s)[0] for s in (16, 33, 70)] + [np.diag([0.5, -1.0, 2.0])]
    b = L.to_device_batch(mats)
    f = L.features(b).cpu().numpy()
    for H, row in zip(mats, f):
        ref = omlp.features(H)
        assert np.abs(row[:4] - ref[:4]).max() <= 1e-5 * max(1.0, np.abs(ref[:4]).max())
        assert np.array_equal(row[4:36], ref[4:36].astype(np.float32))
        assert abs(row[36] - ref[36]) <= 1e-7


def test_trace_hd_and_labels(L):
    import torch
    mats = [cube_hamiltonian(s, 7 + s)[0] for s in (20, 48, 96)]
    b = L.to_device_batch(mats)
    D = torch.from_numpy(np.concatenate([np.eye(m.shape[0]).ravel() for m in mats])).cuda()
    t = L.trace_hd(b, D).cpu().numpy()
    assert np.allclose(t, [np.trace(m) for m in mats], atol=1e-4)
    lab = L.labels(b)
    eps = lab["eps"].cpu().numpy()
    gersh = lab["gersh"].cpu().numpy()
    u = lab["u"].cpu().numpy()
    for i, H in enumerate(mats):
        w = np.linalg.eigvalsh(H)
        emin, emax = oracle.gershgorin_bounds(H)
        assert abs(gersh[i, 0] - emin) < 1e-9 and abs(gersh[i, 1] - emax) < 1e-9
        # within the edge degeneracy: between the two lowest (highest) eigenvalues
        assert w[0] - 1e-3 <= eps[0, i] <= w[1] + 1e-3
        assert w[-2] - 1e-3 <= eps[1, i] <= w[-1] + 1e-3
        # bound fractions of the Gershgorin width, as the definition states them
        wd = emax - emin
        assert u[i, 0] == np.float32(max((eps[0, i] - gersh[i, 0]) / (gersh[i, 1] - gersh[i, 0]),
                                         0.0))
        assert u[i, 1] == np.float32(max((gersh[i, 1] - eps[1, i]) / (gersh[i, 1] - gersh[i, 0]),
                                         0.0))
        assert 0.0 <= u[i, 0] <= (w[1] - emin) / wd + 1e-3


def test_solve_inputs_and_targets_follow_their_definitions(L):
    import torch
    rng = np.random.default_rng(5)
    B, kmax, margin, tau = 7, 70, 0.03, 2.0
    Y = rng.standard_normal((B, 2 + kmax)).astype(np.float32) * 3.0
    Y[:, :2] = rng.uniform(-0.05, 0.6, (B, 2)).astype(np.float32)
    Y[3, :2] = [0.7, 0.6]  # crossing predictions -> the Gershgorin enclosure
    G = np.stack([rng.uniform(-60, -10, B), rng.uniform(5, 60, B)], 1)
    bounds, bits, plen = L.solve_inputs(torch.from_numpy(Y).cuda(), torch.from_numpy(G).cuda(),
                                        margin, logit_tau=tau)
    bounds, bits, plen = bounds.cpu().numpy(), bits.cpu().numpy(), plen.cpu().numpy()
    for i in range(B):
        w = G[i, 1] - G[i, 0]
        lo = G[i, 0] + w * max(float(Y[i, 0]) - margin, 0.0)
        hi = G[i, 1] - w * max(float(Y[i, 1]) - margin, 0.0)
        if not hi > lo:
            lo, hi = G[i, 0], G[i, 1]
        assert bounds[i, 0] == lo and bounds[i, 1] == hi
        word = [0, 0, 0, 0]
        for k in range(kmax):
            if Y[i, 2 + k] > 0:
                word[k // 64] |= 1 << (k % 64)
        assert [int(v) & (2 ** 64 - 1) for v in bits[i]] == word
        L_ = 0
        while L_ < kmax and abs(Y[i, 2 + L_]) >= tau:
            L_ += 1
        assert plen[i] == L_
    assert bounds[3, 0] == G[3, 0] and bounds[3, 1] == G[3, 1]
    # targets and masks
    iters = torch.tensor([0, 5, 70, 80, 3, 64, 65], dtype=torch.int32, device="cuda:0")
    reject = torch.tensor([0, 0, 0, 0, 1, 0, 0], dtype=torch.int32, device="cuda:0")
    wb = torch.from_numpy(rng.integers(-2 ** 62, 2 ** 62, (B, 4))).cuda()
    T, M = L.targets(torch.from_numpy(Y).cuda(), kmax, bits=wb, iters=iters, reject=reject)
    T, M, wbh = T.cpu().numpy(), M.cpu().numpy(), wb.cpu().numpy()
    for i in range(B):
        assert T[i, 0] == Y[i, 0] and T[i, 1] == Y[i, 1] and M[i, 0] == 1 and M[i, 1] == 1
        for k in range(kmax):
            assert T[i, 2 + k] == float((int(wbh[i, k // 64]) >> (k % 64)) & 1)
            assert M[i, 2 + k] == float(k < int(iters[i]) and not int(reject[i]))


def _rand_problem(seed, B=40, kmax=12, hidden=32):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((B, omlp.N_FEAT)).astype(np.float32)
    T = np.concatenate([rng.uniform(0, 0.3, (B, 2)), rng.uniform(size=(B, kmax)) > 0.5], 1)
    M = np.concatenate([np.ones((B, 2)), rng.uniform(size=(B, kmax)) > 0.2], 1)
    return X, T.astype(np.float32), M.astype(np.float32), hidden, kmax


def test_gradient_and_adam_match_oracle(L):
    import torch
    X, T, M, hid, kmax = _rand_problem(1)
    P = L.Predictor(hidden=hid, kmax=kmax, seed=3)
    p0 = P.params.cpu().numpy().astype(np.float64)
    Xd, Td, Md = (torch.from_numpy(a).cuda() for a in (X, T, M))
    g, loss = P.gradient(Xd, Td, Md)
    lref, gref = omlp.loss_and_grad(p0, X.astype(np.float64), T.astype(np.float64),
                                    M.astype(np.float64), omlp.N_FEAT, hid, 2 + kmax)
    g = g.cpu().numpy()
    assert abs(float(loss) - lref) <= 1e-5 * max(1.0, lref)
    assert np.abs(g - gref).max() <= 1e-4 * max(1.0, np.abs(gref).max())
    # one Adam step (step 1) against the oracle's update
    P.train_step(Xd, Td, Md, 1e-2)
    p1, _, _ = omlp.adam_step(p0, gref, np.zeros_like(p0), np.zeros_like(p0), 1, 1e-2)
    assert np.abs(P.params.cpu().numpy() - p1).max() <= 1e-5


def test_forward_fp16_matches_oracle_with_rounded_weights(L):
    import torch
    X, T, M, hid, kmax = _rand_problem(2)
    P = L.Predictor(hidden=hid, kmax=kmax, seed=4)
    Y = P.predict(torch.from_numpy(X).cuda()).cpu().numpy()
    ph = P.params.cpu().numpy().astype(np.float16).astype(np.float64)
    Yref, _ = omlp.mlp_forward(ph, X.astype(np.float64), omlp.N_FEAT, hid, 2 + kmax)
    assert np.abs(Y - Yref).max() <= 1e-4 * max(1.0, np.abs(Yref).max())


def test_judge_rejects_wrong_predictions_and_keeps_d(L):
    import torch
    mats = [batch_instance(i, 40)[0] for i in range(4)]
    nocc = [m.shape[0] // 2 for m in mats]
    b = L.to_device_batch(mats)
    plain = L.batched_solve(b, nocc)
    B = len(mats)
    # predicted bits = complement of the real sequence: rejected at the first
    # product with a clear margin
    wrong = (~plain["bits"]).contiguous()
    plen = torch.full((B,), 60, dtype=torch.int32, device="cuda:0")
    r = L.batched_solve(b, nocc, pred_bits=wrong, pred_len=plen, judge_delta=1e-3)
    assert r["fallback"].cpu().numpy().tolist() == [1] * B
    assert torch.equal(r["iters"], plain["iters"])
    assert (r["D"] - plain["D"]).abs().max().item() <= 1e-6
    # bounds that cut the spectrum: the run leaves [0, 1] and falls back
    lo, hi = plain["bounds"][:, 0], plain["bounds"][:, 1]
    bad = torch.stack([lo + 0.6 * (hi - lo), hi], 1).contiguous()
    r = L.batched_solve(b, nocc, bounds=bad)
    assert r["fallback"].cpu().numpy().tolist() == [1] * B
    assert (r["D"] - plain["D"]).abs().max().item() <= 1e-6
    # the real sequence and exact-ish bounds are accepted
    lab = L.labels(b)
    e1, eN = lab["eps"][0], lab["eps"][1]
    w = lab["gersh"][:, 1] - lab["gersh"][:, 0]
    good = torch.stack([e1 - 0.02 * w, eN + 0.02 * w], 1).contiguous()
    r = L.batched_solve(b, nocc, bounds=good)
    assert r["fallback"].sum().item() == 0
    assert r["iters"].double().mean().item() < plain["iters"].double().mean().item()


def test_trained_predictor_saves_iterations(L):
    """Train on SP2-labelled cube instances, evaluate on fresh ones: fewer
    products in total (a rejected predicted run counts) than the plain method,
    D still within the batched gate."""
    rng = np.random.default_rng(11)
    train_sites = rng.integers(32, 129, size=160)
    eval_sites = rng.integers(64, 129, size=40)
    margin, kmax = 0.02, 80
    tr_mats = [cube_hamiltonian(int(s), 10000 + i)[0] for i, s in enumerate(train_sites)]
    tr = L.to_device_batch(tr_mats)
    tr_nocc = [m.shape[0] // 2 for m in tr_mats]
    lab = L.label_batch(tr, tr_nocc, margin, kmax)
    P = L.Predictor(hidden=128, kmax=kmax, seed=0)
    l1 = P.fit(lab["X"], lab["T"], lab["M"], epochs=150, batch=64, lr=2e-3)
    assert l1[-1] < l1[0]
    T2, M2 = L.branch_labels(P, tr, tr_nocc, lab, margin)
    l2 = P.fit(lab["X"], T2, M2, epochs=150, batch=64, lr=1e-3)
    assert l2[-1] < l2[0]
    mats = [cube_hamiltonian(int(s), 50000 + i)[0] for i, s in enumerate(eval_sites)]
    ev = L.to_device_batch(mats)
    nocc = [m.shape[0] // 2 for m in mats]
    plain = L.batched_solve(ev, nocc)
    gersh = plain["bounds"]
    Y = P.predict(L.features(ev))
    rb = L.batched_solve(ev, nocc, bounds=L.predicted_bounds(Y, gersh, margin))
    lr = L.solve_learned(P, ev, nocc, gersh, margin, judge_delta=0.5, tau=2.0)
    pp = plain["products"].double().mean().item()
    pb = rb["products"].double().mean().item()
    pl = lr["products"].double().mean().item()
    fb_b = rb["fallback"].double().mean().item()
    fb_l = lr["fallback"].double().mean().item()
    plen = lr["pred_len"].double().mean().item()
    print(f"products per solve (rejected runs included): plain {pp:.2f}, predicted bounds "
          f"{pb:.2f} (fallback {fb_b:.2f}), bounds + predicted prefix of {plen:.1f} branches "
          f"{pl:.2f} (fallback {fb_l:.2f})")
    assert pb < pp and fb_b <= 0.2
    assert pl < pp and fb_l <= 0.3
    # D meets the split-precision gate of the batched solver (see test_gpu_batched)
    for r in (rb, lr):
        Dl = r["D"].cpu().numpy()
        for H, no, o, k in zip(mats[:4], nocc, ev["offsets"], ev["n"]):
            ref = oracle.sp2_plain(H, no, 1e-10)["D"]
            w = np.linalg.eigvalsh(H)
            emin, emax = oracle.gershgorin_bounds(H)
            g = min(0.2 * 2.0 ** -22 * (emax - emin) / (w[no] - w[no - 1]) + 1e-6, 1e-2)
            assert np.abs(Dl[o:o + k * k].reshape(k, k) - ref).max() <= g
