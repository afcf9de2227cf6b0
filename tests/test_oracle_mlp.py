"""Pins of the learned-initialisation network's FP64 oracle: finite-difference
gradients, torch's Adam, feature and target definitions, and the
decode(targets) round trip."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import mlp
import workloads


@pytest.mark.parametrize("D,Kmax", [(1, 8), (3, 10)])
def test_backward_matches_finite_differences(D, Kmax):
    rng = np.random.default_rng(D)
    p = mlp.init_params(D, Kmax, seed=3)
    _, _, F = mlp.feat_dims(D)
    o, opad = mlp.out_dims(D, Kmax)
    B = 5
    X = rng.standard_normal((B, F))
    T = rng.standard_normal((B, opad))
    SP = mlp.slot_size(D)
    Mk = np.zeros((B, opad))
    for b in range(B):
        K = 1 + b % Kmax
        for s in range(Kmax):
            Mk[b, s * SP] = 1
            T[b, s * SP] = 1.0 if s < K else 0.0
            if s < K:
                Mk[b, s * SP + 1:(s + 1) * SP] = 1

    def loss(pp):
        f = mlp.forward(pp, X, round_bf16=False)
        return mlp.loss_and_grad_out(f["out"], T, Mk, D, Kmax)[0]

    f = mlp.forward(p, X, round_bf16=False)
    L, G = mlp.loss_and_grad_out(f["out"], T, Mk, D, Kmax)
    g = mlp.backward(p, f, G)
    h = 1e-6
    for name in p:
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, 6, replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = loss(p)
            flat[idx] = old - h
            lm = loss(p)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, an)


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    p = {"W": rng.standard_normal((4, 3)), "b": rng.standard_normal(4)}
    tp = {k: torch.tensor(v.copy(), requires_grad=True) for k, v in p.items()}
    opt = torch.optim.Adam(list(tp.values()), lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    state = {}
    for t in range(1, 6):
        g = {k: rng.standard_normal(v.shape) for k, v in p.items()}
        mlp.adam_step(p, g, state, 1e-2, t)
        for k in tp:
            tp[k].grad = torch.tensor(g[k])
        opt.step()
    for k in p:
        np.testing.assert_allclose(p[k], tp[k].detach().numpy(), rtol=1e-12, atol=1e-14)


def test_features_1v():
    rng = np.random.default_rng(1)
    v = rng.standard_normal((20000, 1)) * 0.3 + 0.2
    a = np.ones(20000)
    f, mean, sd = mlp.cell_features(v, a)
    y = (v[:, 0] - 0.2) / 0.3
    assert mean[0] == pytest.approx(v.mean(), rel=1e-13)
    assert sd[0] == pytest.approx(v.std(), rel=1e-12)
    assert f[0] == pytest.approx(stats.skew(v[:, 0]), abs=1e-10)
    assert f[1] == pytest.approx(stats.kurtosis(v[:, 0]), abs=1e-10)
    assert f[2] == pytest.approx(math.log(20000) / 10)
    assert f[3:67].sum() == pytest.approx(64.0)
    assert np.all(f[67:] == 0)
    # Gaussian histogram: centre bins near 64 * pdf * width
    c = f[3 + 32]
    assert c == pytest.approx(64 * stats.norm.pdf(0.0625) * 0.125, rel=0.08)
    del y


def test_features_3v_weighted():
    wl = workloads.with_weights(workloads.bimaxwellian_1d3v(C=1, ppc=5000))
    v = wl.v.T.astype(np.float64)
    a = wl.alpha
    f, mean, sd = mlp.cell_features(v, a)
    w = a / a.sum()
    y = (v - mean) / sd
    np.testing.assert_allclose(f[0:3], (w[:, None] * y ** 3).sum(0), atol=1e-12)
    assert f[6] == pytest.approx((w * y[:, 0] * y[:, 1]).sum(), abs=1e-12)
    assert f[10:522].sum() == pytest.approx(512.0)
    assert f.shape == (576,)


@pytest.mark.parametrize("D,Kmax", [(1, 8), (3, 10)])
def test_decode_of_targets_reproduces_the_fit(D, Kmax):
    rng = np.random.default_rng(4 + D)
    K = 3
    P = 1 + D + D * (D + 1) // 2
    mean = rng.standard_normal(D)
    sd = rng.uniform(0.5, 2.0, D)
    prm = np.zeros((K, P))
    w = rng.dirichlet(np.ones(K))
    for k in range(K):
        A = rng.standard_normal((D, D)) * 0.3 + np.eye(D)
        S = A @ A.T
        prm[k, 0] = w[k]
        prm[k, 1:1 + D] = rng.standard_normal(D)
        t = 1 + D
        for a_ in range(D):
            for b_ in range(a_, D):
                prm[k, t] = S[a_, b_]
                t += 1
    T, Mk = mlp.cell_targets(K, prm, mean, sd, D, Kmax)
    out = T.copy()
    SP = mlp.slot_size(D)
    out[0:Kmax * SP:SP] = np.where(T[0:Kmax * SP:SP] > 0, 5.0, -5.0)
    K0, dec = mlp.decode(out, mean, sd, 10000, D, Kmax)
    assert K0 == K
    order = np.argsort(prm[:, 1])  # decode returns components sorted by whitened mu_0
    np.testing.assert_allclose(dec, prm[order], rtol=1e-10, atol=1e-12)


def test_bf16_rounding():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).standard_normal(10000) * 10.0 ** np.random.default_rng(1).uniform(-5, 5, 10000)
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).double().numpy()
    np.testing.assert_array_equal(mlp.bf16(x), ref)
