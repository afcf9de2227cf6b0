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


def _slot_out(D, Kmax, slots):
    """A network output vector from per-slot tuples (presence logit, log
    weight, mu (D), log diag (D), off-diagonals (D(D-1)/2))."""
    SP = mlp.slot_size(D)
    o, opad = mlp.out_dims(D, Kmax)
    out = np.zeros(opad)
    for s, vals in enumerate(slots):
        flat = [vals[0], vals[1], *vals[2], *vals[3], *vals[4]]
        assert len(flat) == SP
        out[s * SP:(s + 1) * SP] = flat
    for s in range(len(slots), Kmax):
        out[s * SP] = -9.0
    return out


def test_decode_caps_K0_so_that_the_penalised_weights_stay_positive():
    # 3V: T = 9, so N - T K0 / 2 > 0 allows K0 <= 4 at N = 20 and K0 = 1 at
    # N = 9.  Six slots are present; the cap drops the smallest log weights
    # one at a time (hand table: log weights 0.1, -2, 0.5, -1, 0.3, 0.2 ->
    # slots 0, 2, 4, 5 at N = 20; slot 2 alone at N = 9).
    D, Kmax = 3, 10
    lw = [0.1, -2.0, 0.5, -1.0, 0.3, 0.2]
    slots = [(1.0, lw[s], [0.1 * s, 0.0, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]) for s in range(6)]
    out = _slot_out(D, Kmax, slots)
    mean, sd = np.zeros(3), np.ones(3)
    K0, prm = mlp.decode(out, mean, sd, 20, D, Kmax)
    assert K0 == 4
    np.testing.assert_allclose(prm[:, 1], [0.0, 0.2, 0.4, 0.5])  # slots 0, 2, 4, 5 in slot order
    e = np.exp([0.1, 0.5, 0.3, 0.2])
    np.testing.assert_allclose(prm[:, 0], e / e.sum(), rtol=1e-14)
    K0, prm = mlp.decode(out, mean, sd, 9, D, Kmax)
    assert K0 == 1
    assert prm[0, 1] == pytest.approx(0.2) and prm[0, 0] == 1.0
    # 1V: T = 2, N = 3 allows K0 <= 2
    slots1 = [(2.0, w_, [0.5 * s], [0.0], []) for s, w_ in enumerate([0.0, 1.0, -1.0])]
    K0, prm = mlp.decode(_slot_out(1, 8, slots1), np.zeros(1), np.ones(1), 3, 1, 8)
    assert K0 == 2
    np.testing.assert_allclose(prm[:, 1], [0.0, 0.5])


def test_decode_keeps_at_least_the_most_likely_slot():
    # every presence logit below the threshold: the slot of the largest
    # logit alone, with weight 1, its mean and covariance
    D, Kmax = 1, 8
    slots = [(-3.0, 0.0, [1.0], [0.0], []), (-0.5, 0.7, [-2.0], [np.log(0.5)], []),
             (-1.0, 0.0, [3.0], [0.0], [])]
    mean, sd = np.array([10.0]), np.array([2.0])
    K0, prm = mlp.decode(_slot_out(D, Kmax, slots), mean, sd, 1000, D, Kmax)
    assert K0 == 1
    # mu = mean + sd * (-2) = 6; Sigma = (sd * 0.5)^2 = 1
    np.testing.assert_allclose(prm[0], [1.0, 6.0, 1.0], rtol=1e-14)
    # a higher threshold does the same even when some logits are positive
    K0, prm = mlp.decode(_slot_out(D, Kmax, [(0.5, 0.0, [1.0], [0.0], [])]), mean, sd, 1000, D,
                         Kmax, presence_logit=1.0)
    assert K0 == 1 and prm[0, 1] == pytest.approx(12.0)


def test_decode_clamps_the_log_diagonal():
    # log diag of the whitened Cholesky factor clamped to [-10, 5]: 20 -> 5,
    # -30 -> -10, 1 kept; 3V with zero off-diagonals gives a diagonal
    # covariance sd_d^2 exp(2 clamp(ld_d))
    D, Kmax = 3, 10
    slots = [(4.0, 0.0, [0.0, 0.0, 0.0], [20.0, -30.0, 1.0], [0.0, 0.0, 0.0])]
    sd = np.array([1.0, 2.0, 3.0])
    K0, prm = mlp.decode(_slot_out(D, Kmax, slots), np.zeros(3), sd, 1000, D, Kmax)
    assert K0 == 1
    # upper-triangle order: 00, 01, 02, 11, 12, 22
    S = prm[0, 4:]
    np.testing.assert_allclose(S, [np.exp(10.0), 0.0, 0.0, 4.0 * np.exp(-20.0), 0.0, 9.0 * np.exp(2.0)],
                               rtol=1e-14)
    # the off-diagonal entries of L enter unclamped: L10 = 3 gives
    # Sigma_01 = sd0 sd1 * L00 * L10
    slots = [(4.0, 0.0, [0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [3.0, 0.0, 0.0])]
    K0, prm = mlp.decode(_slot_out(D, Kmax, slots), np.zeros(3), sd, 1000, D, Kmax)
    np.testing.assert_allclose(prm[0, 4:], [1.0, 2.0 * 3.0, 0.0, 4.0 * (9.0 + 1.0), 0.0, 9.0], rtol=1e-14)


@pytest.mark.parametrize("D", [1, 3])
def test_features_of_a_zero_variance_cell_are_zero(D):
    # a cell whose velocities are all equal (in one dimension for 3V) cannot
    # be whitened: its feature vector is all zero and its sd is returned as 0
    rng = np.random.default_rng(3)
    v = rng.standard_normal((50, D))
    v[:, D - 1] = 0.25
    f, mean, sd = mlp.cell_features(v, rng.uniform(0.5, 1.5, 50))
    assert f.shape == (mlp.feat_dims(D)[2],)
    assert np.all(f == 0.0)
    assert sd[D - 1] == 0.0 and mean[D - 1] == pytest.approx(0.25)
