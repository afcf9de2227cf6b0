"""The learned-initialisation pipeline on the GPU against the FP64 oracle of
the network (oracle/mlp.py): features, targets, forward, gradients (BF16
tensor-core GEMMs: per-tensor relative error <= 1e-2 and cosine >= 0.999),
Adam's first step, decode, EM from supplied mixtures, and the gain of the
trained network over the paper's random initialisation."""
import os

import numpy as np
import pytest

import oracle
from oracle import mlp
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
NTHREADS = os.cpu_count() or 4


@pytest.fixture(scope="module")
def gm():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2007_12273_gb300 import build, gm as gm_
    build.build()
    gm_.load()
    return gm_


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def bf16_round(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).double().numpy()


@pytest.mark.parametrize("which", ["1v", "3v"])
def test_features_match_oracle(gm, which):
    wl = (workloads.with_weights(workloads.mixture_1d1v(C=40, mean_n=500, clip=(50, 900))) if which == "1v"
          else workloads.bimaxwellian_1d3v(C=20, ppc=700))
    cfg = gm.config(wl.params)
    feat, wstat = gm.gm_features(cfg, dev(wl.cell_off), dev(wl.v), dev(wl.alpha))
    feat = feat.float().cpu().numpy()
    wstat = wstat.cpu().numpy()
    D = wl.D
    for j in range(wl.C):
        sl = slice(wl.cell_off[j], wl.cell_off[j + 1])
        f, mean, sd = mlp.cell_features(wl.v[:, sl].T, wl.alpha[sl])
        # FP32 whitening statistics (the features are BF16 and the whitening
        # only maps the network's start back to the cell): the mean within
        # 2e-6 of the cell's spread, the spread within 2e-6 relative
        np.testing.assert_allclose(wstat[j, :D], mean, rtol=0, atol=2e-6 * sd.max())
        np.testing.assert_allclose(wstat[j, D:], sd, rtol=2e-6)
        one = 2.0 * (64 if D == 1 else 512) / (sl.stop - sl.start)  # a particle near a bin edge
        np.testing.assert_allclose(feat[j], bf16_round(f), rtol=1e-2, atol=one)


@pytest.mark.parametrize("which", ["1v", "3v"])
def test_targets_and_decode_match_oracle(gm, which):
    wl = (workloads.mixture_1d1v(C=30, mean_n=600, clip=(100, 900)) if which == "1v"
          else workloads.bimaxwellian_1d3v(C=12, ppc=600))
    D, Kmax = wl.D, wl.params["Kmax"]
    fit = oracle.compress(wl.params, wl.cell_off, wl.x, wl.v, wl.alpha, nthreads=NTHREADS)
    cfg = gm.config(wl.params)
    _, wstat = gm.gm_features(cfg, dev(wl.cell_off), dev(wl.v), dev(wl.alpha))
    T, Mk = gm.gm_mlp_targets(cfg, dev(fit["K"]), dev(fit["params"]), wstat)
    T, Mk = T.cpu().numpy(), Mk.cpu().numpy()
    rng = np.random.default_rng(3)
    outs = np.zeros((wl.C, gm.out_width(D, Kmax)), dtype=np.float32)
    for j in range(wl.C):
        sl = slice(wl.cell_off[j], wl.cell_off[j + 1])
        _, mean, sd = mlp.cell_features(wl.v[:, sl].T, wl.alpha[sl])
        t, m = mlp.cell_targets(fit["K"][j], fit["params"][j], mean, sd, D, Kmax)
        np.testing.assert_array_equal(Mk[j], m)
        np.testing.assert_allclose(T[j], t, rtol=1e-5, atol=1e-6)
        outs[j] = (t + 0.3 * rng.standard_normal(t.shape)).astype(np.float32)
    for thr in (0.0, -0.75, -2.5):  # presence-logit thresholds (exact in FP32)
        K0, prm = gm.gm_mlp_decode(cfg, dev(outs), wstat, dev(wl.cell_off), presence_logit=thr)
        K0, prm = K0.cpu().numpy(), prm.cpu().numpy()
        for j in range(wl.C):
            sl = slice(wl.cell_off[j], wl.cell_off[j + 1])
            _, mean, sd = mlp.cell_features(wl.v[:, sl].T, wl.alpha[sl])
            k0, dec = mlp.decode(outs[j].astype(np.float64), mean, sd, sl.stop - sl.start, D, Kmax,
                                 presence_logit=thr)
            assert K0[j] == k0
            # FP32 whitening statistics: means and covariances within 1e-5
            # relative (1e-7 absolute for means near zero)
            np.testing.assert_allclose(prm[j, :k0], dec, rtol=1e-5, atol=1e-7)


def _net_and_batch(gm, D, Kmax, B, seed):
    rng = np.random.default_rng(seed)
    F, O = gm.feat_width(D), gm.out_width(D, Kmax)
    p = mlp.init_params(D, Kmax, seed=seed)
    for k in p:
        if k.startswith("b"):
            p[k] = 0.1 * rng.standard_normal(p[k].shape)
    pr = {k: bf16_round(v) if k.startswith("W") else v.astype(np.float32).astype(np.float64)
          for k, v in p.items()}
    X = bf16_round(rng.standard_normal((B, F)) * 0.5)
    SP = gm.slot_size(D)
    T = (rng.standard_normal((B, O)) * 0.5).astype(np.float32).astype(np.float64)
    Mk = np.zeros((B, O))
    for b in range(B):
        K = 1 + b % Kmax
        for s in range(Kmax):
            Mk[b, s * SP] = 1
            T[b, s * SP] = 1.0 if s < K else 0.0
            if s < K:
                Mk[b, s * SP + 1:(s + 1) * SP] = 1
    net = gm.Net(D, Kmax)
    net.load([p[f"W{i}"] for i in range(1, 5)], [p[f"b{i}"] for i in range(1, 5)])
    return net, pr, X, T, Mk


@pytest.mark.parametrize("D,Kmax", [(1, 8), (3, 10)])
def test_forward_and_gradients_match_oracle(gm, D, Kmax):
    B = 256
    net, pr, X, T, Mk = _net_and_batch(gm, D, Kmax, B, seed=D)
    Xd = dev(X.astype(np.float32)).to(torch.bfloat16)
    out = net.forward(Xd).cpu().numpy()
    f = mlp.forward(pr, X)
    scale = np.abs(f["out"]).max()
    assert np.abs(out - f["out"]).max() <= 1e-2 * scale
    loss = net.train_step(Xd, dev(T.astype(np.float32)), dev(Mk.astype(np.float32)), lr=0.0)
    Lo, G = mlp.loss_and_grad_out(f["out"], T, Mk, D, Kmax)
    g = mlp.backward(pr, f, G)
    assert float(loss.item()) == pytest.approx(Lo, rel=2e-2)
    assert int(net.err.item()) == 0
    for l in range(4):
        for nm, gpu in ((f"W{l+1}", net.gW[l]), (f"b{l+1}", net.gb[l])):
            a = gpu.double().cpu().numpy().ravel()
            b = g[nm].ravel()
            rel = np.linalg.norm(a - b) / np.linalg.norm(b)
            cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
            assert rel <= 1e-2 and cos >= 0.999, (nm, rel, cos)


def test_adam_first_step_and_loss_decreases(gm):
    D, Kmax, B = 1, 8, 512
    net, pr, X, T, Mk = _net_and_batch(gm, D, Kmax, B, seed=5)
    Xd = dev(X.astype(np.float32)).to(torch.bfloat16)
    Td, Mkd = dev(T.astype(np.float32)), dev(Mk.astype(np.float32))
    W0 = [w.clone() for w in net.W]
    net.train_step(Xd, Td, Mkd, lr=1e-3)
    # Adam's first step moves every parameter by lr * g / (|g| + eps)
    for l in range(4):
        gW = net.gW[l]
        exp = W0[l] - 1e-3 * gW / (gW.abs() + 1e-8)
        torch.testing.assert_close(net.W[l], exp, rtol=0, atol=2e-6)
    losses = []
    for _ in range(60):
        losses.append(float(net.train_step(Xd, Td, Mkd, lr=1e-3).item()))
    assert losses[-1] < 0.5 * losses[0]


def test_compress_from_given_mixtures_matches_oracle(gm):
    wl = workloads.mixture_1d1v(C=48, mean_n=800, clip=(200, 1500), seed=11)
    fit = oracle.compress(wl.params, wl.cell_off, wl.x, wl.v, wl.alpha, nthreads=NTHREADS)
    # initial mixtures: the oracle's fits with perturbed means, plus one
    # invalid component (zero covariance) in every other cell
    rng = np.random.default_rng(2)
    K0 = fit["K"].copy()
    ip = fit["params"].copy()
    ip[:, :, 1] += 0.02 * rng.standard_normal(ip[:, :, 1].shape) * (ip[:, :, 0] > 0)
    for j in range(0, wl.C, 2):
        if K0[j] < wl.params["Kmax"]:
            ip[j, K0[j]] = [0.1, 0.0, 0.0]
            K0[j] += 1
    ref = oracle.compress(wl.params, wl.cell_off, wl.x, wl.v, wl.alpha, nthreads=NTHREADS,
                          init_K=K0, init_params=ip)
    cfg = gm.config(wl.params)
    out = gm.gm_compress(cfg, dev(wl.cell_off), dev(wl.x), dev(wl.v), dev(wl.alpha),
                         init_K=dev(K0), init_params=dev(ip))
    g = {k: v.cpu().numpy() for k, v in out.items()}
    rel = np.abs(g["lnL"] - ref["lnL"]) / np.abs(ref["lnL"])
    agree = (g["K"] == ref["K"]) & (rel <= 1e-5)
    assert agree.mean() >= 0.9, (np.flatnonzero(~agree), rel[~agree])
    # warm starts converge in few sweeps
    assert ref["sweeps"].mean() < 200


def test_learned_initialisation_gain(gm):
    """Train on the method's own fits; on held-out cells the learned start
    needs fewer sweeps and reaches the plain EM's penalised likelihood."""
    from paper_2007_12273_gb300 import learned
    tr = workloads.mixture_1d1v(C=8192, seed=101)
    ev = workloads.mixture_1d1v(C=2048, seed=202)
    cfg = gm.config(tr.params)
    t = lambda a: dev(a)
    feat, T, Mk, _ = learned.fit_targets(cfg, t(tr.cell_off), t(tr.x), t(tr.v), t(tr.alpha))
    net = gm.Net(1, tr.params["Kmax"])
    net.init_weights(seed=1)
    hist = learned.train(net, feat, T, Mk, epochs=40, batch=1024, lr=1e-3)
    assert hist["loss"][-1] < 0.6 * hist["loss"][0]
    plain = gm.gm_compress(cfg, t(ev.cell_off), t(ev.x), t(ev.v), t(ev.alpha))
    lrn = learned.compress_learned(net, cfg, t(ev.cell_off), t(ev.x), t(ev.v), t(ev.alpha))
    sp = plain["sweeps"].double().mean().item()
    sl = lrn["sweeps"].double().mean().item()
    Lp = plain["lnL"].cpu().numpy()
    Ll = lrn["lnL"].cpu().numpy()
    reach = np.mean(Ll >= Lp - 1e-4 * np.abs(Lp))
    print(f"learned init: sweeps {sl:.1f} vs plain {sp:.1f}; reaches plain L (1e-4): {reach:.3f}; "
          f"mean L {Ll.mean():.3f} vs {Lp.mean():.3f}")
    assert sl < 0.8 * sp
    assert reach >= 0.5
