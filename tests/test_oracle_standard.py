"""Pins of the oracle's standard (non-adaptive) EM, K-means initialisation
and Anderson acceleration (Sec. 4), each against something other than the
oracle itself: numpy's linear solve, EM's monotonicity theorem, the
sample moments, the single-Gaussian closed form, and scipy's K-means."""
import math

import numpy as np
import pytest

import oracle
import workloads


def test_anderson_on_an_affine_map_matches_the_linear_solve():
    """On G(x) = A x + b, Anderson acceleration with memory >= n is a
    Krylov method: it reaches the fixed point (I - A)^-1 b in about n + 1
    steps, while the plain iteration converges like rho(A)^k."""
    rng = np.random.default_rng(0)
    n = 6
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    A = Q @ np.diag(np.linspace(0.5, 0.85, n)) @ Q.T + 0.01 * rng.standard_normal((n, n))
    assert np.abs(np.linalg.eigvals(A)).max() < 0.97
    b = rng.standard_normal(n)
    xstar = np.linalg.solve(np.eye(n) - A, b)
    x, res = oracle.aa_affine(A, b, np.zeros(n), memory=n, iters=n + 3)
    assert np.abs(x - xstar).max() <= 1e-8 * np.abs(xstar).max()
    assert res[-1] <= 1e-8 * res[0]
    x0, res0 = oracle.aa_affine(A, b, np.zeros(n), memory=0, iters=n + 3)
    assert res0[-1] > 1e3 * res[-1]  # memory 0 is the plain fixed-point iteration
    np.testing.assert_allclose(x0, A @ oracle.aa_affine(A, b, np.zeros(n), 0, n + 2)[0] + b,
                               rtol=1e-12, atol=1e-14)


def _cells(wl, js):
    for j in js:
        sl = slice(wl.cell_off[j], wl.cell_off[j + 1])
        yield j, wl.v[:, sl].T.astype(np.float64), wl.alpha[sl]


def test_standard_em_never_decreases_the_likelihood():
    """EM's monotonicity (Dempster, Laird & Rubin): without acceleration the
    unpenalised L(theta_i) does not decrease."""
    wl = workloads.mixture_1d1v(C=6, mean_n=600, clip=(100, 1500), seed=21)
    for j, vv, a in _cells(wl, range(wl.C)):
        r = oracle.std_cell(dict(wl.params), vv, a, cell=j, init=0, trace_cap=2000)
        tr = r["Ltrace"]
        assert tr.shape[0] >= 2
        assert np.all(np.diff(tr) >= -1e-10 * np.abs(tr[1:])), j


@pytest.mark.parametrize("init,aa", [(0, 0), (1, 0), (0, 5), (1, 5)])
def test_standard_output_has_the_sample_moments(init, aa):
    """The output is a standard EM step (eq. omegak-mle with eqs. muk,
    sigmak), so its mass, mean and covariance are the cell's weighted sample
    moments (Sec. 2.3.1), with or without acceleration."""
    wl = workloads.with_weights(workloads.bimaxwellian_1d3v(C=4, ppc=500, seed=22))
    p = dict(wl.params)
    r = oracle.standard(p, wl.cell_off, wl.x, wl.v, wl.alpha, init=init, aa_memory=aa)
    D = wl.D
    for j, vv, a in _cells(wl, range(wl.C)):
        K = r["K"][j]
        prm = r["params"][j, :K]
        w = prm[:, 0]
        mu = prm[:, 1:1 + D]
        W = a.sum()
        m = (a[:, None] * vv).sum(0) / W
        S = ((a[:, None] * (vv - m)).T @ (vv - m)) / W
        assert abs(w.sum() - 1.0) <= 1e-13
        np.testing.assert_allclose(w @ mu, m, rtol=0, atol=1e-12 * np.abs(vv).max())
        M2 = np.zeros((D, D))
        for k in range(K):
            Sk = np.zeros((D, D))
            t = 1 + D
            for i in range(D):
                for jj in range(i, D):
                    Sk[i, jj] = Sk[jj, i] = prm[k, t]
                    t += 1
            M2 += w[k] * (Sk + np.outer(mu[k], mu[k]))
        np.testing.assert_allclose(M2 - np.outer(m, m), S, rtol=0, atol=1e-12 * np.abs(S).max())
        assert r["status"][j] & oracle.ST_EM_MAXSWEEPS == 0


def test_standard_single_component_is_the_closed_form():
    """K = 1: one EM step gives the weighted sample mean and covariance, and
    L = -N/2 (D ln 2 pi + ln |Sigma| + D)."""
    wl = workloads.with_weights(workloads.bimaxwellian_1d3v(C=2, ppc=300, seed=23))
    p = dict(wl.params, Kmax=1)
    for j, vv, a in _cells(wl, range(wl.C)):
        r = oracle.std_cell(p, vv, a, cell=j, init=0)
        N = vv.shape[0]
        W = a.sum()
        m = (a[:, None] * vv).sum(0) / W
        S = ((a[:, None] * (vv - m)).T @ (vv - m)) / W
        assert r["K"] == 1
        np.testing.assert_allclose(r["params"][0, 1:4], m, rtol=1e-13, atol=1e-15)
        L = -0.5 * N * (3 * math.log(2 * math.pi) + np.linalg.slogdet(S)[1] + 3)
        assert abs(r["lnL"] - L) <= 1e-10 * abs(L)


def test_kmeans_matches_scipy_from_the_same_centres():
    """Well-separated clusters (no near ties): the oracle's Lloyd iteration
    in whitened coordinates ends with scipy's kmeans2 partition from the
    same initial centres; the components are its clusters' shares, means
    and covariances."""
    vq = pytest.importorskip("scipy.cluster.vq")
    rng = np.random.default_rng(24)
    centres = np.array([[-3.0, 0.0, 1.0], [2.0, 2.5, -1.0], [0.5, -3.0, 2.0]])
    vv = np.concatenate([c + 0.3 * rng.standard_normal((200, 3)) for c in centres])
    ah = np.ones(vv.shape[0])
    picks = np.array([5, 210, 450])
    K, prm, passes = oracle.kmeans(vv, ah, picks)
    mean = vv.mean(0)
    sd = vv.std(0)
    y = (vv - mean) / sd
    cb, lab = vq.kmeans2(y, y[picks].copy(), iter=50, minit="matrix")
    assert K == 3 and passes >= 2
    for k in range(3):
        mem = vv[lab == k]
        np.testing.assert_allclose(prm[k, 0], mem.shape[0] / vv.shape[0], rtol=1e-13)
        np.testing.assert_allclose(prm[k, 1:4], mem.mean(0), rtol=1e-12, atol=1e-13)
        C = np.cov(mem.T, bias=True)
        np.testing.assert_allclose(prm[k, 4:], C[np.triu_indices(3)], rtol=1e-11, atol=1e-13)


def test_anderson_and_kmeans_accelerate_standard_em():
    """The paper's observation (Sec. 4): AA, and AA with K-means, need far
    fewer EM iterations than plain EM from random particles; every
    accelerated cell converges."""
    wl = workloads.mixture_1d1v(C=32, mean_n=800, clip=(100, 2000), seed=25)
    p = dict(wl.params)
    plain = oracle.standard(p, wl.cell_off, wl.x, wl.v, wl.alpha, init=0, aa_memory=0, nthreads=4)
    aa = oracle.standard(p, wl.cell_off, wl.x, wl.v, wl.alpha, init=0, aa_memory=5, nthreads=4)
    kaa = oracle.standard(p, wl.cell_off, wl.x, wl.v, wl.alpha, init=1, aa_memory=5, nthreads=4)
    assert aa["iters"].mean() < 0.5 * plain["iters"].mean()
    assert kaa["iters"].mean() < 0.5 * plain["iters"].mean()
    assert np.all((kaa["status"] & oracle.ST_EM_MAXSWEEPS) == 0)
    assert kaa["aa_steps"].sum() > 0
