"""Pins of the oracle's simultaneous penalised EM with annihilation (the
simultaneous variant of the component-wise EM of Sec. 2.3), each against
something other than the oracle: two steps recomputed here with scipy
densities (eqs. responsibility, omegak, muk, sigmak, lnL-GM, omegak-mle),
the monotonicity of EM for the penalised objective (it is an EM for a MAP
estimate with the prior prod_k omega_k^(-T/2)), the sample moments, the
closed form for one Gaussian, and beams that must end one component each."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
import workloads


def _unpack(D, prm):
    w = prm[0]
    mu = prm[1:1 + D]
    S = np.zeros((D, D))
    t = 1 + D
    for i in range(D):
        for j in range(i, D):
            S[i, j] = S[j, i] = prm[t]
            t += 1
    return w, mu, S


def _pack(D, w, mu, S):
    return np.concatenate([[w], mu, S[np.triu_indices(D)]])


def _resp(D, comps, vv, ah):
    """gamma_pk = ah_p w_k f_k(v_p) / sum_j w_j f_j(v_p) and sum_p ah_p ln sum_k w_k f_k"""
    f = np.stack([w * stats.multivariate_normal(mean=mu, cov=S).pdf(vv).reshape(-1)
                  for w, mu, S in comps], axis=1)
    tot = f.sum(1)
    return ah[:, None] * f / tot[:, None], float(np.sum(ah * np.log(tot)))


def _moments(gam, vv):
    Nk = gam.sum(0)
    out = []
    for k in range(gam.shape[1]):
        if not Nk[k] > 0:
            out.append((0.0, None, None))
            continue
        mu = (gam[:, k, None] * vv).sum(0) / Nk[k]
        d = vv - mu
        S = (gam[:, k, None] * d).T @ d / Nk[k]
        out.append((Nk[k], mu, S))
    return out


def _penalised_step(D, comps, vv, ah):
    """one simultaneous penalised step from comps: (new comps, penalised L at comps)"""
    T = D * (D + 3) / 2
    gam, Lplain = _resp(D, comps, vv, ah)
    K = len(comps)
    L = Lplain - (K * (T + 1) - 1) / 2 * math.log(vv.shape[0]) - T / 2 * sum(
        math.log(w) for w, _, _ in comps)
    mom = _moments(gam, vv)
    keep = [(Nk - T / 2, mu, S) for Nk, mu, S in mom if Nk - T / 2 > 0]
    den = sum(a for a, _, _ in keep)
    return [(a / den, mu, S) for a, mu, S in keep], L


def _final_step(D, comps, vv, ah):
    gam, _ = _resp(D, comps, vv, ah)
    N = vv.shape[0]
    return [(Nk / N, mu, S) for Nk, mu, S in _moments(gam, vv)]


@pytest.mark.parametrize("D", [1, 3])
def test_two_steps_recomputed_with_scipy(D):
    """max_sweeps = 2 from a supplied mixture: the output is the final
    unpenalised step from one penalised step; the supplied mixture holds a
    far, light component that the penalised step must annihilate."""
    rng = np.random.default_rng(40 + D)
    N = 300
    vv = np.concatenate([rng.normal(-1.0, 0.4, (N // 2, D)), rng.normal(1.0, 0.6, (N - N // 2, D))])
    alpha = rng.uniform(0.5, 1.5, N)
    ah = alpha * N / alpha.sum()
    I = np.eye(D)
    init = [(0.45, -0.8 * np.ones(D), 0.3 * I), (0.45, 0.9 * np.ones(D), 0.5 * I),
            (0.10, 25.0 * np.ones(D), 0.2 * I)]
    prm0 = np.stack([_pack(D, *c) for c in init])
    p = dict(D=D, Kmax=4, shape_order=2, tol=0.0, max_sweeps=2, seed=1, L=1.0, q=1.0)
    r = oracle.std_cell(p, vv, alpha, init=2, init_params=prm0, penalised=True, trace_cap=4)
    th1, L0 = _penalised_step(D, init, vv, ah)
    assert len(th1) == 2  # the far component owns nothing
    _, L1 = _penalised_step(D, th1, vv, ah)
    out = _final_step(D, th1, vv, ah)
    assert r["K"] == 2 and r["iters"] == 2
    np.testing.assert_allclose(r["Ltrace"], [L0, L1], rtol=1e-11)
    for k in range(2):
        w, mu, S = _unpack(D, r["params"][k])
        np.testing.assert_allclose(w, out[k][0], rtol=1e-11)
        np.testing.assert_allclose(mu, out[k][1], rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(S, out[k][2], rtol=1e-10, atol=1e-12)
    _, lnL = _resp(D, out, vv, ah)
    assert r["lnL"] == pytest.approx(lnL, rel=1e-11)


@pytest.mark.parametrize("D", [1, 3])
def test_standard_two_iterations_recomputed_with_scipy(D):
    """The plain standard EM of Sec. 4 (no penalty, no annihilation): with
    max_sweeps = 2 from a supplied mixture, the trace holds the unpenalised
    eq. (lnL-GM) at the start and after one EM step (eqs. responsibility,
    muk, sigmak, omegak-mle), and the output is one more EM step; all
    recomputed here with scipy densities.  A light far component stays."""
    rng = np.random.default_rng(50 + D)
    N = 300
    vv = np.concatenate([rng.normal(-1.0, 0.4, (N // 2, D)), rng.normal(1.0, 0.6, (N - N // 2, D))])
    alpha = rng.uniform(0.5, 1.5, N)
    ah = alpha * N / alpha.sum()
    I = np.eye(D)
    init = [(0.45, -0.8 * np.ones(D), 0.3 * I), (0.45, 0.9 * np.ones(D), 0.5 * I),
            (0.10, 1.5 * np.ones(D), 0.2 * I)]
    prm0 = np.stack([_pack(D, *c) for c in init])
    p = dict(D=D, Kmax=4, shape_order=2, tol=0.0, max_sweeps=2, seed=1, L=1.0, q=1.0)
    r = oracle.std_cell(p, vv, alpha, init=2, init_params=prm0, trace_cap=4)
    _, L0 = _resp(D, init, vv, ah)
    th1 = _final_step(D, init, vv, ah)
    _, L1 = _resp(D, th1, vv, ah)
    out = _final_step(D, th1, vv, ah)
    assert r["K"] == 3 and r["iters"] == 2
    np.testing.assert_allclose(r["Ltrace"], [L0, L1], rtol=1e-11)
    for k in range(3):
        w, mu, S = _unpack(D, r["params"][k])
        np.testing.assert_allclose(w, out[k][0], rtol=1e-11)
        np.testing.assert_allclose(mu, out[k][1], rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(S, out[k][2], rtol=1e-10, atol=1e-12)
    _, lnL = _resp(D, out, vv, ah)
    assert r["lnL"] == pytest.approx(lnL, rel=1e-11)


def test_penalised_objective_never_decreases_without_annihilation():
    """Two well-separated beams fitted with Kmax = 2: no component is ever
    annihilated (every N_k >> T/2), so K is constant and the penalised L,
    which differs from the MAP objective by a constant, is non-decreasing."""
    rng = np.random.default_rng(44)
    for cell in range(4):
        vv = np.concatenate([rng.normal(-0.5, 0.05, (700, 1)), rng.normal(0.4, 0.08, (500, 1))])
        alpha = np.ones(vv.shape[0])
        p = dict(D=1, Kmax=2, shape_order=2, tol=1e-9, max_sweeps=400, seed=1, L=1.0, q=1.0)
        r = oracle.std_cell(p, vv, alpha, cell=cell, penalised=True, trace_cap=400)
        tr = r["Ltrace"]
        assert r["K"] == 2 and tr.shape[0] > 3
        assert np.all(np.diff(tr) >= -1e-10 * np.abs(tr[1:])), cell


@pytest.mark.parametrize("init", [0, 1])
def test_output_has_the_sample_moments(init):
    wl = workloads.with_weights(workloads.bimaxwellian_1d3v(C=4, ppc=500, seed=45))
    r = oracle.standard(dict(wl.params), wl.cell_off, wl.x, wl.v, wl.alpha, init=init, penalised=True)
    for j in range(wl.C):
        sl = slice(wl.cell_off[j], wl.cell_off[j + 1])
        vv = wl.v[:, sl].T.astype(np.float64)
        a = wl.alpha[sl]
        m = (a[:, None] * vv).sum(0) / a.sum()
        S = ((a[:, None] * (vv - m)).T @ (vv - m)) / a.sum()
        comps = [_unpack(3, r["params"][j, k]) for k in range(r["K"][j])]
        assert abs(sum(w for w, _, _ in comps) - 1) <= 1e-13
        np.testing.assert_allclose(sum(w * mu for w, mu, _ in comps), m, atol=1e-12 * np.abs(vv).max())
        M2 = sum(w * (Sk + np.outer(mu, mu)) for w, mu, Sk in comps)
        np.testing.assert_allclose(M2 - np.outer(m, m), S, atol=1e-12 * np.abs(S).max())


def test_one_gaussian_is_the_closed_form():
    wl = workloads.with_weights(workloads.bimaxwellian_1d3v(C=2, ppc=300, seed=46))
    p = dict(wl.params, Kmax=1)
    for j in range(wl.C):
        sl = slice(wl.cell_off[j], wl.cell_off[j + 1])
        vv = wl.v[:, sl].T.astype(np.float64)
        a = wl.alpha[sl]
        r = oracle.std_cell(p, vv, a, cell=j, penalised=True)
        N = vv.shape[0]
        m = (a[:, None] * vv).sum(0) / a.sum()
        S = ((a[:, None] * (vv - m)).T @ (vv - m)) / a.sum()
        assert r["K"] == 1
        np.testing.assert_allclose(r["params"][0, 1:4], m, rtol=1e-13, atol=1e-15)
        L = -0.5 * N * (3 * math.log(2 * math.pi) + np.linalg.slogdet(S)[1] + 3)
        assert abs(r["lnL"] - L) <= 1e-10 * abs(L)


def test_separated_beams_are_covered_with_their_shares():
    """Three narrow, far-apart beams from Kmax = 8 random particles.  The
    penalised weights annihilate components that own fewer than T/2
    particles (never all of them), and the final unpenalised step gives
    omega_k = N_k / N: every component of weight >= 1 % sits on a beam, and
    the weights on each beam add up to its share of the particles (the
    responsibilities across beams are below 1e-100).  Unlike the
    component-wise schedule, simultaneous updates let several components
    share a beam, each with far more than T/2 particles, so K need not end
    at 3."""
    rng = np.random.default_rng(47)
    centres = np.array([-3.0, 0.0, 2.5])
    shares = np.array([0.5, 0.3, 0.2])
    for cell in range(8):
        n = (2000 * shares).astype(int)
        vv = np.concatenate([rng.normal(c, 0.05, m) for c, m in zip(centres, n)])[:, None]
        p = dict(D=1, Kmax=8, shape_order=2, tol=1e-6, max_sweeps=1000, seed=3, L=1.0, q=1.0)
        r = oracle.std_cell(p, vv, np.ones(vv.shape[0]), cell=cell, penalised=True)
        K = r["K"]
        assert 3 <= K < 8
        mus = r["params"][:K, 1]
        ws = r["params"][:K, 0]
        beam = np.argmin(np.abs(mus[:, None] - centres[None, :]), axis=1)
        big = ws >= 0.01
        assert np.all(np.abs(mus[big] - centres[beam[big]]) <= 0.1)
        np.testing.assert_allclose(np.bincount(beam, weights=ws, minlength=3), shares, atol=1e-9)
