"""Pins of the FP64 oracle to things other than itself: closed forms the paper
derives, textbook special cases, library routines (scipy/numpy), brute force
on tiny inputs and invariants.  CPU only."""
import json
import math
import os

import numpy as np
import pytest
from scipy import interpolate, stats

import oracle
import workloads

HERE = os.path.dirname(os.path.abspath(__file__))


def _params(D, Kmax, **kw):
    p = workloads.method_params(D, Kmax, 2, 1.0)
    p.update(kw)
    return p


def _wmoments(vv, a):
    """textbook weighted mean / biased covariance (numpy)"""
    mean = np.average(vv, axis=0, weights=a)
    cov = np.atleast_2d(np.cov(vv.T, aweights=a, bias=True))
    return mean, cov


def _unpack(prm, D):
    w = prm[0]
    mu = prm[1:1 + D]
    S = np.zeros((D, D))
    t = 1 + D
    for i in range(D):
        for j in range(i, D):
            S[i, j] = S[j, i] = prm[t]
            t += 1
    return w, mu, S


# --------------------------------------------------------------------------
# Philox4x32-10 and the uniform map
# --------------------------------------------------------------------------
def test_uniform52_range_and_resolution():
    # (m + 1/2) 2^-52 with m the 52 high bits: extremes are 2^-53 and 1 - 2^-53
    assert oracle.uniform52(0, 0) == 2.0 ** -53
    assert oracle.uniform52(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert oracle.uniform52(0x80000000, 0) == 0.5 + 2.0 ** -53
    # the 12 low bits of the second word are dropped
    assert oracle.uniform52(7, 0xFFF) == oracle.uniform52(7, 0)


def _curand():
    import ctypes as ct
    import ctypes.util
    cands = [ctypes.util.find_library("curand")]
    for root in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if root:
            cands += [os.path.join(root, "lib64", "libcurand.so"),
                      os.path.join(root, "lib", "libcurand.so")]
    for c in cands:
        if not c:
            continue
        try:
            return ct.CDLL(c)
        except OSError:
            continue
    return None


def test_philox_matches_curand_host_generator():
    # The oracle's Philox4x32-10 (Salmon et al., SC'11) against cuRAND's host
    # generator of the same name, called through its public API on the CPU:
    # with a 64-bit seed its output block t (4 words) is the bijection at
    # counter (0, 0, t, 0) under the key (low, high) words of the seed.
    import ctypes as ct
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not found")
    philox_rng = 161  # CURAND_RNG_PSEUDO_PHILOX4_32_10
    nb = 4096
    for seed in (0x0123456789ABCDEF, 1, 20071227, 0xFFFFFFFF00000001):
        gen = ct.c_void_p()
        assert lib.curandCreateGeneratorHost(ct.byref(gen), philox_rng) == 0
        try:
            assert lib.curandSetPseudoRandomGeneratorSeed(gen, ct.c_ulonglong(seed)) == 0
            buf = np.zeros(4 * nb, dtype=np.uint32)
            assert lib.curandGenerate(gen, buf.ctypes.data_as(ct.c_void_p), ct.c_size_t(buf.size)) == 0
        finally:
            lib.curandDestroyGenerator(gen)
        key = (seed & 0xFFFFFFFF, seed >> 32)
        for t, block in enumerate(buf.reshape(nb, 4)):
            np.testing.assert_array_equal(oracle.philox((0, 0, t, 0), key), block)


def test_philox_statistics():
    key = np.array([0x12345678, 0x9ABCDEF0], np.uint32)
    words = np.array([oracle.philox([i, 3, 5, 0], key) for i in range(20000)])
    bits = np.unpackbits(words.view(np.uint8))
    assert abs(bits.mean() - 0.5) < 0.003
    # byte histogram chi-square (255 dof)
    h = np.bincount(words.view(np.uint8).ravel(), minlength=256)
    e = h.sum() / 256
    chi2 = ((h - e) ** 2 / e).sum()
    assert stats.chi2.sf(chi2, 255) > 1e-4
    # avalanche: one flipped counter bit changes about half the output bits
    base = oracle.philox([0, 0, 0, 0], key)
    flips = []
    for b in range(32):
        o = oracle.philox([1 << b, 0, 0, 0], key)
        flips.append(np.unpackbits((o ^ base).view(np.uint8)).sum())
    assert 48 < np.mean(flips) < 80
    # distinct keys give unrelated streams
    o2 = np.array([oracle.philox([i, 3, 5, 0], key + 1) for i in range(64)])
    assert not np.any(o2 == words[:64])


# --------------------------------------------------------------------------
# Shape functions and deposition (Sec. 2.4.1)
# --------------------------------------------------------------------------
def test_shape_functions_match_scipy_bsplines():
    b1 = interpolate.BSpline.basis_element([-1.0, 0.0, 1.0], extrapolate=False)
    b2 = interpolate.BSpline.basis_element([-1.5, -0.5, 0.5, 1.5], extrapolate=False)
    for s in np.linspace(-1.7, 1.7, 341):
        e1 = np.nan_to_num(b1(s))
        e2 = np.nan_to_num(b2(s))
        assert abs(oracle.shape(1, s) - e1) < 1e-14
        assert abs(oracle.shape(2, s) - e2) < 1e-14
    # partition of unity over integer shifts
    for s in np.linspace(-0.5, 0.5, 11):
        for order in (1, 2):
            tot = sum(oracle.shape(order, s + i) for i in range(-3, 4))
            assert abs(tot - 1.0) < 1e-14


@pytest.mark.parametrize("order,xi,expect", [
    (1, 0.5, (0.0, 1.0, 0.0)),       # CIC at the cell centre
    (1, 0.0, (0.5, 0.5, 0.0)),       # CIC at the left face
    (1, 0.75, (0.0, 0.75, 0.25)),
    (2, 0.5, (0.125, 0.75, 0.125)),  # S2 at the centre
    (2, 0.0, (0.5, 0.5, 0.0)),       # S2 at the left face
    (2, 0.25, (0.28125, 0.6875, 0.03125)),
])
def test_deposit_single_particle_by_hand(order, xi, expect):
    # one particle in cell 0 of a 5-cell periodic mesh, dx = 2: the left
    # neighbour of node 0 is node 4 (periodic wrap)
    C, dx = 5, 2.0
    p = workloads.method_params(1, 1, order, C * dx)
    cell_off = np.array([0, 1, 1, 1, 1, 1])
    x = np.array([xi * dx])
    m = oracle.moments(p, cell_off, x, np.zeros((1, 1)), np.array([3.0]))
    rho = m["rho"] * dx / 3.0
    assert rho[4] == pytest.approx(expect[0], abs=1e-14)
    assert rho[0] == pytest.approx(expect[1], abs=1e-14)
    assert rho[1] == pytest.approx(expect[2], abs=1e-14)
    assert np.abs(rho[2:4]).max() < 1e-15


@pytest.mark.parametrize("D", [1, 3])
def test_moments_of_particles_and_of_mixtures_match_numpy(D):
    # the moments the conservation checks compare (Sec. 2.3.1, 2.4.2):
    # W = sum alpha, p = sum alpha v, M2 = sum alpha v v^T (upper triangle,
    # row-major), E = sum alpha |v|^2 / 2; of a mixture with total weight W:
    # p = W sum w_k mu_k, M2 = W sum w_k (Sigma_k + mu_k mu_k^T), E = tr M2 / 2
    rng = np.random.default_rng(90 + D)
    counts = np.array([0, 1, 17, 250, 40])
    C = counts.shape[0]
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    n = int(off[-1])
    v = rng.standard_normal((D, n)) * 0.3 + 0.1
    a = rng.uniform(0.5, 1.5, n)
    x = (np.repeat(np.arange(C), counts) + rng.random(n)) * 1.0
    p = workloads.method_params(D, 3, 2, float(C))
    m = oracle.moments(p, off, x, v, a)
    iu = np.triu_indices(D)
    for j in range(C):
        sl = slice(off[j], off[j + 1])
        vj, aj = v[:, sl], a[sl]
        assert m["W"][j] == pytest.approx(aj.sum(), rel=1e-14, abs=1e-300)
        np.testing.assert_allclose(m["p"][j], (aj * vj).sum(1), rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(m["M2"][j], ((aj * vj) @ vj.T)[iu], rtol=1e-13, atol=1e-15)
        assert m["E"][j] == pytest.approx(0.5 * (aj * vj ** 2).sum(), rel=1e-13, abs=1e-300)
    # mixtures
    K = np.array([0, 1, 2, 3, 3], dtype=np.int32)
    prm = np.zeros((C, 3, 1 + D + len(iu[0])))
    W = rng.uniform(1.0, 5.0, C)
    comps = {}
    for j in range(C):
        w = rng.dirichlet(np.ones(K[j])) if K[j] else np.zeros(0)
        for k in range(K[j]):
            mu = rng.standard_normal(D)
            A = rng.standard_normal((D, D))
            S = A @ A.T + 0.1 * np.eye(D)
            prm[j, k] = np.concatenate([[w[k]], mu, S[iu]])
            comps.setdefault(j, []).append((w[k], mu, S))
    mm = oracle.mixture_moments(p, K, prm, W)
    for j in range(C):
        if not K[j]:
            continue
        pe = W[j] * sum(w * mu for w, mu, _ in comps[j])
        M2 = W[j] * sum(w * (S + np.outer(mu, mu)) for w, mu, S in comps[j])
        assert mm["W"][j] == pytest.approx(W[j], rel=1e-15)
        np.testing.assert_allclose(mm["p"][j], pe, rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(mm["M2"][j], M2[iu], rtol=1e-13, atol=1e-15)
        assert mm["E"][j] == pytest.approx(0.5 * np.trace(M2), rel=1e-13)


@pytest.mark.parametrize("D,K", [(1, 1), (1, 4), (3, 2), (3, 5)])
def test_penalised_L_against_scipy(D, K):
    # eq. (lnL-GM): sum_p ah_p ln sum_k w_k f_k(v_p) - (d/2) ln N
    # - (T/2) sum_k ln w_k with T = D (D + 3) / 2, d = K (T + 1) - 1, the
    # densities from scipy
    rng = np.random.default_rng(7 * D + K)
    N = 120
    vv = rng.standard_normal((N, D))
    ah = rng.uniform(0.5, 1.5, N)
    ah *= N / ah.sum()
    iu = np.triu_indices(D)
    w = rng.dirichlet(np.ones(K))
    rows, dens = [], np.zeros(N)
    for k in range(K):
        mu = rng.standard_normal(D) * 0.5
        A = rng.standard_normal((D, D))
        S = A @ A.T + 0.3 * np.eye(D)
        rows.append(np.concatenate([[w[k]], mu, S[iu]]))
        dens += w[k] * stats.multivariate_normal(mean=mu, cov=S).pdf(vv).reshape(-1)
    T = D * (D + 3) / 2
    ref = np.sum(ah * np.log(dens)) - (K * (T + 1) - 1) / 2 * math.log(N) - T / 2 * np.log(w).sum()
    assert oracle.penalised_L(D, np.stack(rows), vv, ah) == pytest.approx(ref, rel=1e-12)


def test_deposit_conserves_total_charge():
    wl = workloads.with_weights(workloads.mixture_1d1v(C=16, mean_n=50, clip=(5, 100)))
    m = oracle.moments(wl.params, wl.cell_off, wl.x, wl.v, wl.alpha)
    dx = wl.params["L"] / wl.C
    assert m["rho"].sum() * dx == pytest.approx(wl.alpha.sum(), rel=1e-13)


# --------------------------------------------------------------------------
# Compression (Sec. 2.2-2.3)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("D", [1, 3])
def test_single_component_is_weighted_sample_moments(D):
    # K = 1: eqs. (muk), (sigmak) with gamma_p1 = alpha_p are the weighted
    # sample mean and the biased covariance
    rng = np.random.default_rng(11 + D)
    N = 300
    vv = rng.standard_normal((N, D)) @ np.triu(rng.uniform(0.2, 1.0, (D, D))) + 0.3
    a = rng.uniform(0.5, 2.0, N)
    r = oracle.em_cell(_params(D, 1), vv, a)
    assert r["K"] == 1
    w, mu, S = _unpack(r["params"][0], D)
    mean, cov = _wmoments(vv, a)
    assert w == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_allclose(mu, mean, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(S, cov, rtol=1e-12, atol=1e-14)
    assert r["W"] == pytest.approx(a.sum(), rel=1e-14)
    # closed form of eq. (lnL-GM) at the ML Gaussian: the quadratic terms sum
    # to N*D, so L = -N/2 (D ln 2pi + ln|Sigma| + D) - (T/2) ln N   (d = T)
    T = D * (D + 3) / 2
    Lc = -N / 2 * (D * math.log(2 * math.pi) + math.log(np.linalg.det(cov)) + D) \
        - T / 2 * math.log(N)
    assert r["lnL"] == pytest.approx(Lc, rel=1e-12)


@pytest.mark.parametrize("D,Kmax,N", [(1, 3, 8), (1, 6, 8), (3, 2, 20)])
def test_lnL_brute_force_small_cells(D, Kmax, N):
    # eq. (lnL-GM) recomputed by a direct double loop with scipy densities
    rng = np.random.default_rng(5 + N + Kmax)
    for trial in range(4):
        vv = np.concatenate([rng.normal(-1, 0.3, (N // 2, D)), rng.normal(1, 0.5, (N - N // 2, D))])
        a = rng.uniform(0.5, 1.5, N)
        r = oracle.em_cell(_params(D, Kmax, seed=trial), vv, a, cell=trial)
        K = r["K"]
        ah = a * N / a.sum()
        s = 0.0
        for p in range(N):
            f = 0.0
            for k in range(K):
                w, mu, S = _unpack(r["params"][k], D)
                f += w * stats.multivariate_normal(mean=mu, cov=S).pdf(vv[p])
            s += ah[p] * math.log(f)
        T = D * (D + 3) / 2
        d = K * (T + 1) - 1
        pen = sum(math.log(r["params"][k][0]) for k in range(K))
        L = s - d / 2 * math.log(N) - T / 2 * pen
        assert r["lnL"] == pytest.approx(L, rel=1e-11, abs=1e-11)


@pytest.mark.parametrize("D", [1, 3])
def test_final_step_conserves_mass_mean_covariance(D):
    # Sec. 2.3.1: after the unpenalised step, sum w_k mu_k = sample mean and
    # sum w_k (Sigma_k + mu_k mu_k^T) - mean mean^T = sample covariance
    wl = workloads.with_weights(
        workloads.mixture_1d1v(C=6, mean_n=400, clip=(100, 800)) if D == 1
        else workloads.bimaxwellian_1d3v(C=4, ppc=300))
    out = oracle.compress(wl.params, wl.cell_off, wl.x, wl.v, wl.alpha)
    for j in range(wl.C):
        sl = slice(wl.cell_off[j], wl.cell_off[j + 1])
        vv = wl.v[:, sl].T.astype(np.float64)
        a = wl.alpha[sl]
        mean, cov = _wmoments(vv, a)
        K = out["K"][j]
        mm = np.zeros(D)
        m2 = np.zeros((D, D))
        ws = 0.0
        for k in range(K):
            w, mu, S = _unpack(out["params"][j, k], D)
            ws += w
            mm += w * mu
            m2 += w * (S + np.outer(mu, mu))
        assert ws == pytest.approx(1.0, abs=1e-14)
        np.testing.assert_allclose(mm, mean, rtol=0, atol=1e-13 * (1 + np.abs(mean).max()))
        scale = np.abs(cov).max() + np.abs(mean).max() ** 2
        np.testing.assert_allclose(m2 - np.outer(mean, mean), cov, rtol=0, atol=1e-12 * scale)
        assert out["W"][j] == pytest.approx(a.sum(), rel=1e-14)


def test_component_wise_schedule_one_sweep():
    # Sec. 2.3 steps 1-3: component k's E-step sees the *updated* parameters
    # of components < k.  Recomputed here with scipy densities for one sweep.
    rng = np.random.default_rng(3)
    N, D = 60, 1
    vv = np.concatenate([rng.normal(-1, 0.4, 30), rng.normal(1.2, 0.3, 30)])[:, None]
    a = rng.uniform(0.5, 1.5, N)
    ah = a * N / a.sum()
    init = np.array([[0.3, -0.5, 0.5], [0.3, 0.4, 0.6], [0.4, 1.5, 0.2]])
    r = oracle.em_cell(_params(1, 3), vv, a, init_params=init, only_sweeps=1)
    comps = [list(c) for c in init]
    T = 2.0
    for k in range(3):
        dens = np.array([c[0] * stats.norm(c[1], math.sqrt(c[2])).pdf(vv[:, 0]) for c in comps])
        g = ah * dens[k] / dens.sum(axis=0)
        Nk = g.sum()
        mu = (g * vv[:, 0]).sum() / Nk
        var = (g * (vv[:, 0] - mu) ** 2).sum() / Nk
        comps[k] = [(Nk - T / 2) / (N - T * 3 / 2), mu, var]
        s = sum(c[0] for c in comps)
        for c in comps:
            c[0] /= s
    assert r["K"] == 3
    np.testing.assert_allclose(r["params"][:3], np.array(comps), rtol=1e-12, atol=1e-14)


def test_far_component_is_annihilated():
    # a component far from every particle gets N_k ~ 0 <= T/2 and is removed
    # (eq. omegak); the survivor is then the K = 1 textbook fit
    rng = np.random.default_rng(8)
    vv = rng.normal(0.0, 1.0, (500, 1))
    a = np.ones(500)
    init = np.array([[0.5, 0.0, 1.0], [0.5, 80.0, 1.0]])
    r = oracle.em_cell(_params(1, 2), vv, a, init_params=init, only_sweeps=1, trace_cap=4)
    assert r["K"] == 1
    assert r["Ktrace"][-1] < 0  # the sweep removed a component
    r2 = oracle.em_cell(_params(1, 2), vv, a, init_params=init)
    w, mu, S = _unpack(r2["params"][0], 1)
    mean, cov = _wmoments(vv, a)
    assert r2["K"] == 1 and mu[0] == pytest.approx(mean[0], abs=1e-14)
    assert S[0, 0] == pytest.approx(cov[0, 0], rel=1e-13)


def test_well_separated_beams_split_by_beam():
    # two beams 40 thermal widths apart: responsibilities are 0/1 between
    # the beams to double precision, so the components of each beam carry
    # exactly that beam's mass, mean and variance (the hard split)
    for seed in range(3):
        rng = np.random.default_rng(100 + seed)
        n1, n2 = 700, 1300
        v1 = rng.normal(-1.0, 0.05, n1)
        v2 = rng.normal(1.0, 0.05, n2)
        vv = np.concatenate([v1, v2])[:, None]
        r = oracle.em_cell(_params(1, 8, seed=seed), vv, np.ones(n1 + n2), cell=seed)
        assert r["K"] >= 2
        comps = [_unpack(r["params"][k], 1) for k in range(r["K"])]
        for sgn, vb, nb in ((-1, v1, n1), (1, v2, n2)):
            grp = [c for c in comps if np.sign(c[1][0]) == sgn]
            w = sum(c[0] for c in grp)
            m1 = sum(c[0] * c[1][0] for c in grp) / w
            m2 = sum(c[0] * (c[2][0, 0] + c[1][0] ** 2) for c in grp) / w
            assert w == pytest.approx(nb / (n1 + n2), rel=1e-12)
            assert m1 == pytest.approx(vb.mean(), rel=1e-12)
            assert m2 - m1 ** 2 == pytest.approx(vb.var(), rel=1e-9)
    # with one initial component per beam the fit is exactly two components
    init = np.array([[0.5, -0.9, 0.01], [0.5, 0.9, 0.01]])
    r = oracle.em_cell(_params(1, 2), vv, np.ones(n1 + n2), init_params=init)
    assert r["K"] == 2
    assert r["params"][0][1] == pytest.approx(v1.mean(), rel=1e-12)
    assert r["params"][1][2] == pytest.approx(v2.var(), rel=1e-10)


def test_single_3v_maxwellian_collapses_to_one_component():
    # in 3V the MML penalty (T/2 = 4.5 particles per component) removes the
    # redundant components of a single anisotropic Maxwellian at 128
    # particles per cell; more particles keep more components (the trend of
    # Sec. 3.2: 1.8, 2.1, 3.3 Gaussians for 128, 512, 1024 particles)
    kbar = []
    for ppc in (128, 1024):
        ks = []
        for seed in range(6):
            wl = workloads.bimaxwellian_1d3v(C=1, ppc=ppc, seed=300 + seed)
            ks.append(oracle.em_cell(wl.params, wl.v.T, wl.alpha, cell=seed)["K"])
        kbar.append(np.mean(ks))
        if ppc == 128:
            assert sum(k == 1 for k in ks) >= 5, ks
    assert kbar[1] >= kbar[0]


def test_stopping_rule_is_the_first_quiet_sweep():
    # Sec. 2.3 step 4 with readings 2 and 5: after each sweep, stop when the
    # relative change of the penalised L is within tol AND the sweep removed
    # no component; the trace (L and K after initialisation and after each
    # sweep, K negative for a removing sweep) must stop at the first such
    # sweep, K must never grow, and K0 = Kmax for these cells (N >> Kmax).
    wl = workloads.with_weights(workloads.mixture_1d1v(C=10, mean_n=400, clip=(100, 800), seed=71))
    tol = wl.params["tol"]
    for j in range(wl.C):
        sl = slice(wl.cell_off[j], wl.cell_off[j + 1])
        r = oracle.em_cell(dict(wl.params), wl.v[:, sl].T, wl.alpha[sl], cell=j, trace_cap=2000)
        L, Kt = r["Ltrace"], r["Ktrace"]
        S = r["sweeps"]
        assert r["status"] & oracle.ST_EM_MAXSWEEPS == 0
        assert L.shape[0] == S + 1 and Kt[0] == wl.params["Kmax"]
        quiet = [Kt[s] > 0 and abs(L[s] - L[s - 1]) <= tol * abs(L[s - 1]) for s in range(1, S + 1)]
        assert quiet[-1] and not any(quiet[:-1]), j
        assert np.all(np.diff(np.abs(Kt)) <= 0)
        assert abs(r["K"]) == abs(Kt[-1]) or r["status"] & oracle.ST_COV_NOT_PD


def test_L_nondecreasing_between_removals():
    # the component-wise EM is a generalised EM for eq. (lnL-GM): L does not
    # decrease over a sweep that removes nothing
    wl = workloads.mixture_1d1v(C=3, mean_n=500, clip=(100, 900))
    for j in range(wl.C):
        sl = slice(wl.cell_off[j], wl.cell_off[j + 1])
        r = oracle.em_cell(wl.params, wl.v[:, sl].T, wl.alpha[sl], cell=j, trace_cap=1200)
        L, Kt = r["Ltrace"], r["Ktrace"]
        clean = Kt[1:] > 0
        d = np.diff(L)[clean]
        assert (d >= -1e-9 * np.abs(L[1:][clean])).all()


@pytest.mark.parametrize("D,Kmax,N,K0", [
    # hand-computed: T = D (D + 3) / 2; K0 = the largest K <= min(Kmax, N)
    # with N - T K / 2 > 0 (a component must be able to survive eq. omegak),
    # at least 1
    (1, 8, 3, 2),    # T = 2: 3 - K > 0 -> K <= 2
    (1, 8, 8, 7),    # 8 - K > 0 -> K <= 7
    (1, 8, 12, 8),   # Kmax binds
    (3, 10, 4, 1),   # T = 9: 4 - 4.5 K > 0 fails for K = 1: floor of 1
    (3, 10, 9, 1),   # 9 - 4.5 K > 0 -> K < 2 (a tie removes)
    (3, 10, 10, 2),  # K < 2.22
    (3, 10, 14, 3),  # K < 3.11
])
def test_initial_component_count_for_small_cells(D, Kmax, N, K0):
    rng = np.random.default_rng(N + 10 * D)
    vv = rng.standard_normal((N, D))
    r = oracle.em_cell(_params(D, Kmax), vv, np.ones(N), trace_cap=8)
    assert r["Ktrace"][0] == K0


def test_collapsed_component_is_removed_at_the_covariance_floor():
    # Reading 11: no regularisation; a component whose covariance fails the
    # Cholesky floor in a sweep is removed and COV_NOT_PD is set.  30
    # particles share one velocity far from a normal bulk; a supplied
    # component sitting on them (covariance 1e-4 I) gets responsibility
    # exactly 0 from the bulk, so its M-step covariance is exactly 0.
    D = 3
    rng = np.random.default_rng(81)
    vv = np.concatenate([rng.standard_normal((200, D)), np.tile([0.0, 0.0, 5.0], (30, 1))])
    al = np.ones(vv.shape[0])
    iu = np.triu_indices(D)
    init = np.stack([np.concatenate([[0.87], np.zeros(D), np.eye(D)[iu]]),
                     np.concatenate([[0.13], [0.0, 0.0, 5.0], 1e-4 * np.eye(D)[iu]])])
    p = _params(D, 4)
    r1 = oracle.em_cell(p, vv, al, init_params=init, only_sweeps=1, trace_cap=8)
    assert r1["K"] == 1 and r1["status"] & oracle.ST_COV_NOT_PD
    assert list(r1["Ktrace"]) == [2, -1]
    r = oracle.em_cell(p, vv, al, init_params=init)
    assert r["K"] == 1 and r["status"] & oracle.ST_COV_NOT_PD
    w, mu, S = r["params"][0][0], r["params"][0][1:1 + D], r["params"][0][1 + D:]
    assert w == pytest.approx(1.0, rel=1e-14)
    np.testing.assert_allclose(mu, vv.mean(0), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(S, np.cov(vv.T, bias=True)[iu], rtol=1e-11, atol=1e-14)
    # the standard EM of Sec. 4 and its simultaneous penalised variant drop
    # the component the same way
    for penalised in (False, True):
        rs = oracle.std_cell(dict(p, max_sweeps=50), vv, al, init=2, init_params=init,
                             penalised=penalised)
        assert rs["K"] == 1 and rs["status"] & oracle.ST_COV_NOT_PD, penalised
        np.testing.assert_allclose(rs["params"][0][1:1 + D], vv.mean(0), rtol=1e-12, atol=1e-14)


def test_degenerate_cell():
    vv = np.full((20, 1), 0.25)
    r = oracle.em_cell(_params(1, 4), vv, np.ones(20))
    assert r["K"] == 1 and r["status"] & oracle.ST_DEGENERATE
    assert r["params"][0][1] == pytest.approx(0.25)
    r0 = oracle.em_cell(_params(1, 4), np.zeros((0, 1)), np.zeros(0))
    assert r0["K"] == 0 and r0["status"] & oracle.ST_EMPTY


# --------------------------------------------------------------------------
# Mass-matrix solve (Sec. 2.4.1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [3, 4, 7, 64])
def test_cyclic_tridiagonal_matches_dense_solve(n):
    rng = np.random.default_rng(n)
    a = rng.uniform(0.05, 0.3, n)
    c = rng.uniform(0.05, 0.3, n)
    b = rng.uniform(0.8, 1.2, n) + a + c
    d = rng.standard_normal(n)
    A = np.zeros((n, n))
    for i in range(n):
        A[i, (i - 1) % n] += a[i]
        A[i, i] += b[i]
        A[i, (i + 1) % n] += c[i]
    x = oracle.cyclic_tridiag(a, b, c, d)
    np.testing.assert_allclose(x, np.linalg.solve(A, d), rtol=1e-12, atol=1e-14)


# --------------------------------------------------------------------------
# Reconstruction (Sec. 2.4)
# --------------------------------------------------------------------------
def _roundtrip(wl, nthreads=4):
    out = oracle.compress(wl.params, wl.cell_off, wl.x, wl.v, wl.alpha, nthreads=nthreads)
    rec = oracle.reconstruct(wl.params, out["K"], out["params"], out["W"], out["rho_target"],
                             wl.cell_off, nthreads=nthreads, want_raw=True)
    return out, rec


@pytest.mark.parametrize("which", ["two_stream_s1", "mixture_s2", "bimax3v"])
def test_reconstruction_conserves_charge_momentum_energy(which):
    if which == "two_stream_s1":
        wl = workloads.two_stream_1d1v(C=8, ppc=256)
    elif which == "mixture_s2":
        wl = workloads.mixture_1d1v(C=12, mean_n=300, clip=(50, 600))
    else:
        wl = workloads.bimaxwellian_1d3v(C=6, ppc=300)
    out, rec = _roundtrip(wl)
    skipped = (rec["status"] & oracle.ST_PROJ_SKIPPED) != 0
    assert skipped.mean() < 0.25
    m0 = oracle.moments(wl.params, wl.cell_off, wl.x, wl.v, wl.alpha)
    m1 = oracle.moments(wl.params, wl.cell_off, rec["x"], rec["v"], rec["alpha"])
    # Gauss' law: the corrected weights reproduce the stored density on
    # every node
    np.testing.assert_allclose(m1["rho"], out["rho_target"], rtol=0,
                               atol=1e-12 * np.abs(out["rho_target"]).max())
    # momentum and energy of every projected cell equal the original
    # particles'; a skipped cell (Sec. 2.4.2 failure mode) keeps its samples
    for j in range(wl.C):
        sl = slice(wl.cell_off[j], wl.cell_off[j + 1])
        if skipped[j]:
            np.testing.assert_array_equal(rec["v"][:, sl], rec["v_raw"][:, sl])
            continue
        pabs = (wl.alpha[sl] * np.abs(wl.v[:, sl].astype(np.float64))).sum()
        assert np.abs(m1["p"][j] - m0["p"][j]).max() <= 1e-12 * pabs
        assert abs(m1["E"][j] - m0["E"][j]) <= 1e-12 * m0["E"][j]
    # positions stay in their cells
    dx = wl.params["L"] / wl.C
    cell = np.repeat(np.arange(wl.C), np.diff(wl.cell_off))
    assert np.all(rec["x"] >= cell * dx) and np.all(rec["x"] < (cell + 1) * dx)


@pytest.mark.parametrize("order", [1, 2])
def test_gauss_correction_is_the_mass_matrix_equation(order):
    # Sec. 2.4.1, eqs. (p-weight-correction), (new-p-weight): every resampled
    # particle of cell j gets the same dA_j, and dA solves M dA = dx (rho' -
    # rho) with M_ij = q sum_{p in j} S(x_i - x_p).  M, rho and the residual
    # are built here from scipy's B-spline basis and a dense product.
    wl = workloads.mixture_1d1v(C=12, mean_n=300, clip=(50, 600), seed=23, shape_order=order)
    p = dict(wl.params, q=-0.8)
    out = oracle.compress(p, wl.cell_off, wl.x, wl.v, wl.alpha, nthreads=4)
    rec = oracle.reconstruct(p, out["K"], out["params"], out["W"], out["rho_target"], wl.cell_off,
                             nthreads=4)
    C, L, q = wl.C, p["L"], p["q"]
    dx = L / C
    knots = [-1.0, 0.0, 1.0] if order == 1 else [-1.5, -0.5, 0.5, 1.5]
    S = interpolate.BSpline.basis_element(knots, extrapolate=False)
    M = np.zeros((C, C))
    for j in range(C):
        a, b = wl.cell_off[j], wl.cell_off[j + 1]
        base = out["W"][j] / (b - a)
        # one shift per cell
        np.testing.assert_allclose(rec["alpha"][a:b] - base, rec["dA"][j], rtol=0,
                                   atol=1e-13 * base)
        for i in range(C):
            d = ((i + 0.5) * dx - rec["x"][a:b] + L / 2) % L - L / 2
            M[i, j] = q * np.nan_to_num(S(d / dx)).sum()
        # partition of unity: a column sums to q N'_j
        assert M[:, j].sum() == pytest.approx(q * (b - a), rel=1e-13)
    n_out = np.diff(wl.cell_off)
    rho_raw = M @ (out["W"] / n_out) / dx
    rhs = dx * (out["rho_target"] - rho_raw)
    res = M @ rec["dA"] - rhs
    assert np.abs(res).max() <= 1e-12 * dx * np.abs(out["rho_target"]).max()
    assert np.abs(rhs).max() > 1e-6 * dx * np.abs(out["rho_target"]).max()  # not trivial


def test_projection_is_one_scalar_affine_map_per_cell():
    # Sec. 2.4.2, eqs. (alpha), (beta): a projected cell's velocities are
    # v' = a (v + beta) with ONE scalar a > 0 for all D axes and a vector
    # beta.  With the conservation of momentum and energy (tested above),
    # that form fixes a and beta uniquely; a per-axis scaling would also
    # conserve both and is excluded here.
    wl = workloads.with_weights(workloads.bimaxwellian_1d3v(C=6, ppc=300))
    out, rec = _roundtrip(wl)
    done = 0
    for j in range(wl.C):
        if rec["status"][j] & oracle.ST_PROJ_SKIPPED:
            continue
        sl = slice(wl.cell_off[j], wl.cell_off[j + 1])
        u, w = rec["v_raw"][:, sl], rec["v"][:, sl]
        slopes = []
        for d in range(wl.D):
            A = np.stack([u[d], np.ones(u.shape[1])], axis=1)
            coef, *_ = np.linalg.lstsq(A, w[d], rcond=None)
            resid = w[d] - A @ coef
            assert np.abs(resid).max() <= 1e-12 * np.abs(w[d]).max(), (j, d)
            slopes.append(coef[0])
        slopes = np.array(slopes)
        assert slopes.min() > 0
        np.testing.assert_allclose(slopes, slopes[0], rtol=1e-12)
        done += 1
    assert done >= 4


def test_sampling_matches_mixture_distribution():
    # ancestral sampling, eq. (mix-dist-1): the raw samples of one cell follow
    # the mixture CDF (KS test) and positions are uniform in the cell
    D = 1
    p = workloads.method_params(1, 3, 2, 4.0, recon_seed=9)
    C = 4
    prm = np.zeros((C, 3, 3))
    comps = np.array([[0.2, -0.7, 0.04], [0.5, 0.1, 0.25], [0.3, 1.4, 0.01]])
    prm[:] = comps
    K = np.full(C, 3, np.int32)
    n = 20000
    out_off = np.arange(C + 1, dtype=np.int64) * n
    W = np.full(C, float(n))
    # a target density equal to uniform sampling's expectation keeps dA tiny
    rho_t = np.full(C, float(n))
    rec = oracle.reconstruct(p, K, prm, W, rho_t, out_off, want_raw=True)
    for j in range(C):
        v = rec["v_raw"][0, j * n:(j + 1) * n]
        cdf = lambda t: sum(w * stats.norm(m, math.sqrt(s)).cdf(t) for w, m, s in comps)
        assert stats.kstest(v, cdf).pvalue > 1e-3
        xs = rec["x"][j * n:(j + 1) * n] - j * 1.0
        assert stats.kstest(xs, "uniform").pvalue > 1e-3


def test_sampling_3v_covariance():
    p = workloads.method_params(3, 2, 2, 2.0, recon_seed=4)
    C, n = 2, 40000
    S1 = np.array([[0.04, 0.01, 0.0], [0.01, 0.09, -0.02], [0.0, -0.02, 0.16]])
    S2 = np.diag([0.01, 0.25, 0.25])
    mu1, mu2 = np.array([0.1, -0.2, 0.3]), np.array([-0.5, 0.0, 0.2])

    def rec_(w, mu, S):
        return [w, *mu, S[0, 0], S[0, 1], S[0, 2], S[1, 1], S[1, 2], S[2, 2]]
    prm = np.zeros((C, 2, 10))
    prm[:, 0] = rec_(0.35, mu1, S1)
    prm[:, 1] = rec_(0.65, mu2, S2)
    out_off = np.arange(C + 1, dtype=np.int64) * n
    rec = oracle.reconstruct(p, np.full(C, 2, np.int32), prm, np.full(C, float(n)),
                             np.full(C, float(n)), out_off, want_raw=True)
    mean = 0.35 * mu1 + 0.65 * mu2
    cov = 0.35 * (S1 + np.outer(mu1, mu1)) + 0.65 * (S2 + np.outer(mu2, mu2)) - np.outer(mean, mean)
    for j in range(C):
        v = rec["v_raw"][:, j * n:(j + 1) * n]
        se = np.sqrt(np.diag(cov) / n)
        assert np.all(np.abs(v.mean(axis=1) - mean) < 5 * se)
        assert np.abs(np.cov(v, bias=True) - cov).max() < 6 * np.sqrt(2.0 / n) * np.abs(cov).max()


def test_sampling_3v_marginals_are_independent_normals():
    # the 3V Box-Muller draws (two pairs of 32-bit uniforms from one Philox
    # block): with one component of covariance diag(1, 4, 9) each coordinate
    # divided by its standard deviation is N(0, 1) (KS test) and the three
    # are uncorrelated
    p = workloads.method_params(3, 1, 2, 2.0, recon_seed=11)
    C, n = 2, 50000
    prm = np.zeros((C, 1, 10))
    prm[:, 0] = [1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 4.0, 0.0, 9.0]
    out_off = np.arange(C + 1, dtype=np.int64) * n
    rec = oracle.reconstruct(p, np.full(C, 1, np.int32), prm, np.full(C, float(n)),
                             np.full(C, float(n)), out_off, want_raw=True)
    sd = np.array([1.0, 2.0, 3.0])
    for j in range(C):
        y = rec["v_raw"][:, j * n:(j + 1) * n] / sd[:, None]
        for d in range(3):
            assert stats.kstest(y[d], "norm").pvalue > 1e-3, (j, d)
        r = np.corrcoef(y)
        assert np.abs(r - np.eye(3)).max() < 5.0 / math.sqrt(n)


def test_projection_failure_is_skipped_and_flagged():
    # Sec. 2.4.2: a negative numerator 2 E N' - p^2 (a cold drifting cell
    # whose weights the Gauss step lowers) skips the projection
    p = workloads.method_params(1, 1, 2, 3.0, recon_seed=1)
    C, n = 3, 50
    prm = np.zeros((C, 1, 3))
    prm[:, 0] = [1.0, 1.0, 1e-6]
    out_off = np.arange(C + 1, dtype=np.int64) * n
    W = np.full(C, float(n))
    rho_t = np.array([float(n), 0.5 * n, float(n)])
    rec = oracle.reconstruct(p, np.ones(C, np.int32), prm, W, rho_t, out_off, want_raw=True)
    assert rec["status"][1] & oracle.ST_PROJ_SKIPPED
    np.testing.assert_array_equal(rec["v"][:, n:2 * n], rec["v_raw"][:, n:2 * n])


def test_twice_restarted_variable_weights():
    # Sec. 3.2: a second compression of the Gauss-corrected (non-identical
    # weight) particles still conserves exactly
    wl = workloads.mixture_1d1v(C=8, mean_n=300, clip=(100, 500))
    out, rec = _roundtrip(wl)
    wl2 = workloads.Workload("second", wl.cell_off, rec["x"], rec["v"], rec["alpha"], wl.params)
    assert np.ptp(rec["alpha"]) > 0
    out2, rec2 = _roundtrip(wl2)
    m0 = oracle.moments(wl.params, wl.cell_off, wl.x, wl.v, wl.alpha)
    m2 = oracle.moments(wl.params, wl.cell_off, rec2["x"], rec2["v"], rec2["alpha"])
    np.testing.assert_allclose(m2["rho"], out["rho_target"], rtol=1e-11)
    np.testing.assert_allclose(m2["E"], m0["E"], rtol=1e-11)


def test_paper_two_stream_statistics():
    # Sec. 3.1 reports about 2 Gaussians per cell (Kmax = 8, 156 particles
    # per cell) and a compression ratio near 75; a weak, statistical pin
    g = json.load(open(os.path.join(HERE, "golden", "paper_statistics.json")))["two_stream_1d1v"]
    wl = workloads.two_stream_1d1v(C=32, ppc=g["ppc"])
    out = oracle.compress(wl.params, wl.cell_off, wl.x, wl.v, wl.alpha, nthreads=4)
    kbar = out["K"].mean()
    assert g["Kbar_range"][0] <= kbar <= g["Kbar_range"][1]
    cr = g["numbers_per_particle"] * g["ppc"] / (kbar * 3)
    assert g["cr_range"][0] <= cr <= g["cr_range"][1]
