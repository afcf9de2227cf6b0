"""GPU parity of the standard (non-adaptive) EM with K-means initialisation
and Anderson acceleration (gm_compress_standard, Sec. 4) against the FP64
oracle, through the C ABI, on seeded inputs.

Plain standard EM (random or K-means start): a cell agrees when it has
the same component count and its unpenalised log-likelihood is within 1e-5
(relative); the stopping test is knife-edge in the same way as the adaptive
EM's (the FP32 E-step moves the iteration at which the relative change of L
first falls below tol), so a cell that disagrees is rerun in the oracle for
exactly the GPU's number of iterations (tol = 0) and must then agree (or,
if it ran into the iteration cap, be within 200 iterations' worth of the
oracle's own last change of L).

Anderson acceleration extrapolates from differences of successive EM
residuals; near convergence those differences are of the size of the FP32
E-step's rounding, so the GPU and the FP64 oracle take different
extrapolations and their trajectories part.  The extrapolation's own
arithmetic is therefore checked apart from the EM map (gm_anderson_affine
against the oracle on affine maps), and the accelerated EM by what it must
deliver: convergence, the oracle's iteration count, no worse a mean
likelihood than the oracle's accelerated fit, and fewer iterations than the
plain EM on the GPU.  Moments of every output equal the particle moments to
1e-12 (the output is an FP64 standard EM step)."""
import os

import numpy as np
import pytest

import oracle
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


def run_both(gm, wl, init, aa, penalised=False, **cfg_over):
    p = dict(wl.params, **cfg_over)
    cfg = gm.config(p)
    out = gm.gm_compress_standard(cfg, dev(wl.cell_off), dev(wl.x), dev(wl.v), dev(wl.alpha),
                                  init=init, aa_memory=aa, penalised=penalised)
    torch.cuda.synchronize()
    g = {k: t.cpu().numpy() for k, t in out.items()}
    ref = oracle.standard(p, wl.cell_off, wl.x, wl.v, wl.alpha, init=init, aa_memory=aa,
                          nthreads=NTHREADS, penalised=penalised)
    return p, g, ref, out


def agreement(p, g, ref, wl, init, aa, penalised=False, lag_converged=0):
    """(natural agreement, agreement at equal iterations).  A cell that
    disagrees is rerun in the oracle for the GPU's number of iterations; it
    agrees if K is the same and lnL is within 1e-5, or, if it ran into the
    iteration cap, within 200 iterations' worth of the oracle's last change
    of L.  With lag_converged > 0 (the penalised variant, whose slow
    trajectories drift apart in FP32 and FP64 even at equal iterations) a
    converged cell may also be within lag_converged iterations' worth of
    the oracle's own change of the output's lnL between iterations it - 1
    and it."""
    rel = np.abs(g["lnL"] - ref["lnL"]) / np.maximum(np.abs(ref["lnL"]), 1e-300)
    nat = (g["K"] == ref["K"]) & (rel <= 1e-5)
    eq = nat.copy()
    lagged = 0
    for j in np.flatnonzero(~nat):
        sl = slice(wl.cell_off[j], wl.cell_off[j + 1])
        it = max(int(g["iters"][j]), 1)
        run = lambda n: oracle.std_cell(dict(p, tol=0.0, max_sweeps=n), wl.v[:, sl].T, wl.alpha[sl],
                                        cell=j, init=init, aa_memory=aa, trace_cap=n + 2,
                                        penalised=penalised)
        r = run(it)
        diff = abs(g["lnL"][j] - r["lnL"])
        if r["K"] != g["K"][j]:
            continue
        if diff <= 1e-5 * abs(r["lnL"]):
            eq[j] = True
        elif g["status"][j] & oracle.ST_EM_MAXSWEEPS:
            tr = r["Ltrace"]
            dL = abs(tr[-1] - tr[-2]) if tr.shape[0] >= 2 else 0.0
            eq[j] = diff <= 200 * dL
        elif lag_converged > 0 and it > 1:
            r1 = run(it - 1)
            eq[j] = r1["K"] == r["K"] and diff <= lag_converged * abs(r["lnL"] - r1["lnL"])
            lagged += int(eq[j])
    if lagged:
        print(f"  {lagged} converged cell(s) within {lag_converged} iterations of the oracle's trajectory")
    return nat.mean(), eq.mean()


def check_moments(gm, wl, out):
    cfg = gm.config(wl.params)
    m0 = {k: t.cpu().numpy() for k, t in gm.gm_moments(cfg, dev(wl.cell_off), dev(wl.x), dev(wl.v),
                                                          dev(wl.alpha)).items()}
    mm = {k: t.cpu().numpy() for k, t in gm.gm_mixture_moments(cfg, out["K"], out["params"],
                                                                 out["W"]).items()}
    ok = m0["W"] > 0
    np.testing.assert_allclose(mm["W"][ok], m0["W"][ok], rtol=1e-14)
    for j in np.flatnonzero(ok):
        sl = slice(wl.cell_off[j], wl.cell_off[j + 1])
        pabs = (wl.alpha[sl] * np.abs(wl.v[:, sl].astype(np.float64))).sum()
        assert np.abs(mm["p"][j] - m0["p"][j]).max() <= 1e-12 * pabs
        assert abs(mm["E"][j] - m0["E"][j]) <= 1e-12 * m0["E"][j]


def check_accelerated(gm, wl, p, g, ref, init):
    """the accelerated fit: converged, in the oracle's number of
    iterations, no worse than the oracle's accelerated fit in the typical
    cell (median) nor much worse on average, and faster than plain EM from
    the same start on the GPU"""
    conv_g = np.mean((g["status"] & oracle.ST_EM_MAXSWEEPS) == 0)
    conv_o = np.mean((ref["status"] & oracle.ST_EM_MAXSWEEPS) == 0)
    ratio = g["iters"].mean() / ref["iters"].mean()
    rel = (g["lnL"] - ref["lnL"]) / np.abs(ref["lnL"])
    dl = np.mean(rel)
    cfg = gm.config(p)
    plain = gm.gm_compress_standard(cfg, dev(wl.cell_off), dev(wl.x), dev(wl.v), dev(wl.alpha),
                                    init=init, aa_memory=0)
    it_plain = plain["iters"].double().mean().item()
    print(f"  converged GPU {conv_g:.3f} oracle {conv_o:.3f}; iterations GPU {g['iters'].mean():.1f} "
          f"oracle {ref['iters'].mean():.1f} (ratio {ratio:.2f}), plain GPU {it_plain:.1f}; "
          f"mean relative lnL GPU - oracle {dl:+.2e} (median {np.median(rel):+.2e}, "
          f"worse by 1 %: {np.mean(rel < -1e-2):.3f})")
    assert conv_g >= 0.9
    assert 0.6 <= ratio <= 1.6
    # the two sides' extrapolations part (rounding), so single cells land in
    # other local optima: typical cells agree, the mean is not much lower
    assert np.median(rel) >= -1e-4
    assert dl >= -3e-3
    assert np.mean(rel < -1e-2) <= 0.1
    assert g["iters"].mean() < 0.8 * it_plain  # 1V: ~0.15-0.25; 3V, Kmax 10, K-means: ~0.65
    assert g["aa_steps"].sum() > 0


@pytest.mark.parametrize("init,aa", [(0, 0), (1, 0), (0, 5), (1, 5)])
def test_standard_1v_matches_oracle(gm, init, aa):
    wl = workloads.mixture_1d1v(C=64, mean_n=900, clip=(100, 3000), seed=51)
    p, g, ref, out = run_both(gm, wl, init, aa)
    print(f"standard 1V init {init} aa {aa}:")
    if aa == 0:
        nat, eq = agreement(p, g, ref, wl, init, aa)
        print(f"  natural {nat:.3f}, equal iterations {eq:.3f}")
        assert eq >= 0.95 and nat >= 0.5, (nat, eq)
    else:
        check_accelerated(gm, wl, p, g, ref, init)
    np.testing.assert_allclose(g["W"], ref["W"], rtol=1e-13)
    np.testing.assert_allclose(g["rho_target"], ref["rho_target"], rtol=1e-12,
                               atol=1e-13 * np.abs(ref["rho_target"]).max())
    if init == 1:  # Lloyd's decisions are taken on the same FP32 coordinates
        assert np.mean(g["km_passes"] == ref["km_passes"]) >= 0.95
    check_moments(gm, wl, out)


@pytest.mark.parametrize("init,aa", [(0, 0), (1, 5)])
def test_standard_3v_matches_oracle(gm, init, aa):
    wl = workloads.with_weights(workloads.bimaxwellian_1d3v(C=32, ppc=800, seed=52))
    p, g, ref, out = run_both(gm, wl, init, aa)
    print(f"standard 3V init {init} aa {aa}:")
    if aa == 0:
        nat, eq = agreement(p, g, ref, wl, init, aa)
        print(f"  natural {nat:.3f}, equal iterations {eq:.3f}")
        assert eq >= 0.95 and nat >= 0.4, (nat, eq)
    else:
        check_accelerated(gm, wl, p, g, ref, init)
    if init == 1:
        assert np.mean(g["km_passes"] == ref["km_passes"]) >= 0.9
    check_moments(gm, wl, out)


PENALISED_CASES = [("mixture_1d1v", 0), ("bimaxwellian_1d3v", 0), ("bimaxwellian_1d3v", 1),
                   ("two_stream_1d1v", 0)]


@pytest.mark.parametrize("which,init", PENALISED_CASES)
def test_penalised_simultaneous_em_matches_oracle(gm, which, init):
    """The simultaneous penalised EM with annihilation (penalised = 1): K
    and lnL cell by cell, with the equal-iteration rule for the cells that
    stop at another iteration (penalised L in the trace; converged cells
    may lag by 20 iterations of the oracle's own progress); exact
    moments."""
    if which == "mixture_1d1v":
        wl = workloads.mixture_1d1v(C=64, mean_n=900, clip=(100, 3000), seed=51)
    elif which == "bimaxwellian_1d3v":
        wl = workloads.with_weights(workloads.bimaxwellian_1d3v(C=32, ppc=800, seed=52))
    else:
        wl = workloads.two_stream_1d1v()
    p, g, ref, out = run_both(gm, wl, init, 0, penalised=True)
    nat, eq = agreement(p, g, ref, wl, init, 0, penalised=True, lag_converged=20)
    print(f"penalised {which} init {init}: natural {nat:.3f}, equal iterations {eq:.3f}; K GPU "
          f"{g['K'].mean():.2f} oracle {ref['K'].mean():.2f}; iterations GPU {g['iters'].mean():.1f} "
          f"oracle {ref['iters'].mean():.1f}")
    assert eq >= 0.95 and nat >= 0.4, (nat, eq)
    assert abs(g["K"].mean() - ref["K"].mean()) <= 0.1 * ref["K"].mean()
    np.testing.assert_allclose(g["W"], ref["W"], rtol=1e-13)
    check_moments(gm, wl, out)


def test_penalised_keeps_one_component_and_rejects_anderson(gm):
    """A 12-particle cell with Kmax = 8 (1V: T/2 = 1): K0 is lowered to keep
    N - T K0 / 2 > 0 and annihilation leaves at least one component; AA is
    not defined for the penalised variant."""
    counts = np.array([12, 3, 40, 0])
    wl = workloads.mixture_1d1v(C=4, counts=counts, seed=56)
    p, g, ref, out = run_both(gm, wl, 0, 0, penalised=True)
    assert np.all(g["K"][counts > 0] >= 1)
    np.testing.assert_array_equal(g["K"], ref["K"])
    rel = np.abs(g["lnL"] - ref["lnL"]) / np.maximum(np.abs(ref["lnL"]), 1e-300)
    assert np.all(rel[counts > 3] <= 1e-5)
    cfg = gm.config(wl.params)
    with pytest.raises(RuntimeError):
        gm.gm_compress_standard(cfg, dev(wl.cell_off), dev(wl.x), dev(wl.v), dev(wl.alpha),
                                aa_memory=3, penalised=True)


@pytest.mark.parametrize("n,memory", [(6, 6), (24, 3), (160, 8), (40, 0)])
def test_anderson_step_matches_oracle_on_affine_maps(gm, n, memory):
    """The kernel's Anderson step, alone, on G(x) = A x + b: the residual
    norms of the oracle's implementation (FP64 both; the dot products are
    summed in a different order) while they are above 1e-4 of the first;
    below that the least-squares problem is ill-conditioned (its Gram matrix
    squares the conditioning of the residual differences), so the GPU must
    only have converged as far, and its iterate lie within what the final
    residuals allow, |x - x*| <= |r| / (1 - rho(A))."""
    rng = np.random.default_rng(n + memory)
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    A = Q @ np.diag(np.linspace(0.3, 0.9, n)) @ Q.T + 0.005 * rng.standard_normal((n, n))
    b = rng.standard_normal(n)
    x0 = rng.standard_normal(n)
    iters = 14
    xo, ro = oracle.aa_affine(A, b, x0, memory, iters)
    xg, rg = gm.gm_anderson_affine(dev(A), dev(b), dev(x0), memory, iters)
    xg, rg = xg.cpu().numpy(), rg.cpu().numpy()
    well = ro >= 1e-4 * ro[0]
    print(f"n {n} memory {memory}: {well.sum()} well-conditioned steps, max relative residual "
          f"difference {np.max(np.abs(rg[well] - ro[well]) / ro[well]):.1e}; final residual GPU "
          f"{rg[-1]:.1e} oracle {ro[-1]:.1e}")
    assert well.sum() >= 4
    np.testing.assert_allclose(rg[well], ro[well], rtol=1e-7)
    assert np.all(rg[~well] <= 1e-3 * ro[0])
    rho = np.abs(np.linalg.eigvals(A)).max()
    assert rho < 0.95
    np.testing.assert_allclose(xg, xo, rtol=0, atol=2 * (rg[-1] + ro[-1]) / (1 - rho) + 1e-12)


def test_standard_first_step_from_kmeans_is_the_oracle_s(gm):
    """One EM step (max_sweeps = 1) shows the initialisation itself: the
    K-means partition (same number of passes, same component count) and
    the FP64 step from it."""
    wl = workloads.mixture_1d1v(C=40, mean_n=700, clip=(100, 2000), seed=53)
    p, g, ref, out = run_both(gm, wl, 1, 0, max_sweeps=1)
    assert np.mean(g["km_passes"] == ref["km_passes"]) >= 0.95
    assert np.mean(g["K"] == ref["K"]) >= 0.95
    same = g["K"] == ref["K"]
    rel = np.abs(g["lnL"] - ref["lnL"]) / np.abs(ref["lnL"])
    assert np.mean(rel[same] <= 1e-5) >= 0.95
    assert np.all(g["iters"] == 1)


def test_standard_edge_cells(gm):
    """Empty cells, cells with fewer particles than Kmax, identical
    velocities, Kmax = 1, cells larger than the shared tile."""
    counts = np.array([0, 1, 2, 5, 9, 300, 0, 5000, 40])
    wl = workloads.mixture_1d1v(C=counts.shape[0], counts=counts, seed=54)
    wl.v[0, wl.cell_off[8]:wl.cell_off[9]] = 0.25  # identical velocities
    for kmax, init, aa in ((8, 0, 0), (8, 1, 5), (1, 0, 0)):
        p, g, ref, out = run_both(gm, wl, init, aa, Kmax=kmax, smem_particles=1024)
        mask = oracle.ST_EMPTY | oracle.ST_DEGENERATE | oracle.ST_TOO_FEW
        np.testing.assert_array_equal(g["status"] & mask, ref["status"] & mask)
        assert g["K"][0] == 0 and g["K"][6] == 0
        assert g["K"][8] == 1
        np.testing.assert_allclose(g["W"], ref["W"], rtol=1e-13)
        if kmax == 1:
            rel = np.abs(g["lnL"] - ref["lnL"]) / np.maximum(np.abs(ref["lnL"]), 1e-300)
            ok = (counts > 0) & ((g["status"] & oracle.ST_DEGENERATE) == 0)
            assert np.all(rel[ok] <= 1e-6)


def test_standard_arguments_are_checked(gm):
    wl = workloads.mixture_1d1v(C=4, mean_n=100, clip=(50, 200), seed=55)
    cfg = gm.config(wl.params)
    with pytest.raises(RuntimeError):
        gm.gm_compress_standard(cfg, dev(wl.cell_off), dev(wl.x), dev(wl.v), dev(wl.alpha),
                                aa_memory=9)
    with pytest.raises(RuntimeError):
        gm.gm_compress_standard(cfg, dev(wl.cell_off), dev(wl.x), dev(wl.v), dev(wl.alpha), init=2)
