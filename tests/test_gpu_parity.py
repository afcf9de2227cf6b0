"""GPU (sm_103a) parity of the CUDA path against the FP64 oracle, through the
C ABI, on seeded inputs.

Tolerances:
  * selected component count K and per-cell penalised log-likelihood
    (1e-5 relative): naturally equal in most cells; the rest must agree
    under the equal-sweep rule of parity_helpers (the FP32 E-step moves the
    knife-edge stopping sweep; unconverged cells drift along flat
    directions); each test states both rates it requires;
  * moments of the fit vs the particles': 1e-12 relative (exact, Sec. 2.3.1);
  * reconstruction: positions bit-identical; corrected weights and dA
    1e-12 relative; velocities 2e-6 relative to the cell's spread (FP32
    Box-Muller normals against the oracle's FP64 ones);
  * charge on every node, momentum and energy of every projected cell:
    1e-12 relative.
"""
import os

import numpy as np
import pytest

import oracle
import workloads
from parity_helpers import agreement

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


def host(t):
    return t.detach().cpu().numpy()


def run_gpu_compress(gm, wl, **over):
    cfg = gm.config(wl.params, **over)
    out = gm.gm_compress(cfg, dev(wl.cell_off), dev(wl.x), dev(wl.v), dev(wl.alpha))
    torch.cuda.synchronize()
    return {k: host(v) for k, v in out.items()}, out


def check_compress_parity(g, ref, min_k=0.95, min_agree=0.85, wl=None, cells=None):
    """Asserts the natural rates: the same K in at least min_k of the cells,
    the same K and lnL within 1e-5 in at least min_agree.  Prints the rate
    after the equal-sweep rule of parity_helpers as a diagnostic.  Returns
    (K rate, natural rate)."""
    from parity_helpers import same_k
    ks = same_k(g, ref)
    if wl is not None:
        agree, eq = agreement(g, ref, wl, cells)
    else:
        rel = np.abs(g["lnL"] - ref["lnL"]) / np.maximum(np.abs(ref["lnL"]), 1e-300)
        agree = ks & (rel <= 1e-5)
        eq = agree.copy()
    print(f"parity: K {ks.mean():.3f}, K + lnL {agree.mean():.3f} (at equal sweeps {eq.mean():.3f})")
    bad = np.flatnonzero(~agree)
    assert ks.mean() >= min_k, (np.flatnonzero(~ks), g["K"][~ks], ref["K"][~ks])
    assert agree.mean() >= min_agree, (bad, g["K"][bad], ref["K"][bad])
    np.testing.assert_allclose(g["W"], ref["W"], rtol=1e-13)
    if cells is None:
        np.testing.assert_allclose(g["rho_target"], ref["rho_target"], rtol=1e-12,
                                   atol=1e-13 * np.abs(ref["rho_target"]).max())
    # status bits that do not depend on the FP32 trajectory
    mask = oracle.ST_EMPTY | oracle.ST_DEGENERATE | oracle.ST_TOO_FEW
    np.testing.assert_array_equal(g["status"] & mask, ref["status"] & mask)
    return ks.mean(), agree.mean()


def check_fit_moments(gm, wl, out_dev):
    cfg = gm.config(wl.params)
    m0 = gm.gm_moments(cfg, dev(wl.cell_off), dev(wl.x), dev(wl.v), dev(wl.alpha))
    mm = gm.gm_mixture_moments(cfg, out_dev["K"], out_dev["params"], out_dev["W"])
    m0 = {k: host(v) for k, v in m0.items()}
    mm = {k: host(v) for k, v in mm.items()}
    ok = m0["W"] > 0
    np.testing.assert_allclose(mm["W"][ok], m0["W"][ok], rtol=1e-14)
    D = wl.D
    for j in np.flatnonzero(ok):
        sl = slice(wl.cell_off[j], wl.cell_off[j + 1])
        pabs = (wl.alpha[sl] * np.abs(wl.v[:, sl].astype(np.float64))).sum()
        assert np.abs(mm["p"][j] - m0["p"][j]).max() <= 1e-12 * pabs
        assert abs(mm["E"][j] - m0["E"][j]) <= 1e-12 * m0["E"][j]
        assert np.abs(mm["M2"][j] - m0["M2"][j]).max() <= 1e-12 * 2 * m0["E"][j]
    # the oracle's moments routine agrees with the GPU's
    mo = oracle.moments(wl.params, wl.cell_off, wl.x, wl.v, wl.alpha)
    np.testing.assert_allclose(m0["E"], mo["E"], rtol=1e-12)
    np.testing.assert_allclose(m0["rho"], mo["rho"], rtol=1e-12, atol=1e-13 * np.abs(mo["rho"]).max())
    assert D in (1, 3)


# ---------------------------------------------------------------------------
# compression
# ---------------------------------------------------------------------------
def test_compress_two_stream_full(gm):
    wl = workloads.two_stream_1d1v()  # 32 cells x 1024, FP64 v, CIC
    g, gd = run_gpu_compress(gm, wl)
    ref = oracle.compress(wl.params, wl.cell_off, wl.x, wl.v, wl.alpha, nthreads=NTHREADS)
    check_compress_parity(g, ref, min_k=0.96, min_agree=0.96, wl=wl)
    check_fit_moments(gm, wl, gd)


@pytest.mark.parametrize("precision", [0, 1])
def test_compress_mixture_ragged(gm, precision):
    # uneven counts across several tiles, cells larger than the shared tile
    # (global-scratch path), a ragged tail and tiny cells
    rng = np.random.default_rng(5)
    counts = rng.integers(200, 3000, 40)
    counts[3] = 5000   # above the default 1V tile
    counts[7] = 11     # just above the "too few" limit
    counts[8] = 10
    counts[9] = 3
    wl = workloads.mixture_1d1v(C=40, counts=counts, seed=77)
    g, gd = run_gpu_compress(gm, wl, precision=precision)
    ref = oracle.compress(wl.params, wl.cell_off, wl.x, wl.v, wl.alpha, nthreads=NTHREADS)
    # the FP64 M-step and corrected convergence test (precision 0, the
    # default) follow the oracle's stopping sweep; the FP32 option stops
    # within a few sweeps of it on most cells but not on the cells that creep
    # at a rate near tol (measured 78-90 % natural agreement)
    check_compress_parity(g, ref, min_k=0.95 if precision == 0 else 0.8,
                          min_agree=0.95 if precision == 0 else 0.6, wl=wl)
    check_fit_moments(gm, wl, gd)


@pytest.mark.parametrize("smem_particles", [0, 1024])
def test_compress_3v(gm, smem_particles):
    wl = workloads.bimaxwellian_1d3v(C=24, ppc=1500)
    g, gd = run_gpu_compress(gm, wl, smem_particles=smem_particles)
    ref = oracle.compress(wl.params, wl.cell_off, wl.x, wl.v, wl.alpha, nthreads=NTHREADS)
    check_compress_parity(g, ref, min_k=0.95, min_agree=0.85, wl=wl)
    check_fit_moments(gm, wl, gd)


def test_compress_variable_weights_and_edge_cells(gm):
    counts = np.array([0, 1, 2, 7, 300, 0, 500, 64])
    wl = workloads.with_weights(workloads.mixture_1d1v(C=8, counts=counts, seed=3))
    # a cell whose particles all share one velocity
    v = wl.v.copy()
    v[:, wl.cell_off[7]:wl.cell_off[8]] = np.float32(0.125)
    wl = workloads.Workload("edge", wl.cell_off, wl.x, v, wl.alpha, wl.params)
    g, gd = run_gpu_compress(gm, wl)
    ref = oracle.compress(wl.params, wl.cell_off, wl.x, wl.v, wl.alpha)
    np.testing.assert_array_equal(g["K"], ref["K"])
    np.testing.assert_array_equal(g["status"] & (oracle.ST_EMPTY | oracle.ST_DEGENERATE),
                                  ref["status"] & (oracle.ST_EMPTY | oracle.ST_DEGENERATE))
    assert g["K"][0] == 0 and g["K"][5] == 0 and g["K"][7] == 1
    check_compress_parity(g, ref, min_k=1.0, min_agree=1.0, wl=wl)


@pytest.mark.parametrize("D", [1, 3])
def test_compress_and_reconstruct_at_the_largest_kmax(gm, D):
    """Kmax = 16, the largest the library accepts: every per-component array
    of the EM kernel at full size (16 initial components); the fits and the
    reconstruction of the oracle's fits against the oracle."""
    if D == 1:
        wl = workloads.mixture_1d1v(C=24, mean_n=1200, clip=(100, 3000), seed=91, Kmax=16)
    else:
        wl = workloads.bimaxwellian_1d3v(C=20, ppc=800, seed=92, Kmax=16)
    g, gd = run_gpu_compress(gm, wl)
    ref = oracle.compress(wl.params, wl.cell_off, wl.x, wl.v, wl.alpha, nthreads=NTHREADS)
    check_compress_parity(g, ref, min_k=0.9, min_agree=0.85, wl=wl)
    check_fit_moments(gm, wl, gd)
    gr, o = recon_both(gm, wl, ref)
    np.testing.assert_array_equal(gr["x"], o["x"])
    np.testing.assert_allclose(gr["alpha"], o["alpha"], rtol=1e-12)
    np.testing.assert_array_equal(gr["status"], o["status"])


def test_compress_kmax1_is_sample_moments(gm):
    wl = workloads.bimaxwellian_1d3v(C=6, ppc=700)
    wl.params["Kmax"] = 1
    g, gd = run_gpu_compress(gm, wl)
    ref = oracle.compress(wl.params, wl.cell_off, wl.x, wl.v, wl.alpha)
    np.testing.assert_array_equal(g["K"], 1)
    np.testing.assert_allclose(g["params"], ref["params"], rtol=1e-11, atol=1e-14)
    np.testing.assert_allclose(g["lnL"], ref["lnL"], rtol=1e-6)


# ---------------------------------------------------------------------------
# reconstruction (same parameters into both paths)
# ---------------------------------------------------------------------------
def recon_both(gm, wl, ref):
    prm = dict(wl.params)
    rcfg = gm.config(prm, seed_key="recon_seed")
    rec = gm.gm_reconstruct(rcfg, dev(ref["K"]), dev(ref["params"]), dev(ref["W"]),
                            dev(ref["rho_target"]), dev(wl.cell_off), n_out=wl.ntot, want_dA=True)
    torch.cuda.synchronize()
    g = {k: host(v) for k, v in rec.items()}
    o = oracle.reconstruct(prm, ref["K"], ref["params"], ref["W"], ref["rho_target"], wl.cell_off,
                           nthreads=NTHREADS)
    return g, o


@pytest.mark.parametrize("which", ["two_stream", "mixture", "bimax3v"])
def test_reconstruct_parity_and_conservation(gm, which):
    if which == "two_stream":
        wl = workloads.two_stream_1d1v(C=16, ppc=512)
    elif which == "mixture":
        wl = workloads.mixture_1d1v(C=100, mean_n=300, clip=(20, 800), counts="uniform")
    else:
        wl = workloads.bimaxwellian_1d3v(C=70, ppc=400)
    ref = oracle.compress(wl.params, wl.cell_off, wl.x, wl.v, wl.alpha, nthreads=NTHREADS)
    g, o = recon_both(gm, wl, ref)
    np.testing.assert_array_equal(g["x"], o["x"])
    np.testing.assert_allclose(g["dA"], o["dA"], rtol=0, atol=1e-12 * np.abs(o["alpha"]).max())
    np.testing.assert_allclose(g["alpha"], o["alpha"], rtol=1e-12)
    np.testing.assert_array_equal(g["status"], o["status"])
    # velocities: FP32 Box-Muller vs FP64
    for j in range(wl.C):
        sl = slice(wl.cell_off[j], wl.cell_off[j + 1])
        scale = np.abs(o["v"][:, sl]).max() + 1e-30
        assert np.abs(g["v"][:, sl] - o["v"][:, sl]).max() <= 2e-6 * scale, j
    # invariants of the GPU output
    cfg = gm.config(wl.params)
    m0 = {k: host(v) for k, v in gm.gm_moments(cfg, dev(wl.cell_off), dev(wl.x), dev(wl.v),
                                                 dev(wl.alpha)).items()}
    m1 = {k: host(v) for k, v in gm.gm_moments(cfg, dev(wl.cell_off), dev(g["x"]), dev(g["v"]),
                                                 dev(g["alpha"])).items()}
    rt = ref["rho_target"]
    np.testing.assert_allclose(m1["rho"], rt, rtol=0, atol=1e-12 * np.abs(rt).max())
    proj = (g["status"] & oracle.ST_PROJ_SKIPPED) == 0
    assert proj.mean() > 0.9
    for j in np.flatnonzero(proj):
        sl = slice(wl.cell_off[j], wl.cell_off[j + 1])
        pabs = (wl.alpha[sl] * np.abs(wl.v[:, sl].astype(np.float64))).sum()
        assert np.abs(m1["p"][j] - m0["p"][j]).max() <= 1e-12 * pabs
        assert abs(m1["E"][j] - m0["E"][j]) <= 1e-12 * m0["E"][j]


@pytest.mark.parametrize("C", [2048, 9001])
def test_reconstruct_large_mesh_block_solve(gm, C):
    """Meshes of 2048 cells and more take the multi-CTA mass-matrix solve
    (blocks of ~64 rows eliminated across the GPU, the interface system on
    one CTA): dA against the oracle's direct cyclic solve, and the charge
    on every node."""
    wl = workloads.mixture_1d1v(C=C, mean_n=40, clip=(12, 90), seed=41)
    ref = oracle.compress(wl.params, wl.cell_off, wl.x, wl.v, wl.alpha, nthreads=NTHREADS)
    g, o = recon_both(gm, wl, ref)
    np.testing.assert_array_equal(g["x"], o["x"])
    np.testing.assert_allclose(g["dA"], o["dA"], rtol=0, atol=1e-12 * np.abs(o["alpha"]).max())
    np.testing.assert_allclose(g["alpha"], o["alpha"], rtol=1e-12)
    cfg = gm.config(wl.params)
    m1 = {k: host(v) for k, v in gm.gm_moments(cfg, dev(wl.cell_off), dev(g["x"]), dev(g["v"]),
                                                 dev(g["alpha"])).items()}
    rt = ref["rho_target"]
    np.testing.assert_allclose(m1["rho"], rt, rtol=0, atol=1e-12 * np.abs(rt).max())


def test_reconstruct_small_meshes_and_empty_cells(gm):
    for C in (1, 2, 3, 5, 70):
        rng = np.random.default_rng(C)
        wl = workloads.mixture_1d1v(C=C, counts=rng.integers(30, 200, C), seed=C)
        ref = oracle.compress(wl.params, wl.cell_off, wl.x, wl.v, wl.alpha)
        out_off = wl.cell_off.copy()
        if C >= 5:  # one cell gets no resampled particle
            n = np.diff(out_off)
            n[2] = 0
            out_off = np.concatenate([[0], np.cumsum(n)])
        prm = dict(wl.params)
        rcfg = gm.config(prm, seed_key="recon_seed")
        rec = gm.gm_reconstruct(rcfg, dev(ref["K"]), dev(ref["params"]), dev(ref["W"]),
                                dev(ref["rho_target"]), dev(out_off), n_out=int(out_off[-1]),
                                want_dA=True)
        g = {k: host(v) for k, v in rec.items()}
        o = oracle.reconstruct(prm, ref["K"], ref["params"], ref["W"], ref["rho_target"], out_off)
        np.testing.assert_array_equal(g["x"], o["x"])
        np.testing.assert_allclose(g["dA"], o["dA"], rtol=1e-11, atol=1e-12)
        np.testing.assert_array_equal(g["status"], o["status"])


# ---------------------------------------------------------------------------
# full-size batched workload in the benchmark's launch configuration
# ---------------------------------------------------------------------------
def test_full_size_batched_sampled_cells(gm):
    wl = workloads.mixture_1d1v()  # 4096 cells, Poisson(2000), FP32 v
    g, gd = run_gpu_compress(gm, wl)
    # the oracle on 64 sampled cells (each keyed by its batch index)
    rng = np.random.default_rng(0)
    cells = np.sort(rng.choice(wl.C, 64, replace=False))
    counts = wl.counts()[cells]
    off = np.concatenate([[0], np.cumsum(counts)])
    idx = np.concatenate([np.arange(wl.cell_off[j], wl.cell_off[j + 1]) for j in cells])
    ref = oracle.compress(wl.params, off, wl.x[idx], wl.v[:, idx], wl.alpha[idx],
                          nthreads=NTHREADS, cell_ids=cells)
    gs = {k: v[cells] for k, v in g.items()}
    check_compress_parity(gs, ref, min_k=0.95, min_agree=0.95, wl=wl, cells=cells)
    # exact moments on every cell
    check_fit_moments(gm, wl, gd)
    # reconstruction invariants on every cell
    rcfg = gm.config(wl.params, seed_key="recon_seed")
    rec = gm.gm_reconstruct(rcfg, gd["K"], gd["params"], gd["W"], gd["rho_target"],
                            dev(wl.cell_off), n_out=wl.ntot)
    cfg = gm.config(wl.params)
    m0 = gm.gm_moments(cfg, dev(wl.cell_off), dev(wl.x), dev(wl.v), dev(wl.alpha))
    m1 = gm.gm_moments(cfg, dev(wl.cell_off), rec["x"], rec["v"], rec["alpha"])
    rt = gd["rho_target"]
    assert float((m1["rho"] - rt).abs().max()) <= 1e-12 * float(rt.abs().max())
    proj = (rec["status"] & gm.ST_PROJ_SKIPPED) == 0
    assert float(proj.double().mean()) > 0.9
    dE = ((m1["E"] - m0["E"]).abs() / m0["E"])[proj]
    assert float(dE.max()) <= 1e-12
    # reconstruction parity on the sampled cells (same parameters)
    sub_off = off
    o = oracle.reconstruct(dict(wl.params, L=float(len(cells))), g["K"][cells], g["params"][cells],
                           g["W"][cells], np.zeros(len(cells)), sub_off, nthreads=NTHREADS,
                           want_raw=True)
    assert o["x"].shape[0] == idx.shape[0]
