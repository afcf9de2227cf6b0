"""GPU parity of the 2D mesh (gm_deposit_2d, gm_reconstruct_2d) against the
FP64 oracle, through the C ABI, on seeded 2D-3V Weibel-shaped inputs.

Reconstruction from identical mixtures (the oracle's fit fed to both
sides): positions bit-identical; dA (iterative on the GPU, dense direct in
the oracle) and alpha' to 1e-11 of their scale; velocities within 2e-6 of
the cell's velocity scale (FP32 Box-Muller normals, as in 1D); status bits
identical.  The exact invariants on every cell: charge on every node to
1e-12 of max |rho'|, momentum and energy of every projected cell to 1e-12.
At the benchmark's full size (128 x 128 cells x 512 particles) the
invariants are checked on every cell and the oracle's dense solve is
replaced by them (it is limited to 2048 cells)."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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
    return t.cpu().numpy()


@pytest.mark.parametrize("Cx,Cy,order", [(5, 3, 2), (16, 16, 2), (7, 4, 1), (1, 6, 2), (6, 1, 2),
                                         (2, 2, 2)])
def test_deposit_matches_oracle(gm, Cx, Cy, order):
    rng = np.random.default_rng(Cx * 31 + Cy)
    counts = rng.integers(0, 60, Cx * Cy)
    counts[0] = 0
    wl = workloads.with_weights(workloads.weibel_2d3v(Cx=Cx, Cy=Cy, counts=counts, shape_order=order,
                                                      seed=70 + Cx))
    p = dict(wl.params, q=-0.7)
    ref = oracle.deposit2d(p, wl.cell_off, wl.x, wl.y, wl.alpha)
    cfg = gm.config(p)
    rho = host(gm.gm_deposit_2d(cfg, gm.mesh2d(p), dev(wl.cell_off), dev(wl.x), dev(wl.y), dev(wl.alpha)))
    np.testing.assert_allclose(rho, ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())
    unit = host(gm.gm_deposit_2d(cfg, gm.mesh2d(p), dev(wl.cell_off), dev(wl.x), dev(wl.y)))
    ref1 = oracle.deposit2d(p, wl.cell_off, wl.x, wl.y, np.ones(wl.ntot))
    np.testing.assert_allclose(unit, ref1, rtol=1e-12, atol=1e-13 * np.abs(ref1).max())


def cell_scale(v, alpha, off):
    return np.array([(np.abs(v[:, s:e]) * alpha[s:e]).sum() for s, e in zip(off[:-1], off[1:])])


def check_invariants(gm, p, out_off, rec, fit_K, fit_prm, fit_W, rho_t):
    cfg = gm.config(p)
    mesh = gm.mesh2d(p)
    rho = gm.gm_deposit_2d(cfg, mesh, out_off, rec["x"], rec["y"], rec["alpha"])
    err = float((rho - rho_t).abs().max() / rho_t.abs().max())
    assert err <= 1e-12, err
    m1 = gm.gm_moments(cfg, out_off, rec["x"], rec["v"], rec["alpha"])
    mm = gm.gm_mixture_moments(cfg, fit_K, fit_prm, fit_W)
    proj = (rec["status"] & gm.ST_PROJ_SKIPPED) == 0
    assert float(proj.double().mean()) > 0.9
    C = out_off.shape[0] - 1
    counts = (out_off[1:] - out_off[:-1])
    cell = torch.repeat_interleave(torch.arange(C, device="cuda"), counts)
    pabs = torch.zeros(C, dtype=torch.float64, device="cuda").index_add_(
        0, cell, rec["alpha"] * rec["v"].abs().sum(0))
    ok = proj & (counts > 0)
    dp = ((m1["p"] - mm["p"]).abs().max(1).values / pabs)[ok]
    dE = ((m1["E"] - mm["E"]).abs() / mm["E"])[ok]
    assert float(dp.max()) <= 1e-12
    assert float(dE.max()) <= 1e-12
    return err


@pytest.mark.parametrize("Cx,Cy,ppc,varw", [(16, 16, 512, False), (16, 16, 128, True), (12, 5, 64, True),
                                            (1, 9, 120, False), (9, 1, 120, False), (2, 3, 40, False)])
def test_reconstruct_matches_oracle(gm, Cx, Cy, ppc, varw):
    wl = workloads.weibel_2d3v(Cx=Cx, Cy=Cy, ppc=ppc, seed=80 + Cx + Cy)
    if varw:
        wl = workloads.with_weights(wl)
    p = dict(wl.params, q=1.3)
    fit = oracle.compress(p, wl.cell_off, wl.x, wl.v, wl.alpha, nthreads=8)
    rho_t = oracle.deposit2d(p, wl.cell_off, wl.x, wl.y, wl.alpha)
    out_off = workloads.resample_offsets(wl.cell_off)
    ref = oracle.reconstruct2d(p, fit["K"], fit["params"], fit["W"], rho_t, out_off, nthreads=8)
    rcfg = gm.config(p, seed_key="recon_seed")
    K, prm, W, rt, oo = dev(fit["K"]), dev(fit["params"]), dev(fit["W"]), dev(rho_t), dev(out_off)
    rec = gm.gm_reconstruct_2d(rcfg, gm.mesh2d(p), K, prm, W, rt, oo, n_out=int(out_off[-1]), want_dA=True)
    torch.cuda.synchronize()
    g = {k: host(t) for k, t in rec.items()}
    np.testing.assert_array_equal(g["x"], ref["x"])
    np.testing.assert_array_equal(g["y"], ref["y"])
    np.testing.assert_array_equal(g["status"].astype(np.uint32), ref["status"])
    dAs = np.abs(ref["dA"]).max()
    assert np.abs(g["dA"] - ref["dA"]).max() <= 1e-11 * dAs
    asc = np.abs(ref["alpha"]).max()
    assert np.abs(g["alpha"] - ref["alpha"]).max() <= 1e-11 * asc
    vs = np.repeat(np.array([np.abs(ref["v"][:, s:e]).max() if e > s else 0.0
                             for s, e in zip(out_off[:-1], out_off[1:])]), np.diff(out_off))
    assert np.all(np.abs(g["v"] - ref["v"]) <= 2e-6 * vs[None, :] + 1e-15)
    check_invariants(gm, p, oo, rec, K, prm, W, rt)


def test_sparse_cells_empty_cells_and_cic(gm):
    """2-8 particles per cell (the slowest case for the solve), a few cells
    without resampled particles, and CIC: the iteration still reaches the
    oracle's dense solution."""
    for counts_kind, order in (("tiny", 2), ("empty", 2), ("tiny", 1)):
        rng = np.random.default_rng(91)
        C = 16 * 16
        counts = rng.integers(2, 9, C) if counts_kind == "tiny" else np.full(C, 64)
        wl = workloads.weibel_2d3v(Cx=16, Cy=16, counts=counts, shape_order=order, seed=92)
        p = dict(wl.params)
        fit = oracle.compress(p, wl.cell_off, wl.x, wl.v, wl.alpha, nthreads=8)
        rho_t = oracle.deposit2d(p, wl.cell_off, wl.x, wl.y, wl.alpha)
        oc = np.diff(wl.cell_off).copy()
        if counts_kind == "empty":
            oc[[5, 77, 200]] = 0
        out_off = np.concatenate([[0], np.cumsum(oc)]).astype(np.int64)
        ref = oracle.reconstruct2d(p, fit["K"], fit["params"], fit["W"], rho_t, out_off, nthreads=8)
        rec = gm.gm_reconstruct_2d(gm.config(p, seed_key="recon_seed"), gm.mesh2d(p), dev(fit["K"]),
                                   dev(fit["params"]), dev(fit["W"]), dev(rho_t), dev(out_off),
                                   n_out=int(out_off[-1]), want_dA=True)
        g = {k: host(t) for k, t in rec.items()}
        assert np.all((g["status"] & gm.ST_MM_NOT_CONVERGED) == 0), counts_kind
        np.testing.assert_array_equal(g["status"].astype(np.uint32), ref["status"])
        assert np.abs(g["dA"] - ref["dA"]).max() <= 1e-10 * np.abs(ref["dA"]).max()


def test_full_size_mesh_invariants(gm):
    """The benchmark mesh: 128 x 128 cells x 512 particles (8.4 M), fitted on
    the GPU, target charge deposited on the GPU, reconstructed; invariants
    on every cell; the oracle on sampled cells of the fit."""
    wl = workloads.weibel_2d3v(Cx=128, Cy=128, ppc=512, Lx=80.0, Ly=80.0, seed=93)
    p = dict(wl.params)
    cfg = gm.config(p)
    mesh = gm.mesh2d(p)
    off, x, y, v, a = dev(wl.cell_off), dev(wl.x), dev(wl.y), dev(wl.v), dev(wl.alpha)
    fit = gm.gm_compress(cfg, off, None, v, a)
    rho_t = gm.gm_deposit_2d(cfg, mesh, off, x, y, a)
    rec = gm.gm_reconstruct_2d(gm.config(p, seed_key="recon_seed"), mesh, fit["K"], fit["params"],
                               fit["W"], rho_t, off, n_out=wl.ntot)
    torch.cuda.synchronize()
    assert int((rec["status"] & gm.ST_MM_NOT_CONVERGED).sum()) == 0
    err = check_invariants(gm, p, off, rec, fit["K"], fit["params"], fit["W"], rho_t)
    print(f"full-size 2D mesh: charge error {err:.2e}, mean K {fit['K'].double().mean().item():.2f}")
    ref_rho = oracle.deposit2d(p, wl.cell_off, wl.x, wl.y, wl.alpha)
    np.testing.assert_allclose(host(rho_t), ref_rho, rtol=1e-12, atol=1e-13 * np.abs(ref_rho).max())
