"""gm_reconstruct_noalloc (scratch in the library's static device array, no
device allocation in the call) against gm_reconstruct, through the C ABI.

This file is collected last so that a run stopping at the first failure has
already run every other test.  It passes alone in a fresh process as well."""
import os

import numpy as np
import pytest

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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _outputs(D, n, C, dev):
    return dict(x=torch.full((n,), np.nan, dtype=torch.float64, device=dev),
                v=torch.full((D, n), np.nan, dtype=torch.float64, device=dev),
                alpha=torch.full((n,), np.nan, dtype=torch.float64, device=dev),
                status=torch.full((C,), -1, dtype=torch.int32, device=dev),
                dA=torch.full((C,), np.nan, dtype=torch.float64, device=dev))


@pytest.mark.parametrize("which", ["mixture_1d1v", "bimaxwellian_1d3v"])
def test_noalloc_matches_reconstruct_twice(gm, which):
    if which == "mixture_1d1v":
        wl = workloads.mixture_1d1v(C=300, mean_n=400, clip=(20, 900), counts="uniform")
    else:
        wl = workloads.bimaxwellian_1d3v(C=200, ppc=300)
    cfg = gm.config(wl.params)
    fit = gm.gm_compress(cfg, _dev(wl.cell_off), _dev(wl.x), _dev(wl.v), _dev(wl.alpha))
    rcfg = gm.config(wl.params, seed_key="recon_seed")
    out_off = _dev(wl.cell_off)
    ref = gm.gm_reconstruct(rcfg, fit["K"], fit["params"], fit["W"], fit["rho_target"], out_off,
                            n_out=wl.ntot, want_dA=True)
    for _ in range(2):  # two calls in a row share (and reuse) the static scratch
        got = _outputs(wl.D, wl.ntot, wl.C, ref["x"].device)
        gm.gm_reconstruct_noalloc(rcfg, fit["K"], fit["params"], fit["W"], fit["rho_target"],
                                  out_off, got, n_out=wl.ntot)
        torch.cuda.synchronize()
        assert torch.equal(got["x"], ref["x"])
        assert torch.equal(got["status"], ref["status"])
        for k in ("v", "alpha", "dA"):
            torch.testing.assert_close(got[k], ref[k], rtol=1e-12, atol=1e-14)


def test_noalloc_rejects_too_many_cells(gm):
    cfg = gm.config(dict(D=1, Kmax=2, shape_order=2, L=40000.0))
    C = 40000
    z = torch.zeros(C, dtype=torch.float64, device="cuda")
    K = torch.zeros(C, dtype=torch.int32, device="cuda")
    off = torch.zeros(C + 1, dtype=torch.int64, device="cuda")
    out = _outputs(1, 0, C, "cuda")
    with pytest.raises(RuntimeError, match="at most 32768 cells"):
        gm.gm_reconstruct_noalloc(cfg, K, torch.zeros((C, 2, 3), dtype=torch.float64, device="cuda"),
                                  z, z, off, out, n_out=0)


def test_noalloc_large_mesh_blocked_solve(gm):
    """32768 cells (the limit) of the 3V generator with 16-48 particles each:
    the mass-matrix solve takes its multi-CTA blocked path (>= 2048 cells),
    whose interface workspace lies at the far end of the static array.
    Bit-identical to gm_reconstruct on two calls in a row, dA against the
    oracle's direct cyclic tridiagonal solve of the same fit, and the mesh
    charge of the output against the target."""
    import oracle
    rng = np.random.default_rng(11)
    C = 32768
    counts = rng.integers(16, 49, C)
    wl = workloads.bimaxwellian_1d3v(C=C, counts=counts, seed=workloads.GEN_SEED_BASE + 40)
    cfg = gm.config(wl.params)
    fit = gm.gm_compress(cfg, _dev(wl.cell_off), _dev(wl.x), _dev(wl.v), _dev(wl.alpha))
    rcfg = gm.config(wl.params, seed_key="recon_seed")
    out_off = _dev(wl.cell_off)
    ref = gm.gm_reconstruct(rcfg, fit["K"], fit["params"], fit["W"], fit["rho_target"], out_off,
                            n_out=wl.ntot, want_dA=True)
    for _ in range(2):
        got = _outputs(wl.D, wl.ntot, wl.C, ref["x"].device)
        gm.gm_reconstruct_noalloc(rcfg, fit["K"], fit["params"], fit["W"], fit["rho_target"],
                                  out_off, got, n_out=wl.ntot)
        torch.cuda.synchronize()
        for k in ("x", "v", "alpha", "dA", "status"):
            assert torch.equal(got[k], ref[k]), k
    h = {k: v.cpu().numpy() for k, v in fit.items() if v is not None}
    o = oracle.reconstruct(wl.params, h["K"], h["params"], h["W"], h["rho_target"], wl.cell_off,
                           nthreads=os.cpu_count() or 4)
    # the blocked partition solve against the direct cyclic solve: 32768
    # unknowns, corrections up to ~0.7 of the weights (16-48 particles per
    # cell); rounding of either solve stays within 1e-11 of the largest
    dA = got["dA"].cpu().numpy()
    scale = np.abs(o["dA"]).max()
    assert np.abs(dA - o["dA"]).max() <= 1e-11 * scale
    # and the charge on every node is the target's to round-off
    m = gm.gm_moments(cfg, out_off, got["x"], got["v"], got["alpha"])
    rt = fit["rho_target"]
    assert torch.allclose(m["rho"], rt, rtol=0, atol=1e-12 * float(rt.abs().max()))


def test_noalloc_short_n_out_is_flagged(gm):
    """A caller whose n_out is shorter than out_off[-1]: every cell whose
    range ends beyond n_out gets GM_ST_BAD_RANGE and nothing is written
    past n_out (the buffers are allocated at full length, the sentinel
    tail must stay untouched)."""
    wl = workloads.mixture_1d1v(C=64, mean_n=100, clip=(20, 200), counts="uniform", seed=91)
    cfg = gm.config(wl.params)
    fit = gm.gm_compress(cfg, _dev(wl.cell_off), _dev(wl.x), _dev(wl.v), _dev(wl.alpha))
    rcfg = gm.config(wl.params, seed_key="recon_seed")
    n_short = int(wl.cell_off[40]) + 5  # inside cell 40
    got = _outputs(wl.D, wl.ntot, wl.C, "cuda")
    gm.gm_reconstruct_noalloc(rcfg, fit["K"], fit["params"], fit["W"], fit["rho_target"],
                              _dev(wl.cell_off), got, n_out=n_short)
    torch.cuda.synchronize()
    st = got["status"].cpu().numpy()
    bad = (st & gm.ST_BAD_RANGE) != 0
    expect = wl.cell_off[1:] > n_short
    np.testing.assert_array_equal(bad, expect)
    x = got["x"].cpu().numpy()
    assert np.all(np.isnan(x[n_short:]))
    assert not np.any(np.isnan(x[: int(wl.cell_off[40])]))
