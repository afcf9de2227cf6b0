"""Full-size 1D-3V workloads in the benchmark's launch configuration
(autotuned EM shape, graph-free direct calls): the 2048-cell x 4000
bi-Maxwellian batch and the 262144-cell log-normal pipeline
(~1.5e8 particles).  The oracle runs on sampled cells (each keyed by its
batch index, so both sides start from the same Philox picks); the exact
invariants are checked on every cell, vectorised on the device:
  * moments of every fit equal the particle moments (W 1e-14, momentum and
    second moments 1e-12 of the cell's scale, energy 1e-12);
  * after reconstruction: charge on every node 1e-12 of max |rho'|, energy
    of every projected cell 1e-12.
Agreement with the oracle: K equal and lnL within 1e-5 (natural), and
the equal-sweep rule of parity_helpers for the cells that stop at different
sweeps (unconverged cells: within 200 sweeps of the oracle's own
progress)."""
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


def segsum(vals, cell, C):
    out = torch.zeros(C, dtype=torch.float64, device=vals.device)
    return out.index_add_(0, cell, vals)


@pytest.mark.parametrize("which", ["bimaxwellian_1d3v", "lognormal_1d3v"])
def test_full_size_3v(gm, which):
    wl = workloads.get(which)
    off, x, v, a = dev(wl.cell_off), dev(wl.x), dev(wl.v), dev(wl.alpha)
    cfg = gm.config(wl.params)
    gm.gm_autotune(cfg, off, x, v, a)
    out = gm.gm_compress(cfg, off, x, v, a)
    rcfg = gm.config(wl.params, seed_key="recon_seed")
    rec = gm.gm_reconstruct(rcfg, out["K"], out["params"], out["W"], out["rho_target"], off,
                            n_out=wl.ntot)
    torch.cuda.synchronize()
    C, D = wl.C, wl.D

    # ---- oracle on sampled cells ------------------------------------------
    rng = np.random.default_rng(1)
    cells = np.sort(rng.choice(C, 40, replace=False))
    counts = wl.counts()[cells]
    soff = np.concatenate([[0], np.cumsum(counts)])
    idx = np.concatenate([np.arange(wl.cell_off[j], wl.cell_off[j + 1]) for j in cells])
    ref = oracle.compress(wl.params, soff, wl.x[idx], np.ascontiguousarray(wl.v[:, idx]),
                          wl.alpha[idx], nthreads=NTHREADS, cell_ids=cells)
    g = {k: t.cpu().numpy()[cells] for k, t in out.items()}
    agree, eq = agreement(g, ref, wl, cells)
    ks = g["K"] == ref["K"]
    print(f"{which}: K {ks.mean():.3f}, K + lnL {agree.mean():.3f}, at equal sweeps {eq.mean():.3f}")
    # the same K on 40 sampled cells; lnL within 1e-5 relative on most: the
    # 3V cells' |L| is often 1-3 % of N (whitened densities near 1), where
    # 1e-5 of |L| is 1e-7 nats per particle, the FP32 E-step's resolution
    # (tests/test_gpu_parity_natural.py measures this on 256 cells)
    assert ks.mean() >= 0.95, (cells[~ks], g["K"][~ks], ref["K"][~ks])
    assert agree.mean() >= 0.85, agree.mean()
    np.testing.assert_allclose(g["W"], ref["W"], rtol=1e-13)

    # ---- exact moments of every fit ------------------------------------------
    counts_t = torch.from_numpy(wl.counts()).cuda()
    cell = torch.repeat_interleave(torch.arange(C, device="cuda"), counts_t)
    m0 = gm.gm_moments(cfg, off, x, v, a)
    mm = gm.gm_mixture_moments(cfg, out["K"], out["params"], out["W"])
    ok = m0["W"] > 0
    assert float(((mm["W"] - m0["W"]).abs() / m0["W"])[ok].max()) <= 1e-14
    pabs = segsum(a * v.double().abs().sum(0), cell, C)
    assert float(((mm["p"] - m0["p"]).abs().max(1).values / pabs)[ok].max()) <= 1e-12
    assert float(((mm["E"] - m0["E"]).abs() / m0["E"])[ok].max()) <= 1e-12
    assert float(((mm["M2"] - m0["M2"]).abs().max(1).values / (2 * m0["E"]))[ok].max()) <= 1e-12

    # ---- reconstruction invariants on every cell ----------------------------
    m1 = gm.gm_moments(cfg, off, rec["x"], rec["v"], rec["alpha"])
    rt = out["rho_target"]
    assert float((m1["rho"] - rt).abs().max()) <= 1e-12 * float(rt.abs().max())
    proj = (rec["status"] & gm.ST_PROJ_SKIPPED) == 0
    assert float(proj.double().mean()) > 0.9
    dE = ((m1["E"] - m0["E"]).abs() / m0["E"])[proj & ok]
    assert float(dE.max()) <= 1e-12
    dp = ((m1["p"] - m0["p"]).abs().max(1).values / pabs)[proj & ok]
    assert float(dp.max()) <= 1e-12


def test_full_size_supplied_starts_lognormal_1d3v(gm):
    """gm_compress_from at full size, the benchmark's learned path after the
    network: most cells start from one component (the closed-form pre-pass,
    with the charge deposit fused into its sums kernel), every 50th cell
    from two (the EM kernel's work list).  The starts stand in for the
    network's output: the plain fit's first component, its first two for
    the listed cells.  Checked: the fused deposit's rho is bit-identical to
    the separate deposit's; sampled cells against the oracle started from
    the same mixtures; the exact moments of every fit; the reconstruction's
    invariants on every cell."""
    wl = workloads.get("lognormal_1d3v")
    off, x, v, a = dev(wl.cell_off), dev(wl.x), dev(wl.v), dev(wl.alpha)
    cfg = gm.config(wl.params)
    C, D = wl.C, wl.D
    plain = gm.gm_compress(cfg, off, x, v, a)
    K0 = torch.ones(C, dtype=torch.int32, device="cuda")
    two = torch.arange(0, C, 50, device="cuda")
    K0[two] = torch.clamp(plain["K"][two], max=2)
    prm = plain["params"].clone()
    prm[:, 2:, :] = 0.0
    one = K0 == 1
    prm[one, 1, :] = 0.0
    prm[:, 0, 0] = torch.where(one, torch.ones_like(prm[:, 0, 0]), prm[:, 0, 0])
    out = gm.gm_compress(cfg, off, x, v, a, init_K=K0, init_params=prm)
    torch.cuda.synchronize()
    assert torch.equal(out["rho_target"], plain["rho_target"])
    assert float((out["sweeps"] == 1).double().mean()) > 0.95

    rng = np.random.default_rng(2)
    cells = np.sort(np.concatenate([rng.choice(C, 30, replace=False), np.arange(0, C, 50)[:10]]))
    counts = wl.counts()[cells]
    soff = np.concatenate([[0], np.cumsum(counts)])
    idx = np.concatenate([np.arange(wl.cell_off[j], wl.cell_off[j + 1]) for j in cells])
    K0h, prmh = K0.cpu().numpy(), prm.cpu().numpy()
    ref = oracle.compress(wl.params, soff, wl.x[idx], np.ascontiguousarray(wl.v[:, idx]),
                          wl.alpha[idx], nthreads=NTHREADS, cell_ids=cells,
                          init_K=K0h[cells], init_params=prmh[cells])
    g = {k: t.cpu().numpy()[cells] for k, t in out.items()}
    ks = g["K"] == ref["K"]
    rel = np.abs(g["lnL"] - ref["lnL"]) / np.abs(ref["lnL"])
    print(f"supplied starts: K {ks.mean():.3f}, K + lnL {(ks & (rel <= 1e-5)).mean():.3f}")
    assert ks.mean() >= 0.95, (cells[~ks], g["K"][~ks], ref["K"][~ks])
    k1 = K0h[cells] == 1
    # the one-component cells are closed forms: exact agreement up to the
    # summation order of the FP64 moments
    assert np.all(ks[k1])
    assert np.all(rel[k1] <= 1e-12 * (1.0 + counts[k1] / np.abs(ref["lnL"][k1]))), rel[k1].max()
    np.testing.assert_allclose(g["W"], ref["W"], rtol=1e-13)

    counts_t = torch.from_numpy(wl.counts()).cuda()
    cell = torch.repeat_interleave(torch.arange(C, device="cuda"), counts_t)
    m0 = gm.gm_moments(cfg, off, x, v, a)
    mm = gm.gm_mixture_moments(cfg, out["K"], out["params"], out["W"])
    ok = m0["W"] > 0
    assert float(((mm["W"] - m0["W"]).abs() / m0["W"])[ok].max()) <= 1e-14
    pabs = segsum(a * v.double().abs().sum(0), cell, C)
    assert float(((mm["p"] - m0["p"]).abs().max(1).values / pabs)[ok].max()) <= 1e-12
    assert float(((mm["E"] - m0["E"]).abs() / m0["E"])[ok].max()) <= 1e-12

    rcfg = gm.config(wl.params, seed_key="recon_seed")
    rec = gm.gm_reconstruct(rcfg, out["K"], out["params"], out["W"], out["rho_target"], off,
                            n_out=wl.ntot)
    m1 = gm.gm_moments(cfg, off, rec["x"], rec["v"], rec["alpha"])
    rt = out["rho_target"]
    assert float((m1["rho"] - rt).abs().max()) <= 1e-12 * float(rt.abs().max())
    proj = (rec["status"] & gm.ST_PROJ_SKIPPED) == 0
    dE = ((m1["E"] - m0["E"]).abs() / m0["E"])[proj & ok]
    assert float(dE.max()) <= 1e-12
