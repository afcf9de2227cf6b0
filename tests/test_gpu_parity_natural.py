"""The parity criterion of the compression on large samples, at the natural
stopping sweep (no re-run of the oracle), through the C ABI: GPU fits with
the default precision (FP64 M-step, corrected FP64 convergence test)
against the FP64 oracle on the same seeded cells.

Measured and asserted, separately:
  * K only: the same selected component count;
  * K + lnL: the same count and the per-cell log-likelihood eq. (lnL-GM)
    within 1e-5 relative;
  * each split by cells that converge on both sides and cells that run into
    max_sweeps on either side (unconverged: both are still moving along a
    flat direction of the likelihood);
  * the fitted parameters element by element (components matched by their
    mean) for the cells that agree, and, for a sample of cells, at equal
    sweep counts (the oracle re-run for the GPU's number of sweeps), where
    only the FP32 E-step separates the two.

Samples: the first 1024 cells of the 4096-cell 1D-1V batch and the first 256
cells of the 2048 x 4000 1D-3V batch (the generator seeds of the benchmark's
rank 0).
"""
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


def first_cells(wl, C):
    n = int(wl.cell_off[C])
    p = dict(wl.params)
    p["L"] = wl.params["L"] * C / wl.C
    return workloads.Workload(wl.name, wl.cell_off[: C + 1].copy(), wl.x[:n].copy(),
                              np.ascontiguousarray(wl.v[:, :n]), wl.alpha[:n].copy(), p)


def matched(prm, K, D):
    """components [K, P] sorted by their first mean coordinate"""
    a = prm[:K]
    return a[np.argsort(a[:, 1], kind="stable")]


def pair_up(a, b, D):
    """a's components reordered to match b's (the assignment that minimises
    the summed distance of the means in units of b's component spreads)"""
    from scipy.optimize import linear_sum_assignment
    sd = np.sqrt(b[:, [2]] if D == 1 else b[:, [4, 7, 9]])
    cost = np.array([[np.sum(((ai[1:1 + D] - bj[1:1 + D]) / sdj) ** 2) for bj, sdj in zip(b, sd)]
                     for ai in a])
    r, c = linear_sum_assignment(cost)
    out = np.empty_like(a)
    out[c] = a[r]
    return out


def param_errors(a, b, D):
    """(weight abs., mean / component sd, covariance / sqrt(S_ii S_jj)) max
    differences of two matched component lists (b the oracle's)"""
    if D == 1:
        sd = np.sqrt(b[:, 2])
        return (np.abs(a[:, 0] - b[:, 0]).max(), (np.abs(a[:, 1] - b[:, 1]) / sd).max(),
                (np.abs(a[:, 2] - b[:, 2]) / b[:, 2]).max())
    sdd = np.sqrt(b[:, [4, 7, 9]])
    idx = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    sc = np.stack([sdd[:, i] * sdd[:, j] for i, j in idx], 1)
    return (np.abs(a[:, 0] - b[:, 0]).max(), (np.abs(a[:, 1:4] - b[:, 1:4]) / sdd).max(),
            (np.abs(a[:, 4:] - b[:, 4:]) / sc).max())


CASES = {
    # workload, cells, floors: K (converged on both sides), K (all cells),
    # K + lnL (converged on both sides); measured on a GB300: 1D-1V 100 /
    # 99.8 / 99.9 %, 1D-3V 100 / 100 / 97.4 %.  The 3V cells' |L| is often
    # 1-3 % of N (whitened densities near 1), where 1e-5 of |L| is 1e-7 nats
    # per particle, the FP32 E-step's resolution; per particle every
    # converged cell with the same K agrees to 1e-5 in 99 % of cells
    # (asserted below).
    "mixture_1d1v": (lambda: workloads.mixture_1d1v(seed=workloads.GEN_SEED_BASE + 1), 1024,
                     0.99, 0.99, 0.99),
    "bimaxwellian_1d3v": (lambda: workloads.bimaxwellian_1d3v(seed=workloads.GEN_SEED_BASE + 1), 256,
                          0.99, 0.99, 0.95),
}


@pytest.mark.parametrize("which", list(CASES))
def test_natural_stop_parity(gm, which):
    make, C, k_conv, k_all, kl_conv = CASES[which]
    wl = first_cells(make(), C)
    D = wl.D
    cfg = gm.config(wl.params)
    out = gm.gm_compress(cfg, dev(wl.cell_off), dev(wl.x), dev(wl.v), dev(wl.alpha))
    g = {k: v.cpu().numpy() for k, v in out.items() if v is not None}
    ref = oracle.compress(wl.params, wl.cell_off, wl.x, wl.v, wl.alpha, nthreads=NTHREADS)
    rel = np.abs(g["lnL"] - ref["lnL"]) / np.abs(ref["lnL"])
    same_k = g["K"] == ref["K"]
    same_kl = same_k & (rel <= 1e-5)
    conv = ((g["status"] & oracle.ST_EM_MAXSWEEPS) == 0) & ((ref["status"] & oracle.ST_EM_MAXSWEEPS) == 0)
    summary = (f"{which} {C} cells: K {same_k.mean():.4f}, K+lnL {same_kl.mean():.4f}; "
               f"converged on both sides ({conv.mean():.3f} of cells): K {same_k[conv].mean():.4f}, "
               f"K+lnL {same_kl[conv].mean():.4f}; max_sweeps on either side: "
               f"K {same_k[~conv].mean() if (~conv).any() else 1.0:.4f}, "
               f"K+lnL {same_kl[~conv].mean() if (~conv).any() else 1.0:.4f}")
    print(summary)
    assert same_k[conv].mean() >= k_conv, summary
    assert same_k.mean() >= k_all, summary
    assert same_kl[conv].mean() >= kl_conv, summary
    per_particle = np.abs(g["lnL"] - ref["lnL"]) / np.maximum(wl.counts(), 1)
    assert np.mean(per_particle[same_k & conv] <= 1e-5) >= 0.99, per_particle[same_k & conv].max()
    # element by element, for the cells that agree and converged: the two
    # sides stop within a few sweeps of each other, and along the
    # likelihood's flat directions a sweep moves the parameters far more
    # than L (relative 1e-3 against 1e-6), and two overlapping components
    # can trade weight and width at almost the same L; 97 % of cells within
    # (weight 5e-4, mean 5e-3 sd, covariance 5e-3) (measured 98-99 %),
    # components paired by their means
    errs = np.array([param_errors(pair_up(g["params"][j][:g["K"][j]], ref["params"][j][:ref["K"][j]], D),
                                  ref["params"][j][:ref["K"][j]], D)
                     for j in np.flatnonzero(same_kl & conv)])
    tol = np.array([5e-4, 5e-3, 5e-3])
    print("element-wise (weight, mean / sd, covariance): 99th percentile",
          np.percentile(errs, 99, axis=0), "max", errs.max(axis=0))
    assert np.mean(np.all(errs <= tol, axis=1)) >= 0.97, np.percentile(errs, 99, axis=0)
    # at equal sweep counts only the FP32 E-step separates the two sides:
    # 16 cells, every 16th (measured max 1.4e-5, 2.4e-4 sd, 1.5e-4)
    eq = []
    for j in range(0, C, C // 16):
        sl = slice(wl.cell_off[j], wl.cell_off[j + 1])
        r = oracle.em_cell(dict(wl.params, tol=0.0, max_sweeps=int(g["sweeps"][j])),
                           wl.v[:, sl].T, wl.alpha[sl], cell=j)
        assert r["K"] == g["K"][j], j
        eq.append(param_errors(pair_up(g["params"][j][:g["K"][j]], r["params"][:r["K"]], D),
                               r["params"][:r["K"]], D))
    eq = np.array(eq)
    assert np.all(eq <= np.array([1e-4, 1e-3, 1e-3])), eq.max(axis=0)
