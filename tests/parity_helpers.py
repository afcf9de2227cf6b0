"""Shared parity measures for EM fits (GPU against the FP64 oracle).

A cell agrees naturally when it selects the same K and its penalised
log-likelihood is within 1e-5 (relative) of the oracle's; the tests assert
the natural rates (K alone, and K with lnL).  With the default FP64 M-step
the GPU's convergence test follows the oracle's stopping sweep (its
log-likelihood is summed in FP64 and corrected for the rounding of the
FP32 E-step constants), so the natural rates are the gate.

As a diagnostic (printed, not asserted) a disagreeing cell is also
compared at equal sweep counts: the oracle is rerun for exactly the GPU's
number of sweeps (tol = 0):
  * a cell the GPU stopped by the convergence test must then agree (same
    K, lnL within 1e-5);
  * a cell that ran into max_sweeps is unconverged on both sides: its
    trajectory is still moving along a flat direction of the likelihood,
    where FP32 and FP64 rounding make the two sides drift a number of
    sweeps apart.  It agrees when K is the same and the lnL difference is
    at most lag_sweeps times the oracle's own change of L over its last
    sweep (the two trajectories are at most that many sweeps apart).
"""
import numpy as np

import oracle


def equal_sweep_agreement(params, v_cell, alpha_cell, cell, K_gpu, lnL_gpu, sweeps_gpu, status_gpu,
                          lag_sweeps=200):
    s = max(int(sweeps_gpu), 1)
    p = dict(params, tol=0.0, max_sweeps=s)
    r = oracle.em_cell(p, v_cell, alpha_cell, cell=int(cell), trace_cap=s + 2)
    diff = abs(lnL_gpu - r["lnL"])
    rel = diff / abs(r["lnL"])
    if r["K"] != K_gpu:
        return False, rel
    if rel <= 1e-5:
        return True, rel
    if status_gpu & oracle.ST_EM_MAXSWEEPS:
        tr = r["Ltrace"]
        dL = abs(tr[-1] - tr[-2]) if len(tr) >= 2 else 0.0
        return bool(diff <= lag_sweeps * dL), rel
    return False, rel


def same_k(g, ref):
    """per-cell flags: the same selected component count"""
    return np.asarray(g["K"]) == np.asarray(ref["K"])


def agreement(g, ref, wl, cells=None):
    """(natural agreement flags, agreement flags after the equal-sweep rule)
    for GPU results g and oracle results ref (dicts of per-cell arrays)."""
    rel = np.abs(g["lnL"] - ref["lnL"]) / np.maximum(np.abs(ref["lnL"]), 1e-300)
    agree = (g["K"] == ref["K"]) & (rel <= 1e-5)
    eq = agree.copy()
    for i in np.flatnonzero(~agree):
        j = int(cells[i]) if cells is not None else int(i)
        sl = slice(wl.cell_off[j], wl.cell_off[j + 1])
        eq[i], _ = equal_sweep_agreement(wl.params, wl.v[:, sl].T, wl.alpha[sl], j, int(g["K"][i]),
                                         float(g["lnL"][i]), int(g["sweeps"][i]), int(g["status"][i]))
    return agree, eq
