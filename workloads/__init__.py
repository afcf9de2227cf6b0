"""Seeded synthetic particle workloads for the GM checkpoint-restart path.

This module only *generates inputs*: per-cell particle positions, velocities
and weights in CSR order, plus the method parameters each workload is run
with.  It holds none of the method's arithmetic, so both the FP64 oracle and
the CUDA path may consume what it produces.

The shapes follow the paper's two test families (Sec. 3): the 1D-1V
electrostatic two-stream problem (Sec. 3.1: L = 2*pi, counter-streaming
beams) and the electromagnetic Weibel problem with anisotropic temperature
(Sec. 3.2: v_thx = 0.1, v_thy,z = 0.3, i.e. T_perp/T_par = 9).  The paper's
own simulation states are not available, so seeded Maxwellian mixtures with
those shapes stand in for them.

Layout of every workload (all numpy arrays):
  cell_off [C+1] int64   CSR offsets; particles of cell j are
                         cell_off[j] .. cell_off[j+1]-1
  x        [Ntot] f64    absolute positions, x in [j*dx, (j+1)*dx)
  v        [D, Ntot]     velocities, SoA, float32 or float64
  alpha    [Ntot] f64    particle weights
  y        [Ntot] f64    (2D meshes only) second coordinate; cells are
                         numbered j = jy * Cx + jx
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GEN_SEED_BASE = 20071227


@dataclass
class Workload:
    name: str
    cell_off: np.ndarray
    x: np.ndarray
    v: np.ndarray
    alpha: np.ndarray
    params: dict = field(default_factory=dict)
    y: np.ndarray | None = None

    @property
    def C(self) -> int:
        return int(self.cell_off.shape[0] - 1)

    @property
    def ntot(self) -> int:
        return int(self.cell_off[-1])

    @property
    def D(self) -> int:
        return int(self.v.shape[0])

    def counts(self) -> np.ndarray:
        return np.diff(self.cell_off)


def method_params(D, Kmax, shape_order, L, seed=1, tol=1e-6, max_sweeps=1000,
                  q=1.0, recon_seed=2):
    """Plain parameter dict of the method (no arithmetic)."""
    return dict(D=D, Kmax=Kmax, shape_order=shape_order, tol=tol,
                max_sweeps=max_sweeps, seed=seed, recon_seed=recon_seed,
                L=float(L), q=float(q))


def _offsets(counts: np.ndarray) -> np.ndarray:
    off = np.zeros(counts.shape[0] + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    return off


def _uniform_positions(rng, counts, dx):
    cell = np.repeat(np.arange(counts.shape[0], dtype=np.int64), counts)
    u = rng.random(cell.shape[0])
    x = (cell + u) * dx
    # keep every particle strictly inside its own cell
    hi = np.nextafter((cell + 1) * dx, -np.inf)
    return np.minimum(x, hi)


def two_stream_1d1v(C=32, ppc=1024, drift=0.2, vth=0.05, eps=0.05,
                    L=2 * math.pi, seed=GEN_SEED_BASE + 0, v_dtype=np.float64):
    """1D-1V electrostatic two-stream cells (Sec. 3.1 shape).

    Positions: uniform in each cell, accepted with probability
    (1 + eps*cos(2*pi*x/L)) / (1 + eps) so that every cell keeps exactly
    ``ppc`` particles.  Velocities: equal mixture of N(+drift, vth^2) and
    N(-drift, vth^2).  Weights 1.
    """
    rng = np.random.default_rng(seed)
    dx = L / C
    xs = []
    for j in range(C):
        got = []
        need = ppc
        while need > 0:
            cand = (j + rng.random(2 * need + 16)) * dx
            acc = rng.random(cand.shape[0]) * (1 + eps) < 1 + eps * np.cos(2 * math.pi * cand / L)
            take = cand[acc][:need]
            got.append(take)
            need -= take.shape[0]
        xj = np.concatenate(got)
        xj = np.minimum(xj, np.nextafter((j + 1) * dx, -np.inf))
        xs.append(xj)
    x = np.concatenate(xs)
    n = x.shape[0]
    sign = np.where(rng.random(n) < 0.5, 1.0, -1.0)
    v = (sign * drift + vth * rng.standard_normal(n)).astype(v_dtype)[None, :]
    counts = np.full(C, ppc, dtype=np.int64)
    return Workload("two_stream_1d1v", _offsets(counts), x, np.ascontiguousarray(v),
                    np.ones(n), method_params(1, 8, 1, L))


def mixture_1d1v(C=4096, mean_n=2000, clip=(200, 8000), counts="poisson",
                 seed=GEN_SEED_BASE + 1, v_dtype=np.float32, Kmax=8,
                 shape_order=2):
    """1D-1V batched cells: each cell holds a random mixture of 1-4 drifting
    Maxwellians (drifts U[-0.5, 0.5], vth U[0.02, 0.1], weights Dirichlet(1)).

    ``counts`` = "poisson" draws N_j ~ Poisson(mean_n); "uniform" draws
    N_j ~ U[clip]; an int array gives the counts directly.  Counts are clipped
    to ``clip``.  Mesh: dx = 1, L = C.
    """
    rng = np.random.default_rng(seed)
    if isinstance(counts, str):
        if counts == "poisson":
            n = rng.poisson(mean_n, C)
        elif counts == "uniform":
            n = rng.integers(clip[0], clip[1] + 1, C)
        else:
            raise ValueError(counts)
        n = np.clip(n, clip[0], clip[1]).astype(np.int64)
    else:
        n = np.asarray(counts, dtype=np.int64)
        assert n.shape[0] == C
    m = rng.integers(1, 5, C)
    drift = rng.uniform(-0.5, 0.5, (C, 4))
    vth = rng.uniform(0.02, 0.1, (C, 4))
    # Dirichlet(1, ..., 1) over the first m components: normalised
    # exponential draws
    w = rng.exponential(1.0, (C, 4)) * (np.arange(4)[None, :] < m[:, None])
    w /= w.sum(axis=1, keepdims=True)
    cw = np.cumsum(w, axis=1)
    cw[:, -1] = 1.0 + 1e-12
    cell = np.repeat(np.arange(C), n)
    u = rng.random(cell.shape[0])
    comp = (u[:, None] >= cw[cell]).sum(axis=1)
    comp = np.minimum(comp, m[cell] - 1)
    v = drift[cell, comp] + vth[cell, comp] * rng.standard_normal(cell.shape[0])
    x = _uniform_positions(rng, n, 1.0)
    return Workload("mixture_1d1v", _offsets(n), x,
                    np.ascontiguousarray(v.astype(v_dtype)[None, :]),
                    np.ones(cell.shape[0]),
                    method_params(1, Kmax, shape_order, float(C)))


def _bimaxwellian_3v(rng, n):
    C = n.shape[0]
    ratio = rng.uniform(4.0, 25.0, C)
    vpar = np.full(C, 0.1)
    vperp = vpar * np.sqrt(ratio)
    drift = rng.uniform(-0.1, 0.1, (C, 3))
    cell = np.repeat(np.arange(C), n)
    z = rng.standard_normal((3, cell.shape[0]))
    v = np.empty((3, cell.shape[0]))
    v[0] = drift[cell, 0] + vpar[cell] * z[0]
    v[1] = drift[cell, 1] + vperp[cell] * z[1]
    v[2] = drift[cell, 2] + vperp[cell] * z[2]
    return v


def bimaxwellian_1d3v(C=2048, ppc=4000, counts=None, seed=GEN_SEED_BASE + 2,
                      v_dtype=np.float32, Kmax=10, shape_order=2):
    """1D-3V electromagnetic-shaped cells: a bi-Maxwellian per cell with the
    parallel axis along x (v_th,par = 0.1), random anisotropy
    T_perp/T_par ~ U[4, 25] and a random drift U[-0.1, 0.1]^3 (the Weibel
    set-up of Sec. 3.2 has T_perp/T_par = 9).  Mesh: dx = 1, L = C.
    """
    rng = np.random.default_rng(seed)
    n = np.full(C, ppc, dtype=np.int64) if counts is None else np.asarray(counts, dtype=np.int64)
    v = _bimaxwellian_3v(rng, n)
    x = _uniform_positions(rng, n, 1.0)
    return Workload("bimaxwellian_1d3v", _offsets(n), x,
                    np.ascontiguousarray(v.astype(v_dtype)), np.ones(x.shape[0]),
                    method_params(3, Kmax, shape_order, float(C)))


def lognormal_1d3v(C=262144, median=512, sigma=0.47, clip=(16, 8192),
                   seed=GEN_SEED_BASE + 4, v_dtype=np.float32, Kmax=10):
    """Full-scale 1D-3V cells with log-normal particle counts
    N_j = round(median * exp(sigma * Z)) clipped to ``clip``; velocities as in
    :func:`bimaxwellian_1d3v`."""
    rng = np.random.default_rng(seed)
    n = np.clip(np.rint(median * np.exp(sigma * rng.standard_normal(C))),
                clip[0], clip[1]).astype(np.int64)
    v = _bimaxwellian_3v(rng, n)
    x = _uniform_positions(rng, n, 1.0)
    return Workload("lognormal_1d3v", _offsets(n), x,
                    np.ascontiguousarray(v.astype(v_dtype)), np.ones(x.shape[0]),
                    method_params(3, Kmax, 2, float(C)))


def weibel_2d3v(Cx=16, Cy=16, ppc=512, counts=None, Lx=10.0, Ly=10.0, eps=0.05,
                seed=GEN_SEED_BASE + 5, v_dtype=np.float32, Kmax=8, shape_order=2):
    """2D-3V cells of the Weibel set-up of Sec. 3.2: a doubly periodic
    Lx x Ly = 10 x 10 domain (skin depths) of Cx x Cy cells (16 x 16 and
    128-1024 particles per cell in the paper), v_th,x = 0.1 and
    v_th,y = v_th,z = 0.3 (T_perp/T_par = 9), here relaxed per cell by a
    factor U[0.8, 1] on the perpendicular speed with a drift N(0, 0.01^2)^3
    (a state late in the linear phase).  Positions: uniform in each cell,
    accepted with probability (1 + eps cos(2 pi x/Lx) cos(2 pi y/Ly)) /
    (1 + eps) so that every cell keeps its count.  Cells are numbered
    j = jy * Cx + jx; params carries Cx, Cy, Lx, Ly."""
    rng = np.random.default_rng(seed)
    C = Cx * Cy
    n = np.full(C, ppc, dtype=np.int64) if counts is None else np.asarray(counts, dtype=np.int64)
    dx, dy = Lx / Cx, Ly / Cy
    cell = np.repeat(np.arange(C, dtype=np.int64), n)
    jx, jy = cell % Cx, cell // Cx
    x = np.empty(cell.shape[0])
    y = np.empty(cell.shape[0])
    todo = np.arange(cell.shape[0])
    while todo.size:
        ux, uy = rng.random(todo.size), rng.random(todo.size)
        xt = (jx[todo] + ux) * dx
        yt = (jy[todo] + uy) * dy
        acc = rng.random(todo.size) * (1 + eps) < 1 + eps * np.cos(2 * math.pi * xt / Lx) * np.cos(
            2 * math.pi * yt / Ly)
        x[todo[acc]] = np.minimum(xt[acc], np.nextafter((jx[todo[acc]] + 1) * dx, -np.inf))
        y[todo[acc]] = np.minimum(yt[acc], np.nextafter((jy[todo[acc]] + 1) * dy, -np.inf))
        todo = todo[~acc]
    vperp = 0.3 * rng.uniform(0.8, 1.0, C)
    drift = 0.01 * rng.standard_normal((C, 3))
    z = rng.standard_normal((3, cell.shape[0]))
    v = np.empty((3, cell.shape[0]))
    v[0] = drift[cell, 0] + 0.1 * z[0]
    v[1] = drift[cell, 1] + vperp[cell] * z[1]
    v[2] = drift[cell, 2] + vperp[cell] * z[2]
    params = method_params(3, Kmax, shape_order, Lx)
    params.update(Cx=int(Cx), Cy=int(Cy), Lx=float(Lx), Ly=float(Ly))
    return Workload("weibel_2d3v", _offsets(n), x, np.ascontiguousarray(v.astype(v_dtype)),
                    np.ones(x.shape[0]), params, y)


def with_weights(wl: Workload, seed=7, lo=0.5, hi=1.5) -> Workload:
    """Copy of ``wl`` with non-identical weights alpha ~ U[lo, hi] (the
    variable-weight case of Sec. 3.2)."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(lo, hi, wl.ntot)
    return Workload(wl.name + "_varw", wl.cell_off, wl.x, wl.v, a, dict(wl.params), wl.y)


# Named workloads: the first is small enough for the oracle to fit in
# seconds; the others are the batched / 3V / full-scale cases.
def mixture_lifted_3v(C=4096, mean_n=2000, clip=(200, 8000), seed=GEN_SEED_BASE + 6,
                      v_dtype=np.float32, Kmax=10, shape_order=2):
    """The 1D-1V batch's cells lifted to 3V: each cell a random mixture of 1-4
    Maxwellians drifting along x (drifts U[-0.5, 0.5], Dirichlet(1) weights)
    with isotropic thermal speed vth U[0.02, 0.1] in x, y and z; counts
    Poisson(mean_n) clipped to ``clip``.  Mesh: dx = 1, L = C."""
    rng = np.random.default_rng(seed)
    n = np.clip(rng.poisson(mean_n, C), clip[0], clip[1]).astype(np.int64)
    m = rng.integers(1, 5, C)
    drift = rng.uniform(-0.5, 0.5, (C, 4))
    vth = rng.uniform(0.02, 0.1, (C, 4))
    w = rng.exponential(1.0, (C, 4)) * (np.arange(4)[None, :] < m[:, None])
    w /= w.sum(axis=1, keepdims=True)
    cw = np.cumsum(w, axis=1)
    cw[:, -1] = 1.0 + 1e-12
    cell = np.repeat(np.arange(C), n)
    u = rng.random(cell.shape[0])
    comp = np.minimum((u[:, None] >= cw[cell]).sum(axis=1), m[cell] - 1)
    th = vth[cell, comp]
    z = rng.standard_normal((3, cell.shape[0]))
    v = np.empty((3, cell.shape[0]))
    v[0] = drift[cell, comp] + th * z[0]
    v[1] = th * z[1]
    v[2] = th * z[2]
    x = _uniform_positions(rng, n, 1.0)
    return Workload("mixture_lifted_3v", _offsets(n), x, np.ascontiguousarray(v.astype(v_dtype)),
                    np.ones(cell.shape[0]), method_params(3, Kmax, shape_order, float(C)))


def get(name: str, **kw) -> Workload:
    if name == "two_stream_1d1v":
        return two_stream_1d1v(**kw)
    if name == "mixture_1d1v":
        return mixture_1d1v(**kw)
    if name == "mixture_1d1v_uniform":
        return mixture_1d1v(counts="uniform", **kw)
    if name == "bimaxwellian_1d3v":
        return bimaxwellian_1d3v(**kw)
    if name == "lognormal_1d3v":
        return lognormal_1d3v(**kw)
    if name == "weibel_2d3v":
        return weibel_2d3v(**kw)
    if name == "mixture_lifted_3v":
        return mixture_lifted_3v(**kw)
    raise KeyError(name)


def resample_offsets(cell_off: np.ndarray) -> np.ndarray:
    """Output CSR offsets with N'_j = N_j (the restart keeps each cell's
    particle count)."""
    return np.array(cell_off, dtype=np.int64, copy=True)
