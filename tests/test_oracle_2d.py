"""Pins of the oracle's 2D mesh (Sec. 2.4.1 in two dimensions, the geometry
of the 2D-3V Weibel runs of Sec. 3.2), each against something other than
the oracle's own 2D code: a deposit written here with scipy's B-spline
basis elements, the reduction of a one-row mesh to the 1D oracle (whose
mass-matrix solve is a cyclic tridiagonal elimination, not the dense 2D
one), exact charge on every node and exact per-cell momentum and energy,
and the uniformity of the sampled positions."""
import numpy as np
import pytest
from scipy import interpolate, stats

import oracle
import workloads

KNOTS = {1: [-1.0, 0.0, 1.0], 2: [-1.5, -0.5, 0.5, 1.5]}


def shape(order, s):
    b = interpolate.BSpline.basis_element(KNOTS[order], extrapolate=False)
    return np.nan_to_num(b(np.asarray(s, dtype=np.float64)))


def deposit_ref(p, cell_off, x, y, alpha):
    """rho_i = q / (dx dy) sum_p alpha_p S(x_i - x_p) S(y_i - y_p), by brute
    force over the 3 x 3 nodes around each particle's cell"""
    Cx, Cy, Lx, Ly = p["Cx"], p["Cy"], p["Lx"], p["Ly"]
    dx, dy = Lx / Cx, Ly / Cy
    cell = np.repeat(np.arange(Cx * Cy), np.diff(cell_off))
    jx, jy = cell % Cx, cell // Cx
    rho = np.zeros(Cx * Cy)
    for b in (-1, 0, 1):
        for a in (-1, 0, 1):
            ix, iy = jx + a, jy + b
            w = shape(p["shape_order"], ((ix + 0.5) * dx - x) / dx) * \
                shape(p["shape_order"], ((iy + 0.5) * dy - y) / dy)
            np.add.at(rho, (iy % Cy) * Cx + ix % Cx, p["q"] * alpha * w / (dx * dy))
    return rho


@pytest.mark.parametrize("order", [1, 2])
def test_deposit_matches_scipy_bsplines(order):
    wl = workloads.with_weights(workloads.weibel_2d3v(Cx=5, Cy=3, ppc=40, shape_order=order, seed=61))
    p = dict(wl.params, q=-1.5)
    rho = oracle.deposit2d(p, wl.cell_off, wl.x, wl.y, wl.alpha)
    ref = deposit_ref(p, wl.cell_off, wl.x, wl.y, wl.alpha)
    np.testing.assert_allclose(rho, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
    # partition of unity: total charge
    dV = (p["Lx"] / p["Cx"]) * (p["Ly"] / p["Cy"])
    assert rho.sum() * dV == pytest.approx(p["q"] * wl.alpha.sum(), rel=1e-13)


def test_single_particle_in_a_corner_wraps_both_ways():
    """One particle near the lower-left corner of cell (0, 0) reaches the
    nodes of the last column and the last row (periodic in x and y)."""
    p = dict(D=3, Kmax=1, shape_order=2, L=4.0, q=1.0, Cx=4, Cy=3, Lx=4.0, Ly=3.0)
    cell_off = np.array([0, 1] + [1] * 11, dtype=np.int64)
    x, y = np.array([0.1]), np.array([0.2])
    rho = oracle.deposit2d(p, cell_off, x, y, np.ones(1)).reshape(3, 4)
    wx = {-1: 0.5 * (1.5 - 0.6) ** 2, 0: 0.75 - 0.4 ** 2, 1: 0.5 * (1.5 - 1.4) ** 2}  # nodes -1, 0, 1
    wy = {-1: 0.5 * (1.5 - 0.7) ** 2, 0: 0.75 - 0.3 ** 2, 1: 0.5 * (1.5 - 1.3) ** 2}
    for b in (-1, 0, 1):
        for a in (-1, 0, 1):
            assert rho[b % 3, a % 4] == pytest.approx(wx[a] * wy[b], rel=1e-14)
    assert rho[1, 2] == 0.0  # node (ix 2, iy 1) is out of reach


def _fit(wl):
    return oracle.compress(wl.params, wl.cell_off, wl.x, wl.v, wl.alpha, nthreads=4)


def test_reconstruction_matches_charge_momentum_and_energy():
    wl = workloads.with_weights(workloads.weibel_2d3v(Cx=8, Cy=6, ppc=200, seed=62))
    p = dict(wl.params, q=2.5)
    fit = _fit(wl)
    rho_t = deposit_ref(p, wl.cell_off, wl.x, wl.y, wl.alpha)
    out_off = workloads.resample_offsets(wl.cell_off)
    r = oracle.reconstruct2d(p, fit["K"], fit["params"], fit["W"], rho_t, out_off, nthreads=4)
    rho = deposit_ref(p, out_off, r["x"], r["y"], r["alpha"])
    np.testing.assert_allclose(rho, rho_t, rtol=0, atol=1e-12 * np.abs(rho_t).max())
    mm = oracle.mixture_moments(p, fit["K"], fit["params"], fit["W"])
    m1 = oracle.moments(p, out_off, r["x"], r["v"], r["alpha"])
    proj = (r["status"] & oracle.ST_PROJ_SKIPPED) == 0
    assert proj.mean() > 0.9
    scale = np.array([(np.abs(r["v"][:, s:e]) * r["alpha"][s:e]).sum()
                      for s, e in zip(out_off[:-1], out_off[1:])])
    assert np.all(np.abs(m1["p"] - mm["p"]).max(1)[proj] <= 1e-12 * scale[proj])
    assert np.all((np.abs(m1["E"] - mm["E"]) / mm["E"])[proj] <= 1e-12)
    # positions stay inside their cells
    Cx, dx, dy = p["Cx"], p["Lx"] / p["Cx"], p["Ly"] / p["Cy"]
    cell = np.repeat(np.arange(wl.C), np.diff(out_off))
    assert np.all(np.floor(r["x"] / dx) == cell % Cx)
    assert np.all(np.floor(r["y"] / dy) == cell // Cx)


@pytest.mark.parametrize("order", [1, 2])
def test_gauss_correction_is_the_9_point_mass_matrix_equation(order):
    """Sec. 2.4.1 on the 2D mesh: every resampled particle of cell j gets the
    same dA_j, and dA solves M dA = dx dy (rho' - rho) with the 9-point
    M_ij = q sum_{p in j} S(x_i - x_p) S(y_i - y_p), built here from scipy's
    B-spline basis; its column sums are q N'_j."""
    wl = workloads.with_weights(workloads.weibel_2d3v(Cx=5, Cy=4, ppc=60, shape_order=order, seed=64))
    p = dict(wl.params, q=-1.2)
    fit = _fit(wl)
    rho_t = deposit_ref(p, wl.cell_off, wl.x, wl.y, wl.alpha)
    out_off = workloads.resample_offsets(wl.cell_off)
    r = oracle.reconstruct2d(p, fit["K"], fit["params"], fit["W"], rho_t, out_off, nthreads=4)
    Cx, Cy = p["Cx"], p["Cy"]
    dx, dy = p["Lx"] / Cx, p["Ly"] / Cy
    C = Cx * Cy
    M = np.zeros((C, C))
    for j in range(C):
        a, b = out_off[j], out_off[j + 1]
        base = fit["W"][j] / (b - a)
        np.testing.assert_allclose(r["alpha"][a:b] - base, r["dA"][j], rtol=0, atol=1e-13 * base)
        for i in range(C):
            ix, iy = i % Cx, i // Cx
            ddx = ((ix + 0.5) * dx - r["x"][a:b] + p["Lx"] / 2) % p["Lx"] - p["Lx"] / 2
            ddy = ((iy + 0.5) * dy - r["y"][a:b] + p["Ly"] / 2) % p["Ly"] - p["Ly"] / 2
            M[i, j] = p["q"] * (shape(order, ddx / dx) * shape(order, ddy / dy)).sum()
        assert M[:, j].sum() == pytest.approx(p["q"] * (b - a), rel=1e-13)
    raw = np.repeat(fit["W"] / np.diff(out_off), np.diff(out_off))
    rho_raw = deposit_ref(p, out_off, r["x"], r["y"], raw)
    rhs = dx * dy * (rho_t - rho_raw)
    res = M @ r["dA"] - rhs
    assert np.abs(res).max() <= 1e-12 * dx * dy * np.abs(rho_t).max()
    assert np.abs(rhs).max() > 1e-6 * dx * dy * np.abs(rho_t).max()


def test_one_row_mesh_is_the_1d_oracle():
    """Cy = 1: every particle's y weights wrap onto the one row and sum to
    one, so M and the right-hand side are the 1D ones: dA equals the 1D
    oracle's (cyclic tridiagonal solve) and x the 1D sampler's."""
    wl2 = workloads.weibel_2d3v(Cx=12, Cy=1, ppc=150, seed=63)
    p2 = dict(wl2.params)
    fit = _fit(wl2)
    rho2 = oracle.deposit2d(p2, wl2.cell_off, wl2.x, wl2.y, wl2.alpha)
    p1 = dict(p2, L=p2["Lx"])
    rho1 = oracle.moments(p1, wl2.cell_off, wl2.x, wl2.v, wl2.alpha)["rho"]
    np.testing.assert_allclose(rho2 * p2["Ly"], rho1, rtol=1e-13)
    r2 = oracle.reconstruct2d(p2, fit["K"], fit["params"], fit["W"], rho2, wl2.cell_off)
    r1 = oracle.reconstruct(p1, fit["K"], fit["params"], fit["W"], rho1, wl2.cell_off)
    np.testing.assert_array_equal(r2["x"], r1["x"])
    np.testing.assert_allclose(r2["dA"], r1["dA"], rtol=1e-11, atol=1e-13 * np.abs(r1["dA"]).max())
    np.testing.assert_allclose(r2["v"], r1["v"], rtol=1e-11, atol=1e-13)


def test_one_column_mesh_solves_the_1d_system_along_y():
    """Cx = 1: M is the cyclic tridiagonal matrix of the y positions
    (assembled here with scipy, solved with numpy)."""
    wl = workloads.weibel_2d3v(Cx=1, Cy=9, ppc=120, seed=64)
    p = dict(wl.params)
    fit = _fit(wl)
    rho_t = oracle.deposit2d(p, wl.cell_off, wl.x, wl.y, wl.alpha)
    r = oracle.reconstruct2d(p, fit["K"], fit["params"], fit["W"], rho_t, wl.cell_off)
    Cy, dy, dx = p["Cy"], p["Ly"] / p["Cy"], p["Lx"]
    M = np.zeros((Cy, Cy))
    cell = np.repeat(np.arange(Cy), np.diff(wl.cell_off))
    for b in (-1, 0, 1):
        w = shape(2, ((cell + b + 0.5) * dy - r["y"]) / dy)
        np.add.at(M, ((cell + b) % Cy, cell), p["q"] * w)
    alpha0 = fit["W"][cell] / np.diff(wl.cell_off)[cell]
    rho0 = deposit_ref(p, wl.cell_off, r["x"], r["y"], alpha0)
    dA = np.linalg.solve(M, dx * dy * (rho_t - rho0))
    np.testing.assert_allclose(r["dA"], dA, rtol=1e-10, atol=1e-13 * np.abs(dA).max())


def test_sampled_positions_are_uniform_in_their_cells():
    wl = workloads.weibel_2d3v(Cx=4, Cy=4, ppc=3000, seed=65)
    p = dict(wl.params)
    fit = _fit(wl)
    rho_t = oracle.deposit2d(p, wl.cell_off, wl.x, wl.y, wl.alpha)
    r = oracle.reconstruct2d(p, fit["K"], fit["params"], fit["W"], rho_t, wl.cell_off)
    dx, dy = p["Lx"] / 4, p["Ly"] / 4
    fx = r["x"] / dx - np.floor(r["x"] / dx)
    fy = r["y"] / dy - np.floor(r["y"] / dy)
    assert stats.kstest(fx, "uniform").pvalue > 1e-3
    assert stats.kstest(fy, "uniform").pvalue > 1e-3
    assert abs(np.corrcoef(fx, fy)[0, 1]) < 0.02


def test_a_cell_without_resampled_particles_is_flagged():
    wl = workloads.weibel_2d3v(Cx=5, Cy=4, ppc=100, seed=66)
    p = dict(wl.params)
    fit = _fit(wl)
    rho_t = oracle.deposit2d(p, wl.cell_off, wl.x, wl.y, wl.alpha)
    counts = np.diff(wl.cell_off).copy()
    counts[7] = 0
    out_off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    r = oracle.reconstruct2d(p, fit["K"], fit["params"], fit["W"], rho_t, out_off)
    assert r["status"][7] & oracle.ST_MM_EMPTY_COL
    assert np.all((r["status"][np.arange(20) != 7] & oracle.ST_MM_EMPTY_COL) == 0)
    # every node away from the empty cell's own equation holds its charge
    rho = deposit_ref(p, out_off, r["x"], r["y"], r["alpha"])
    ok = np.arange(20) != 7
    np.testing.assert_allclose(rho[ok], rho_t[ok], rtol=0, atol=1e-12 * np.abs(rho_t).max())
