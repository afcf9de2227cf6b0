"""The seeded input generators follow their stated recipe (CPU): CSR layout,
positions inside their own cells, dtypes, determinism, and the statistics
of the particle counts and velocity distributions, each checked against
what the recipe fixes with numpy / scipy."""
import math

import numpy as np
import pytest

import workloads


def _cells(wl):
    return np.repeat(np.arange(wl.C), wl.counts())


def _check_layout(wl, D, v_dtype, dx):
    off = wl.cell_off
    assert off.dtype == np.int64 and off[0] == 0 and np.all(np.diff(off) >= 0)
    n = wl.ntot
    assert wl.x.shape == (n,) and wl.x.dtype == np.float64
    assert wl.alpha.shape == (n,) and wl.alpha.dtype == np.float64
    assert wl.v.shape == (D, n) and wl.v.dtype == v_dtype and wl.v.flags.c_contiguous
    assert wl.D == D and wl.params["D"] == D
    if dx is not None:  # 1D mesh: x in [j dx, (j + 1) dx) for the particle's cell j
        cell = _cells(wl)
        assert np.all(wl.x >= cell * dx) and np.all(wl.x < (cell + 1) * dx)
        assert wl.params["L"] == pytest.approx(wl.C * dx)


@pytest.mark.parametrize("name,kw,D,dt,dx", [
    ("two_stream_1d1v", dict(C=8, ppc=256), 1, np.float64, 2 * math.pi / 8),
    ("mixture_1d1v", dict(C=64), 1, np.float32, 1.0),
    ("mixture_1d1v_uniform", dict(C=64), 1, np.float32, 1.0),
    ("bimaxwellian_1d3v", dict(C=16, ppc=500), 3, np.float32, 1.0),
    ("lognormal_1d3v", dict(C=256), 3, np.float32, 1.0),
    ("mixture_lifted_3v", dict(C=32, mean_n=300), 3, np.float32, 1.0),
    ("weibel_2d3v", dict(Cx=4, Cy=3, ppc=100), 3, np.float32, None),
])
def test_layout_determinism_and_seeds(name, kw, D, dt, dx):
    a = workloads.get(name, **kw)
    _check_layout(a, D, dt, dx)
    assert np.all(a.alpha == 1.0)
    b = workloads.get(name, **kw)
    for f in ("cell_off", "x", "v", "alpha"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
    c = workloads.get(name, seed=12345, **kw)
    assert not np.array_equal(a.v, c.v)


def test_mixture_counts_poisson_and_uniform():
    # N_j ~ Poisson(2000) clipped to [200, 8000] (the clip never binds)
    wl = workloads.mixture_1d1v()
    n = wl.counts()
    assert wl.C == 4096 and n.min() >= 200 and n.max() <= 8000
    se = math.sqrt(2000 / 4096)
    assert abs(n.mean() - 2000) < 5 * se
    assert 0.9 < n.var() / 2000 < 1.1
    # the stress variant: N_j ~ U{200 .. 8000}
    u = workloads.mixture_1d1v(C=4096, counts="uniform").counts()
    assert u.min() >= 200 and u.max() <= 8000
    assert abs(u.mean() - 4100) < 5 * (7800 / math.sqrt(12 * 4096))


def test_mixture_velocities_are_drifting_maxwellians():
    # every cell is a mixture of 1-4 Maxwellians with drifts in [-0.5, 0.5]
    # and vth in [0.02, 0.1]: its mean lies in the drift range, its spread
    # between the narrowest vth and that of two beams 1 apart, and a cell
    # that is one Maxwellian (the narrowest spread) passes a normality test
    from scipy import stats
    wl = workloads.mixture_1d1v(C=256)
    sd = []
    for j in range(wl.C):
        v = wl.v[0, wl.cell_off[j]:wl.cell_off[j + 1]].astype(np.float64)
        se = 0.6 / math.sqrt(v.size)
        assert -0.5 - 6 * se < v.mean() < 0.5 + 6 * se
        sd.append(v.std())
    sd = np.array(sd)
    assert sd.min() > 0.02 * 0.9 and sd.max() < math.sqrt(0.1 ** 2 + 0.25)
    j = int(np.argmin(sd))
    v = wl.v[0, wl.cell_off[j]:wl.cell_off[j + 1]].astype(np.float64)
    assert stats.normaltest(v).pvalue > 1e-4


def test_two_stream_beams():
    # equal mixture of N(+0.2, 0.05^2) and N(-0.2, 0.05^2), 1024 per cell
    wl = workloads.two_stream_1d1v()
    assert wl.C == 32 and np.all(wl.counts() == 1024)
    assert wl.params["L"] == pytest.approx(2 * math.pi) and wl.params["shape_order"] == 1
    v = wl.v[0]
    n = v.size
    assert abs(np.mean(v > 0) - 0.5) < 5 * 0.5 / math.sqrt(n)
    pos, neg = v[v > 0], v[v < 0]
    assert abs(pos.mean() - 0.2) < 0.002 and abs(neg.mean() + 0.2) < 0.002
    assert abs(pos.std() - 0.05) < 0.002 and abs(neg.std() - 0.05) < 0.002
    # positions: uniform within each cell up to the weak modulation
    from scipy import stats
    dx = wl.params["L"] / wl.C
    frac = wl.x / dx - _cells(wl)
    assert stats.kstest(frac, "uniform").pvalue > 1e-4


def test_bimaxwellian_anisotropy_and_drift():
    # v_th,par = 0.1 along x, T_perp / T_par in [4, 25], drift in [-0.1, 0.1]^3
    wl = workloads.bimaxwellian_1d3v(C=64)
    assert np.all(wl.counts() == 4000) and wl.params["Kmax"] == 10
    for j in range(wl.C):
        v = wl.v[:, wl.cell_off[j]:wl.cell_off[j + 1]].astype(np.float64)
        var = v.var(axis=1)
        assert abs(var[0] / 0.01 - 1) < 0.12
        assert 4 * 0.85 < var[1] / var[0] < 25 * 1.15
        assert abs(var[2] / var[1] - 1) < 0.15
        se = np.sqrt(var / v.shape[1])
        assert np.all(np.abs(v.mean(axis=1)) < 0.1 + 6 * se)


def test_lognormal_counts():
    # N_j = round(512 exp(0.47 Z)) clipped to [16, 8192]: median 512, mean
    # 512 exp(0.47^2 / 2), log-spread 0.47
    n = workloads.lognormal_1d3v(C=8000).counts()
    assert n.min() >= 16 and n.max() <= 8192
    assert abs(np.median(n) / 512 - 1) < 0.03
    assert abs(n.mean() / (512 * math.exp(0.47 ** 2 / 2)) - 1) < 0.03
    assert abs(np.log(n).std() / 0.47 - 1) < 0.04


def test_weibel_2d_cells_and_temperatures():
    # 2D cells numbered jy * Cx + jx; v_th,x = 0.1, v_th,y = v_th,z in
    # 0.3 [0.8, 1]; drift N(0, 0.01^2)
    Cx, Cy = 8, 6
    wl = workloads.weibel_2d3v(Cx=Cx, Cy=Cy, ppc=2000)
    assert wl.params["Cx"] == Cx and wl.params["Cy"] == Cy and wl.C == Cx * Cy
    dx, dy = wl.params["Lx"] / Cx, wl.params["Ly"] / Cy
    cell = _cells(wl)
    jx, jy = cell % Cx, cell // Cx
    assert np.all(wl.x >= jx * dx) and np.all(wl.x < (jx + 1) * dx)
    assert np.all(wl.y >= jy * dy) and np.all(wl.y < (jy + 1) * dy)
    for j in range(wl.C):
        v = wl.v[:, wl.cell_off[j]:wl.cell_off[j + 1]].astype(np.float64)
        sd = v.std(axis=1)
        assert abs(sd[0] / 0.1 - 1) < 0.08
        assert 0.3 * 0.8 * 0.92 < sd[1] < 0.3 * 1.08
        assert abs(sd[2] / sd[1] - 1) < 0.12
        assert np.all(np.abs(v.mean(axis=1)) < 0.05 + 6 * sd / math.sqrt(v.shape[1]))


def test_with_weights_and_resample_offsets():
    base = workloads.weibel_2d3v(Cx=3, Cy=2, ppc=50)
    wl = workloads.with_weights(base)
    assert wl.alpha.min() >= 0.5 and wl.alpha.max() <= 1.5
    assert abs(wl.alpha.mean() - 1.0) < 5 * (1 / math.sqrt(12 * wl.ntot))
    assert wl.x is base.x and wl.v is base.v and wl.y is base.y
    assert wl.cell_off is base.cell_off and wl.params == base.params
    off = workloads.resample_offsets(base.cell_off)
    np.testing.assert_array_equal(off, base.cell_off)
    assert off is not base.cell_off and off.dtype == np.int64


def test_lifted_mixture_is_isotropic_across_y_z_and_drifts_along_x():
    # the 1D-1V batch lifted to 3V: drifts along x only; in y and z every
    # cell is centred (a mixture of zero-mean Maxwellians), with the same
    # spread in y and z, and no correlation between y and z
    wl = workloads.mixture_lifted_3v(C=128, mean_n=2000)
    for j in range(wl.C):
        v = wl.v[:, wl.cell_off[j]:wl.cell_off[j + 1]].astype(np.float64)
        n = v.shape[1]
        sy, sz = v[1].std(), v[2].std()
        assert abs(v[1].mean()) < 6 * sy / math.sqrt(n) and abs(v[2].mean()) < 6 * sz / math.sqrt(n)
        assert 0.02 * 0.85 < sy < 0.1 * 1.15 and abs(sy / sz - 1.0) < 0.25
        assert abs(np.corrcoef(v[1], v[2])[0, 1]) < 6 / math.sqrt(n)
        assert -0.5 - 0.1 < v[0].mean() < 0.5 + 0.1
    assert wl.params["Kmax"] == 10 and wl.params["D"] == 3
