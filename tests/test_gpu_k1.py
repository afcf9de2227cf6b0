"""The closed-form pre-pass of gm_compress_from (cells whose supplied start
has one valid component, empty and degenerate cells) against the FP64
oracle's one-component fit, through the C ABI: the weight, mean and
covariance are the cell's moments, eq. (lnL-GM) its closed form.

Equal-weight cells take the exact integer-pipe sums (at most 2^14
particles), the others FP64 sums; both are compared, as are a cell above
2^14 particles, an empty cell and a degenerate one."""
import os

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


def batch(D, weights):
    rng = np.random.default_rng(30 + D)
    C = 200
    counts = rng.integers(2, 1500, C)
    counts[5] = 0            # empty
    counts[9] = 17000        # above the integer path's 2^14 particles
    counts[11] = 1           # one particle: degenerate
    if D == 1:
        wl = workloads.mixture_1d1v(C=C, counts=counts, seed=41, Kmax=4)
    else:
        wl = workloads.bimaxwellian_1d3v(C=C, counts=counts, seed=42, Kmax=4)
    if weights == "variable":
        wl = workloads.with_weights(wl)
    # a cell whose velocities span 40 binades (the smallest below the
    # integer path's exact range)
    a, b = wl.cell_off[20], wl.cell_off[21]
    v = wl.v.copy()
    v[:, a:b] *= np.float32(2.0) ** rng.integers(-40, 1, b - a).astype(np.float32)
    return workloads.Workload(wl.name, wl.cell_off, wl.x, v, wl.alpha, wl.params)


@pytest.mark.parametrize("weights", ["equal", "variable"])
@pytest.mark.parametrize("D", [1, 3])
def test_one_component_prepass_matches_oracle(gm, D, weights):
    wl = batch(D, weights)
    p1 = dict(wl.params, Kmax=1)
    ref = oracle.compress(p1, wl.cell_off, wl.x, wl.v, wl.alpha, nthreads=os.cpu_count() or 4)
    P = 1 + D + D * (D + 1) // 2
    Kmax = wl.params["Kmax"]
    # the supplied start: the oracle's own one-component fit in slot 0 (a
    # valid component), nothing in the other slots
    init = np.zeros((wl.C, Kmax, P))
    init[:, 0, :] = ref["params"][:, 0, :]
    init_K = np.ones(wl.C, dtype=np.int32)
    bad = ref["K"] == 0  # empty cell: any start
    init[bad, 0, :] = 0.0
    init[bad, 0, 0] = 1.0
    cfg = gm.config(wl.params)
    out = gm.gm_compress(cfg, dev(wl.cell_off), dev(wl.x), dev(wl.v), dev(wl.alpha),
                         init_K=dev(init_K), init_params=dev(init))
    g = {k: t.cpu().numpy() for k, t in out.items() if t is not None}
    np.testing.assert_array_equal(g["K"], ref["K"])
    np.testing.assert_array_equal(g["status"], ref["status"])
    np.testing.assert_allclose(g["W"], ref["W"], rtol=1e-14)
    ok = ref["K"] == 1
    live = ok & ((ref["status"] & oracle.ST_DEGENERATE) == 0)
    assert np.all(g["sweeps"][live] == 1) and np.all(g["kwork"][live] == 0)
    for j in np.flatnonzero(ok):
        a, b = g["params"][j, 0], ref["params"][j, 0]
        sd = np.sqrt(np.abs(b[1 + D:][[0, 3, 5]] if D == 3 else b[2:3]))
        scale = np.abs(b[1:1 + D]) + sd + 1e-300
        assert a[0] == 1.0
        assert np.all(np.abs(a[1:1 + D] - b[1:1 + D]) <= 1e-13 * scale), (j, a, b)
        cs = (np.outer(sd, sd)[np.triu_indices(D)] if D == 3 else sd ** 2) + 1e-300
        assert np.all(np.abs(a[1 + D:] - b[1 + D:]) <= 1e-12 * cs), (j, a, b)
    # the closed form against the oracle's sum of N log-densities: both FP64,
    # the sum's rounding ~1e-16 N (3V cells' |L| can be a few % of N)
    n = np.diff(wl.cell_off)[live]
    err = np.abs(g["lnL"][live] - ref["lnL"][live]) / (np.abs(ref["lnL"][live]) + n)
    assert err.max() <= 1e-12, err.max()
    # exact moments: the mixture's against the particles' (both on the GPU)
    m0 = gm.gm_moments(cfg, dev(wl.cell_off), dev(wl.x), dev(wl.v), dev(wl.alpha))
    mm = gm.gm_mixture_moments(cfg, out["K"], out["params"], out["W"])
    E0, Em = m0["E"].cpu().numpy(), mm["E"].cpu().numpy()
    assert np.all(np.abs(Em[ok] - E0[ok]) <= 1e-12 * E0[ok])
