"""The roofline accounting of bench.py on hand-counted cases (CPU): FP32
flops, the special-function (MUFU) operations and the FP64 flops of the EM
kernel, from per-cell particle counts, component steps (kwork), sweeps and
final component counts."""
import numpy as np
import pytest

import bench


def test_fp32_flops_and_peak():
    counts = np.array([10, 20])
    kwork = np.array([4, 9])
    assert bench.em_flops(counts, kwork, 1) == (10 * 4 + 20 * 9) * 30
    assert bench.em_flops(counts, kwork, 3) == (10 * 4 + 20 * 9) * 90
    # 152 SMs x 128 lanes x 2 flops x 2 GHz
    assert bench.fp32_peak_tflops(2000.0) == pytest.approx(77.824)


def test_fp64_flops_per_particle():
    # D = 1: moments 2 (1 + 1 + 1); per component 3 + 2 + 1 + 2 + 2
    assert list(bench.fp64_flops_per_particle(1, np.array([0, 1, 4]))) == [6, 16, 46]
    # D = 3: moments 2 (1 + 3 + 6); per component 3 + 6 + 1 + 6 + 12
    assert list(bench.fp64_flops_per_particle(3, np.array([0, 2]))) == [20, 76]


def test_secondary_rooflines():
    counts = np.array([10, 20])
    K = np.array([2, 3])
    kwork = np.array([4, 9])
    sweeps = np.array([2, 3])
    mufu, f64 = bench.em_secondary_rooflines(counts, K, kwork, sweeps, 1, 1e-3, 2000.0)
    # 10 (3 * 4 + 2) + 20 (3 * 9 + 3) MUFU operations in 1 ms
    assert mufu["achieved"] == pytest.approx(740 / 1e-3 / 1e12)
    assert mufu["peak"] == pytest.approx(152 * 16 * 2000e6 / 1e12)
    assert mufu["frac"] == pytest.approx(mufu["achieved"] / mufu["peak"])
    # 10 (6 + 2 * 10) + 20 (6 + 3 * 10) FP64 flops in 1 ms
    assert f64["achieved"] == pytest.approx(980 / 1e-3 / 1e12)
    assert f64["peak"] == bench.FP64_PEAK_TFLOPS
    assert f64["frac"] == pytest.approx(f64["achieved"] / f64["peak"])


def test_oracle_sample_keeps_the_mesh_spacing():
    # the CPU baseline times the oracle on the first cells of the workload:
    # the sample keeps each cell's particles and the cell width dx
    import workloads
    wl = workloads.mixture_1d1v(C=64, mean_n=300, clip=(50, 600))
    sw = bench.sub_workload(wl, 10)
    n = int(wl.cell_off[10])
    assert sw.C == 10 and sw.ntot == n
    assert (sw.cell_off == wl.cell_off[:11]).all()
    assert (sw.x == wl.x[:n]).all() and (sw.v == wl.v[:, :n]).all() and (sw.alpha == wl.alpha[:n]).all()
    assert sw.params["L"] / sw.C == pytest.approx(wl.params["L"] / wl.C)
    assert sw.v.flags.c_contiguous
    assert bench.sub_workload(wl, 1000).C == wl.C  # capped at the workload


def test_strided_oracle_sample():
    # the CPU baseline times the oracle on every k-th cell: each sampled cell
    # keeps its particles, moved into the sample's own periodic mesh of the
    # same dx, and its index in the batch (which keys its initial picks)
    import workloads
    wl = workloads.mixture_1d1v(C=64, mean_n=300, clip=(50, 600))
    sw, cells = bench.strided_sample(wl, 16)
    assert list(cells) == list(range(0, 64, 4))
    dx = wl.params["L"] / wl.C
    assert sw.C == 16 and sw.params["L"] == pytest.approx(16 * dx)
    for i, j in enumerate(cells):
        a, b = wl.cell_off[j], wl.cell_off[j + 1]
        c, d = sw.cell_off[i], sw.cell_off[i + 1]
        assert d - c == b - a
        assert (sw.v[:, c:d] == wl.v[:, a:b]).all() and (sw.alpha[c:d] == wl.alpha[a:b]).all()
        np.testing.assert_allclose(sw.x[c:d], wl.x[a:b] + (i - j) * dx, rtol=0, atol=1e-12)
        assert np.all((sw.x[c:d] >= i * dx - 1e-12) & (sw.x[c:d] < (i + 1) * dx + 1e-12))
    assert sw.v.flags.c_contiguous
    sw2, cells2 = bench.strided_sample(wl, 1000)  # capped at the workload
    assert sw2.C == wl.C and list(cells2) == list(range(64))


def test_dominant_kernel_roofline_accounting():
    # the roofline of the step's largest traced kernel: algorithmic work per
    # launch / its traced time against the unit's peak (FP64 and the 32-bit
    # lanes from unit counts and the clock, HBM measured)
    counts = np.array([100, 300, 600])
    ctx = dict(counts=counts, D=3, K=np.array([1, 1, 2]), kwork=np.array([0, 0, 10]),
               sweeps=np.array([1, 1, 5]), K0=np.array([1, 1, 2]), sm_mhz=2070.0, hbm_gbs=6780.0,
               bf16_tflops=1916.2, F=576, O=112, ms_compress=1.0)
    assert bench.fp64_peak_tflops(2070.0) == pytest.approx(1.25856)
    assert bench.alu_peak_tops(2070.0) == pytest.approx(152 * 128 * 2.07e9 / 1e12)
    kern = {"em_k1_kernel": {"ms": 2.0, "launches_per_step": 1.0},
            "recon_emit_kernel": {"ms": 1.0, "launches_per_step": 1.0}}
    r = bench.kernel_roofline(kern, ctx)
    # x and alpha of every particle (1000 x 16 bytes), v of the one-component
    # cells (K0 == 1: 400 x 12 bytes), in 2 ms
    assert r["kernel"] == "em_k1_kernel" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx((1000 * 16 + 400 * 12) / 2e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6780.0)
    assert r["secondary"][0]["achieved"] == pytest.approx(400 * 22 / 2e-3 / 1e12)
    kern["recon_emit_kernel"]["ms"] = 3.0
    r = bench.kernel_roofline(kern, ctx)
    # emit: 20 staged + 40 written bytes, 8 FP64 flops per particle
    assert r["kernel"] == "recon_emit_kernel" and r["bound"] == "hbm"
    assert r["achieved"] == pytest.approx(1000 * 60 / 3e-3 / 1e9)
    assert r["secondary"][0]["achieved"] == pytest.approx(1000 * 8 / 3e-3 / 1e12)
    kern["recon_stats_kernel"] = {"ms": 4.0, "launches_per_step": 1.0}
    r = bench.kernel_roofline(kern, ctx)
    assert r["kernel"] == "recon_stats_kernel" and r["bound"] == "alu" and r["unit"] == "Tops/s"
    # 2 Philox blocks x 40 + uniforms (2 x 2 + 4 x 1) + Box-Muller 51 + L xi 6 + sums 8 + 3 x 14
    assert bench.STATS_OPS_PER_P[3] == 80 + 8 + 51 + 6 + 8 + 42
    assert r["achieved"] == pytest.approx(1000 * 195 / 4e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.alu_peak_tops(2070.0))
    assert r["secondary"][0]["achieved"] == pytest.approx(1000 * 20 / 4e-3 / 1e9)
    # traffic: the captured DRAM bytes per particle of the workload, times
    # the particles of a launch (null for workloads without a capture)
    assert r["traffic"] is None
    r = bench.kernel_roofline(kern, dict(ctx, workload="lognormal_1d3v"))
    assert r["traffic"] == pytest.approx(1000 * (3.977728e6 + 165.554688e6) / 9324406)
    kern = {"mlp_forward (tc_gemm_kernel x4)": {"ms": 1.0, "launches_per_step": 1.0}}
    r = bench.kernel_roofline(kern, ctx)
    assert r["bound"] == "tensor"
    assert r["achieved"] == pytest.approx(2 * 3 * (576 * 256 + 2 * 256 * 256 + 256 * 112) / 1e-3 / 1e12)
