"""Batching infrastructure on the GPU: the natively captured CUDA graph of
the pipeline replays bit for bit what the direct calls compute, owns its
workspace, and the EM results do not depend on the shared-tile choice that
the autotuner makes."""
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


def inputs(wl):
    return dev(wl.cell_off), dev(wl.x), dev(wl.v), dev(wl.alpha)


def compress_out(gm, cfg, C, device="cuda"):
    P = gm.P_of(cfg.D)
    return dict(K=torch.empty(C, dtype=torch.int32, device=device),
                params=torch.empty((C, cfg.Kmax, P), dtype=torch.float64, device=device),
                W=torch.empty(C, dtype=torch.float64, device=device),
                rho_target=torch.empty(C, dtype=torch.float64, device=device),
                lnL=torch.empty(C, dtype=torch.float64, device=device),
                sweeps=torch.empty(C, dtype=torch.int32, device=device),
                kwork=torch.empty(C, dtype=torch.int32, device=device),
                status=torch.empty(C, dtype=torch.int32, device=device))


def recon_out(D, C, n, device="cuda"):
    return dict(x=torch.empty(n, dtype=torch.float64, device=device),
                v=torch.empty((D, n), dtype=torch.float64, device=device),
                alpha=torch.empty(n, dtype=torch.float64, device=device),
                status=torch.empty(C, dtype=torch.int32, device=device))


def same(a: dict, b: dict):
    for k in a:
        assert torch.equal(a[k], b[k]), k


def test_graph_replays_compress_and_reconstruct_bit_for_bit(gm):
    wl = workloads.mixture_1d1v(C=96, mean_n=900, clip=(100, 3000), seed=31)
    cfg = gm.config(wl.params)
    rcfg = gm.config(wl.params, seed_key="recon_seed")
    off, x, v, a = inputs(wl)
    n = wl.ntot
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ref_c = gm.gm_compress(cfg, off, x, v, a)
        ref_r = gm.gm_reconstruct(rcfg, ref_c["K"], ref_c["params"], ref_c["W"], ref_c["rho_target"],
                                  off, n_out=n)
        oc, orr = compress_out(gm, cfg, wl.C), recon_out(wl.D, wl.C, n)
        g = gm.Graph(s)
        with g:
            gm.gm_compress(cfg, off, x, v, a, out=oc)
            gm.gm_reconstruct(rcfg, oc["K"], oc["params"], oc["W"], oc["rho_target"], off, n_out=n,
                              out=orr)
        g.keep(oc, orr)
        for _ in range(2):
            for t in list(oc.values()) + list(orr.values()):
                t.fill_(0)
            g.launch()
            s.synchronize()
            same(ref_c, oc)
            same(ref_r, orr)
        # a larger direct call grows the shared workspace; the graph keeps its own
        big = workloads.mixture_1d1v(C=512, mean_n=2000, seed=32)
        bcfg = gm.config(big.params)
        gm.gm_compress(bcfg, *inputs(big))
        g.launch()
        s.synchronize()
        same(ref_c, oc)
        g.close()


def test_graph_replays_learned_pipeline(gm):
    wl = workloads.mixture_1d1v(C=64, mean_n=800, clip=(100, 2000), seed=33)
    cfg = gm.config(wl.params)
    off, x, v, a = inputs(wl)
    net = gm.Net(1, cfg.Kmax)
    net.init_weights(seed=5)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        feat, wstat = gm.gm_features(cfg, off, v, a)
        o = net.forward(feat)
        K0, prm = gm.gm_mlp_decode(cfg, o, wstat, off)
        ref = gm.gm_compress(cfg, off, x, v, a, init_K=K0, init_params=prm)
        bufs = (torch.empty_like(feat), torch.empty_like(wstat), torch.empty_like(o),
                torch.empty_like(K0), torch.empty_like(prm))
        oc = compress_out(gm, cfg, wl.C)
        g = gm.Graph(s)
        with g:
            gm.gm_features(cfg, off, v, a, out=(bufs[0], bufs[1]))
            net.forward(bufs[0], out=bufs[2])
            gm.gm_mlp_decode(cfg, bufs[2], bufs[1], off, dest=(bufs[3], bufs[4]))
            gm.gm_compress(cfg, off, x, v, a, out=oc, init_K=bufs[3], init_params=bufs[4])
        g.keep(bufs, oc)
        g.launch()
        s.synchronize()
        same(ref, oc)
        assert torch.equal(K0, bufs[3])
        g.close()


def test_graph_api_errors(gm):
    import ctypes as ct
    lib = gm.load()
    h = ct.c_void_p()
    assert lib.gm_graph_end(None, ct.byref(h)) == gm.GM_ERR_ARG  # nothing captured
    assert lib.gm_graph_launch(None, None) == gm.GM_ERR_ARG
    assert lib.gm_graph_destroy(None) == gm.GM_OK


def test_results_do_not_depend_on_the_shared_tile(gm):
    wl = workloads.mixture_1d1v(C=80, mean_n=1500, clip=(100, 4000), seed=34)
    off, x, v, a = inputs(wl)
    outs = []
    for cap in (0, 256, 4096):  # default, most cells on the global tile, all in shared memory
        cfg = gm.config(wl.params, threads_per_cell=256, smem_particles=cap)
        outs.append(gm.gm_compress(cfg, off, x, v, a))
    torch.cuda.synchronize()
    same(outs[0], outs[1])
    same(outs[0], outs[2])


def test_autotune_picks_a_valid_shape_and_the_fit_stays_on_the_oracle(gm):
    wl = workloads.mixture_1d1v(C=256, mean_n=1500, counts="uniform", clip=(200, 5000), seed=35)
    cfg = gm.config(wl.params)
    off, x, v, a = inputs(wl)
    t = gm.gm_autotune(cfg, off, x, v, a, sweeps_per_trial=8)
    assert cfg.threads_per_cell in (64, 128, 256)
    assert cfg.smem_particles > 0 and cfg.smem_particles % 4 == 0
    ran = [z for z in t if z >= 0]
    assert len(ran) >= 2 and min(ran) > 0
    # the tuned shape and the same CTA size with the default tile agree bit for bit
    out = gm.gm_compress(cfg, off, x, v, a)
    cfg2 = gm.config(wl.params, threads_per_cell=cfg.threads_per_cell)
    out2 = gm.gm_compress(cfg2, off, x, v, a)
    torch.cuda.synchronize()
    same(out, out2)
    # and the fit is the method's: lnL within 1e-5 of the oracle wherever K agrees
    sub = slice(0, 48)
    p = dict(wl.params)
    C2 = 48
    n2 = int(wl.cell_off[C2])
    p["L"] = wl.params["L"] * C2 / wl.C
    ref = oracle.compress(p, wl.cell_off[:C2 + 1], wl.x[:n2], np.ascontiguousarray(wl.v[:, :n2]),
                          wl.alpha[:n2])
    K = out["K"].cpu().numpy()[sub]
    lnL = out["lnL"].cpu().numpy()[sub]
    agree = (K == ref["K"]) & (np.abs(lnL - ref["lnL"]) <= 1e-5 * np.abs(ref["lnL"]))
    assert (K == ref["K"]).mean() >= 0.95 and agree.mean() >= 0.9, agree.mean()


@pytest.mark.parametrize("nt,cap", [(64, 0), (64, 256), (128, 512)])
def test_small_ctas_fit_like_the_oracle(gm, nt, cap):
    """64- and 128-thread CTAs (more cells per SM) with small and default
    tiles: the fit keeps the oracle's K and lnL under the equal-sweep rule,
    1V and 3V."""
    from parity_helpers import agreement
    for wl in (workloads.mixture_1d1v(C=48, mean_n=700, clip=(100, 2000), seed=36),
               workloads.with_weights(workloads.bimaxwellian_1d3v(C=24, ppc=600, seed=37))):
        cfg = gm.config(wl.params, threads_per_cell=nt, smem_particles=cap)
        out = gm.gm_compress(cfg, *inputs(wl))
        g = {k: t.cpu().numpy() for k, t in out.items()}
        ref = oracle.compress(wl.params, wl.cell_off, wl.x, wl.v, wl.alpha, nthreads=8)
        agree, eq = agreement(g, ref, wl)
        ks = g["K"] == ref["K"]
        print(f"nt {nt} cap {cap} D {wl.D}: K {ks.mean():.3f}, K + lnL {agree.mean():.3f}, "
              f"equal sweeps {eq.mean():.3f}")
        assert ks.mean() >= 0.95 and agree.mean() >= 0.85, (ks.mean(), agree.mean())
        np.testing.assert_allclose(g["W"], ref["W"], rtol=1e-13)


def test_autotune_from_a_supplied_start(gm):
    """gm_autotune_from: trials from supplied initial mixtures (the oracle's
    fits of the cells, one component in half of them) pick a valid shape,
    and the fit from the same start with that shape equals the fit with the
    same CTA size and the default tile bit for bit."""
    import ctypes as ct
    wl = workloads.with_weights(workloads.bimaxwellian_1d3v(C=320, ppc=600, seed=38))
    off, x, v, a = inputs(wl)
    ref = oracle.compress(wl.params, wl.cell_off, wl.x, wl.v, wl.alpha, nthreads=8)
    K0 = ref["K"].copy()
    K0[::2] = 1
    prm = ref["params"].copy()
    prm[::2, 0, 0] = 1.0
    K0t, prmt = dev(K0.astype(np.int32)), dev(prm)
    cfg = gm.config(wl.params)
    t = gm.gm_autotune(cfg, off, x, v, a, sweeps_per_trial=8, init_K=K0t, init_params=prmt)
    assert cfg.threads_per_cell in (64, 128, 256)
    assert cfg.smem_particles > 0 and cfg.smem_particles % 4 == 0
    assert len([z for z in t if z > 0]) >= 2
    out = gm.gm_compress(cfg, off, x, v, a, init_K=K0t, init_params=prmt)
    cfg2 = gm.config(wl.params, threads_per_cell=cfg.threads_per_cell)
    out2 = gm.gm_compress(cfg2, off, x, v, a, init_K=K0t, init_params=prmt)
    torch.cuda.synchronize()
    same(out, out2)
    lib = gm.load()
    buf = (ct.c_float * gm.TUNE_CANDIDATES)()
    assert lib.gm_autotune_from(ct.byref(cfg), wl.C, wl.ntot, gm._ptr(off), gm._ptr(x), gm._ptr(v), 0,
                                gm._ptr(a), None, None, 0, buf, None) == gm.GM_ERR_ARG


def test_kernel_trace_times_each_kernel(gm):
    """gm_trace_begin / gm_trace_end: per-kernel device times (CUDA events on
    the launching stream) of a learned-start compress and a reconstruct;
    nothing is recorded inside a graph capture."""
    wl = workloads.mixture_1d1v(C=64, mean_n=400, clip=(50, 900), seed=5)
    cfg = gm.config(wl.params)
    off, x, v, a = inputs(wl)
    fit = gm.gm_compress(cfg, off, x, v, a)
    K0 = torch.ones(wl.C, dtype=torch.int32, device="cuda")
    K0[::2] = 2  # half the cells start with two components: both kernels run
    torch.cuda.synchronize()
    with gm.Trace() as tr:
        out = gm.gm_compress(cfg, off, x, v, a, init_K=K0, init_params=fit["params"])
        gm.gm_reconstruct(cfg, out["K"], out["params"], out["W"], out["rho_target"], off, n_out=wl.ntot)
    t = tr.times
    for k in ("em_k1_kernel", "em_kernel", "recon_stats_kernel", "recon_emit_kernel", "assemble_kernel"):
        assert k in t and t[k][0] > 0.0 and t[k][1] == 1, (k, t)
    assert any(k.startswith("deposit") for k in t)
    # captured launches are not traced
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g = gm.Graph(stream)
        with gm.Trace() as tr2:
            with g:
                gm.gm_compress(cfg, off, x, v, a, stream=stream, out=out)
        g.close()
    assert tr2.times == {}
