"""Learned initialisation of the adaptive EM (not part of the paper): train
the network on cells fitted by the paper's method, then start EM from the
network's predicted mixtures.  All arithmetic runs in the library's kernels
(features, tensor-core network, decode, EM); this module only sequences the
calls."""
from __future__ import annotations

import time

import torch

from . import gm


def fit_targets(cfg, cell_off, x, v, alpha):
    """Plain-EM fits of training cells and the network's inputs / targets."""
    fit = gm.gm_compress(cfg, cell_off, x, v, alpha)
    feat, wstat = gm.gm_features(cfg, cell_off, v, alpha)
    T, Mk = gm.gm_mlp_targets(cfg, fit["K"], fit["params"], wstat)
    return feat, T, Mk, fit


def train(net: gm.Net, feat, T, Mk, epochs: int = 10, batch: int = 1024, lr: float = 1e-3,
          seed: int = 0, log=None) -> dict:
    """Adam on minibatches of whole rows (the last partial batch is
    dropped); returns the mean loss per epoch."""
    C = feat.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    nb = C // batch
    losses = []
    t0 = time.perf_counter()
    for ep in range(epochs):
        perm = torch.randperm(C, generator=g).to(feat.device)
        acc = torch.zeros(1, dtype=torch.float64, device=feat.device)
        for i in range(nb):
            idx = perm[i * batch:(i + 1) * batch]
            net.train_step(feat[idx].contiguous(), T[idx].contiguous(), Mk[idx].contiguous(), lr,
                           loss=acc)
        losses.append(float(acc.item()) / max(nb, 1))
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.4f}")
    torch.cuda.synchronize()
    return {"loss": losses, "seconds": time.perf_counter() - t0, "steps": nb * epochs}


def init_from_net(net: gm.Net, cfg, cell_off, v, alpha, presence_logit: float = 0.0):
    """Features -> network -> initial mixtures (K0, params)."""
    feat, wstat = gm.gm_features(cfg, cell_off, v, alpha)
    out = net.forward(feat)
    return gm.gm_mlp_decode(cfg, out, wstat, cell_off, presence_logit=presence_logit)


def compress_learned(net: gm.Net, cfg, cell_off, x, v, alpha, out=None, presence_logit: float = 0.0):
    """gm_compress started from the network's mixtures."""
    K0, prm = init_from_net(net, cfg, cell_off, v, alpha, presence_logit)
    return gm.gm_compress(cfg, cell_off, x, v, alpha, out=out, init_K=K0, init_params=prm)


def calibrate_presence(net: gm.Net, cfg, cell_off, x, v, alpha, lnL_plain,
                       candidates=(0.0, 0.5, 1.0, 2.0, 4.0, 8.0, 16.0), slack: float = 0.005):
    """The decode's presence-logit threshold for a batch of training cells
    whose plain-EM objective (eq. lnL-GM, ``lnL_plain``) is known: for each
    candidate, EM from the decoded start is timed once and its rate of
    reaching plain EM's objective (within 1e-4 relative) measured; the
    fastest candidate whose rate is within ``slack`` of the best is
    returned, with the table."""
    feat, wstat = gm.gm_features(cfg, cell_off, v, alpha)
    out = net.forward(feat)
    table = {}
    Lp = lnL_plain
    for thr in candidates:
        K0, prm = gm.gm_mlp_decode(cfg, out, wstat, cell_off, presence_logit=thr)
        fit = gm.gm_compress(cfg, cell_off, x, v, alpha, init_K=K0, init_params=prm)  # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        gm.gm_compress(cfg, cell_off, x, v, alpha, init_K=K0, init_params=prm, out=fit)
        e1.record()
        torch.cuda.synchronize()
        reach = float(((fit["lnL"] >= Lp - 1e-4 * Lp.abs())).double().mean())
        table[thr] = {"ms": e0.elapsed_time(e1), "reach": reach,
                      "sweeps": float(fit["sweeps"].double().mean())}
    best = max(r["reach"] for r in table.values())
    ok = [thr for thr, r in table.items() if r["reach"] >= best - slack]
    pick = min(ok, key=lambda thr: table[thr]["ms"])
    return pick, {"picked": pick, "table": {str(k): v for k, v in table.items()}}
