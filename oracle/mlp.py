"""FP64 numpy oracle of the learned-initialisation network (the method's
component count and parameters predicted from per-cell features; not part
of the paper, which initialises EM with randomly chosen particles).

TEST INFRASTRUCTURE: only the tests and the benchmark's CPU legs use it.

Interface shared with the CUDA path (each side implements it separately):

* features of a cell (weights alpha, velocities v, D = 1 or 3):
  W = sum alpha, mean = sum alpha v / W, var_d = sum alpha (v_d - mean_d)^2 / W,
  y = (v - mean) / sqrt(var) (per dimension); expectations E[.] are
  alpha-weighted.
    D = 1: [E y^3, E y^4 - 3, ln(N)/10] + 64-bin histogram of y on [-4, 4)
    D = 3: [E y_d^3 (3), E y_d^4 - 3 (3), E y0 y1, E y0 y2, E y1 y2, ln(N)/10]
           + 8x8x8 histogram of y on [-2.5, 2.5)^3 (index b0*64 + b1*8 + b2)
  histogram entries are (sum of alpha in the bin) / W * nbins, values
  outside the range go to the edge bins; the vector is zero-padded to
  F = 128 (D = 1) or 576 (D = 3).
* network: h1 = relu(x W1^T + b1), h2 = relu(h1 W2^T + b2),
  h3 = relu(h2 W3^T + b3), out = h3 W4^T + b4; hidden width 256; the
  hidden activations are stored in BF16 (round to nearest even), as the
  tensor-core network stores them; backward treats that rounding as the
  identity;
  out has Kmax slots of SP = 2 + 2D + D(D-1)/2 values, zero-padded to a
  multiple of 16:
    [presence logit, log weight, mu (D), log diag of L (D), L10, L20, L21]
  (whitened coordinates; Sigma = L L^T).
* targets from a fit: components sorted by mu_0 (whitened) ascending;
  slot s < K: presence 1, ln omega, mu, log diag and off-diagonals of the
  Cholesky factor of the whitened covariance; slots s >= K: presence 0
  (only the presence enters the loss).
* loss per cell: sum_s softplus(p_s) - t_s p_s
                 + sum_{s<K} sum (pred - target)^2  (all other slot values);
  the batch loss is the mean over cells.
* Adam: beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected.
"""
from __future__ import annotations

import math

import numpy as np

HIDDEN = 256


def feat_dims(D: int):
    nmom = 3 if D == 1 else 10
    nbin = 64 if D == 1 else 512
    fpad = 128 if D == 1 else 576
    return nmom, nbin, fpad


def slot_size(D: int) -> int:
    return 2 + 2 * D + D * (D - 1) // 2


def out_dims(D: int, Kmax: int):
    o = Kmax * slot_size(D)
    return o, (o + 15) // 16 * 16


def cell_features(v: np.ndarray, alpha: np.ndarray) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """v [N, D], alpha [N] -> (feature vector [F], mean [D], sd [D])."""
    v = np.asarray(v, dtype=np.float64)
    a = np.asarray(alpha, dtype=np.float64)
    N, D = v.shape
    nmom, nbin, fpad = feat_dims(D)
    f = np.zeros(fpad)
    W = a.sum()
    mean = (a[:, None] * v).sum(axis=0) / W
    var = (a[:, None] * (v - mean) ** 2).sum(axis=0) / W
    sd = np.sqrt(var)
    if np.any(~(sd > 0)):
        return f, mean, sd
    y = (v - mean) / sd
    w = a / W
    if D == 1:
        f[0] = (w * y[:, 0] ** 3).sum()
        f[1] = (w * y[:, 0] ** 4).sum() - 3.0
        f[2] = math.log(N) / 10.0
        b = np.clip(np.floor((y[:, 0] + 4.0) * 8.0), 0, 63).astype(int)
        h = np.bincount(b, weights=w, minlength=64) * 64
        f[3:3 + 64] = h
    else:
        for d in range(3):
            f[d] = (w * y[:, d] ** 3).sum()
            f[3 + d] = (w * y[:, d] ** 4).sum() - 3.0
        f[6] = (w * y[:, 0] * y[:, 1]).sum()
        f[7] = (w * y[:, 0] * y[:, 2]).sum()
        f[8] = (w * y[:, 1] * y[:, 2]).sum()
        f[9] = math.log(N) / 10.0
        b = np.clip(np.floor((y + 2.5) * (8.0 / 5.0)), 0, 7).astype(int)
        idx = b[:, 0] * 64 + b[:, 1] * 8 + b[:, 2]
        f[10:10 + 512] = np.bincount(idx, weights=w, minlength=512) * 512
    return f, mean, sd


def _unpack(prm, D):
    w = prm[0]
    mu = prm[1:1 + D]
    S = np.zeros((D, D))
    t = 1 + D
    for i in range(D):
        for j in range(i, D):
            S[i, j] = S[j, i] = prm[t]
            t += 1
    return w, mu, S


def cell_targets(K: int, params: np.ndarray, mean: np.ndarray, sd: np.ndarray, D: int,
                 Kmax: int) -> tuple[np.ndarray, np.ndarray]:
    """Targets and loss mask of one cell from its fit (original coordinates)."""
    o, opad = out_dims(D, Kmax)
    SP = slot_size(D)
    t = np.zeros(opad)
    m = np.zeros(opad)
    comps = []
    for k in range(K):
        w, mu, S = _unpack(params[k], D)
        muw = (mu - mean) / sd
        Sw = S / np.outer(sd, sd)
        comps.append((muw[0], w, muw, Sw))
    comps.sort(key=lambda c: c[0])
    for s in range(Kmax):
        base = s * SP
        m[base] = 1.0
        if s < K:
            _, w, muw, Sw = comps[s]
            L = np.linalg.cholesky(Sw)
            t[base] = 1.0
            vals = [math.log(w), *muw, *np.log(np.diag(L))]
            if D == 3:
                vals += [L[1, 0], L[2, 0], L[2, 1]]
            t[base + 1: base + SP] = vals
            m[base + 1: base + SP] = 1.0
    return t, m


def init_params(D: int, Kmax: int, seed: int = 0) -> dict:
    """He-normal weights, zero biases (FP64 masters)."""
    rng = np.random.default_rng(seed)
    _, _, fpad = feat_dims(D)
    _, opad = out_dims(D, Kmax)
    dims = [(HIDDEN, fpad), (HIDDEN, HIDDEN), (HIDDEN, HIDDEN), (opad, HIDDEN)]
    p = {}
    for i, (n, k) in enumerate(dims, 1):
        p[f"W{i}"] = rng.standard_normal((n, k)) * math.sqrt(2.0 / k)
        p[f"b{i}"] = np.zeros(n)
    return p


def bf16(a: np.ndarray) -> np.ndarray:
    """Round to BF16 (via FP32, round to nearest even), returned as FP64."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(p: dict, X: np.ndarray, round_bf16: bool = True) -> dict:
    rnd = bf16 if round_bf16 else (lambda a: a)
    Z1 = X @ p["W1"].T + p["b1"]
    H1 = rnd(np.maximum(Z1, 0.0))
    Z2 = H1 @ p["W2"].T + p["b2"]
    H2 = rnd(np.maximum(Z2, 0.0))
    Z3 = H2 @ p["W3"].T + p["b3"]
    H3 = rnd(np.maximum(Z3, 0.0))
    out = H3 @ p["W4"].T + p["b4"]
    return dict(X=X, H1=H1, H2=H2, H3=H3, out=out)


def loss_and_grad_out(out: np.ndarray, T: np.ndarray, Mk: np.ndarray, D: int,
                      Kmax: int) -> tuple[float, np.ndarray]:
    """Mean batch loss and d loss / d out."""
    B = out.shape[0]
    SP = slot_size(D)
    pres = np.zeros(out.shape[1], dtype=bool)
    pres[0:Kmax * SP:SP] = True
    L = 0.0
    G = np.zeros_like(out)
    p = out[:, pres]
    t = T[:, pres]
    L += (np.logaddexp(0.0, p) - t * p).sum()
    G[:, pres] = 1.0 / (1.0 + np.exp(-p)) - t
    reg = (~pres)[None, :] & (Mk > 0)
    diff = np.where(reg, out - T, 0.0)
    L += (diff ** 2).sum()
    G += 2.0 * diff
    return L / B, G / B


def backward(p: dict, f: dict, G: np.ndarray) -> dict:
    g = {}
    g["W4"] = G.T @ f["H3"]
    g["b4"] = G.sum(axis=0)
    d3 = (G @ p["W4"]) * (f["H3"] > 0)
    g["W3"] = d3.T @ f["H2"]
    g["b3"] = d3.sum(axis=0)
    d2 = (d3 @ p["W3"]) * (f["H2"] > 0)
    g["W2"] = d2.T @ f["H1"]
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ p["W2"]) * (f["H1"] > 0)
    g["W1"] = d1.T @ f["X"]
    g["b1"] = d1.sum(axis=0)
    return g


def adam_step(p: dict, g: dict, state: dict, lr: float, t: int, b1=0.9, b2=0.999, eps=1e-8):
    for k in p:
        m = state.setdefault("m" + k, np.zeros_like(p[k]))
        v = state.setdefault("v" + k, np.zeros_like(p[k]))
        m[:] = b1 * m + (1 - b1) * g[k]
        v[:] = b2 * v + (1 - b2) * g[k] ** 2
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


def decode(out: np.ndarray, mean: np.ndarray, sd: np.ndarray, N: int, D: int, Kmax: int,
           presence_logit: float = 0.0):
    """Initial mixture (original coordinates) from one cell's network output:
    slots whose presence logit exceeds ``presence_logit`` (at least the most
    likely one), capped so that N - T K0 / 2 > 0; weights by softmax of the
    log weights."""
    SP = slot_size(D)
    T_ = D * (D + 3) / 2
    pres = out[0:Kmax * SP:SP]
    order = [s for s in range(Kmax) if pres[s] > presence_logit]
    if not order:
        order = [int(np.argmax(pres))]
    lw = np.array([out[s * SP + 1] for s in order])
    while len(order) > 1 and N - T_ * len(order) / 2 <= 0:
        drop = int(np.argmin(lw))
        order.pop(drop)
        lw = np.delete(lw, drop)
    w = np.exp(lw - lw.max())
    w /= w.sum()
    P = 1 + D + D * (D + 1) // 2
    prm = np.zeros((len(order), P))
    for i, s in enumerate(order):
        base = s * SP
        muw = out[base + 2: base + 2 + D]
        ld = np.clip(out[base + 2 + D: base + 2 + 2 * D], -10.0, 5.0)
        L = np.diag(np.exp(ld))
        if D == 3:
            L[1, 0], L[2, 0], L[2, 1] = out[base + 2 + 2 * D: base + SP]
        Sw = L @ L.T
        S = Sw * np.outer(sd, sd)
        prm[i, 0] = w[i]
        prm[i, 1:1 + D] = mean + sd * muw
        t = 1 + D
        for a in range(D):
            for b in range(a, D):
                prm[i, t] = S[a, b]
                t += 1
    return len(order), prm
