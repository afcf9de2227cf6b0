"""FP64 CPU oracle of the Gaussian-mixture checkpoint-restart method
(Chen, Chacon & Nguyen, arXiv 2007.12273), wrapped for numpy.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The arithmetic
lives in ``gm_oracle.c`` (plain C, FP64, one cell at a time); this module
only builds it with gcc and marshals numpy arrays.  It shares no code with
the CUDA path.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# per-cell status bits (the library's documented values)
ST_EM_MAXSWEEPS = 0x01
ST_COV_NOT_PD = 0x02
ST_TOO_FEW = 0x04
ST_EMPTY = 0x08
ST_DEGENERATE = 0x10
ST_PROJ_SKIPPED = 0x100
ST_NEG_WEIGHT = 0x200
ST_MM_EMPTY_COL = 0x400
ST_NO_MIXTURE = 0x800


def build(force: bool = False) -> str:
    """Compile gm_oracle.c into liboracle.so (gcc, OpenMP, no FP contraction
    so that x86 and Arm hosts round identically)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Cfg(ct.Structure):
    _fields_ = [("D", ct.c_int), ("Kmax", ct.c_int), ("shape_order", ct.c_int),
                ("max_sweeps", ct.c_int), ("tol", ct.c_double), ("seed", ct.c_uint64),
                ("L", ct.c_double), ("q", ct.c_double)]


class _Mesh2d(ct.Structure):
    _fields_ = [("Cx", ct.c_int64), ("Cy", ct.c_int64), ("Lx", ct.c_double), ("Ly", ct.c_double)]


def _mesh(params: dict) -> _Mesh2d:
    return _Mesh2d(int(params["Cx"]), int(params["Cy"]), float(params["Lx"]), float(params["Ly"]))


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ct.CDLL(_LIB)
            P = ct.c_void_p
            lib.oracle_philox4x32_10.argtypes = [P, P, P]
            lib.oracle_uniform52.argtypes = [ct.c_uint32, ct.c_uint32]
            lib.oracle_uniform52.restype = ct.c_double
            lib.oracle_compress.argtypes = [P, ct.c_int64] + [P] * 15 + [ct.c_int]
            lib.oracle_em_cell.argtypes = [P, ct.c_int64, ct.c_int64, P, P, P, ct.c_int, ct.c_int,
                                           P, P, P, P, P, P, P, P, ct.c_int, P]
            lib.oracle_penalised_L.argtypes = [ct.c_int, ct.c_int, P, ct.c_int64, P, P]
            lib.oracle_penalised_L.restype = ct.c_double
            lib.oracle_cyclic_tridiag.argtypes = [ct.c_int64, P, P, P, P, P]
            lib.oracle_reconstruct.argtypes = [P, ct.c_int64] + [P] * 11 + [ct.c_int]
            lib.oracle_moments.argtypes = [P, ct.c_int64] + [P] * 9
            lib.oracle_mixture_moments.argtypes = [P, ct.c_int64] + [P] * 7
            lib.oracle_shape.argtypes = [ct.c_int, ct.c_double]
            lib.oracle_shape.restype = ct.c_double
            lib.oracle_max_threads.restype = ct.c_int
            lib.oracle_standard.argtypes = ([P, ct.c_int64] + [P] * 4 + [ct.c_int] * 4 + [P] * 11
                                            + [ct.c_int])
            lib.oracle_std_cell.argtypes = ([P, ct.c_int64, ct.c_int64, P, P] + [ct.c_int] * 4
                                            + [P] * 9 + [ct.c_int, P, P, ct.c_int])
            lib.oracle_aa_affine.argtypes = [ct.c_int, P, P, P, ct.c_int, ct.c_int, P, P]
            lib.oracle_kmeans.argtypes = [ct.c_int, ct.c_int, ct.c_int64, P, P, P, ct.c_int, P, P, P]
            lib.oracle_deposit2d.argtypes = [P] * 7
            lib.oracle_reconstruct2d.argtypes = [P] * 12 + [ct.c_int]
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ct.c_void_p) if a is not None else None


def _cfg(params: dict, seed_key="seed") -> _Cfg:
    return _Cfg(int(params["D"]), int(params["Kmax"]), int(params["shape_order"]),
                int(params.get("max_sweeps", 1000)), float(params.get("tol", 1e-6)),
                int(params.get(seed_key, 1)), float(params["L"]), float(params.get("q", 1.0)))


def P_of(D: int) -> int:
    return 1 + D + D * (D + 1) // 2


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def philox(ctr, key) -> np.ndarray:
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def uniform52(hi: int, lo: int) -> float:
    return _load().oracle_uniform52(hi, lo)


def shape(order: int, s: float) -> float:
    return _load().oracle_shape(order, s)


def max_threads() -> int:
    return _load().oracle_max_threads()


def compress(params: dict, cell_off, x, v, alpha, nthreads: int = 1, cell_ids=None,
             init_K=None, init_params=None) -> dict:
    """Oracle compression of every cell (Sec. 2.2-2.3, final step of
    Sec. 2.3.1, target charge density of Sec. 2.4.1).  ``cell_ids`` gives
    each cell's index in a larger batch (it keys the initial picks); the
    charge density then refers to the sub-mesh given."""
    lib = _load()
    cfg = _cfg(params)
    cell_off = np.ascontiguousarray(cell_off, dtype=np.int64)
    C = cell_off.shape[0] - 1
    D = cfg.D
    x = _f64(x); v = _f64(v); alpha = _f64(alpha)
    assert v.shape == (D, int(cell_off[-1]))
    out = dict(K=np.zeros(C, np.int32), params=np.zeros((C, cfg.Kmax, P_of(D))),
               W=np.zeros(C), rho_target=np.zeros(C), lnL=np.zeros(C),
               sweeps=np.zeros(C, np.int32), kwork=np.zeros(C, np.int32),
               status=np.zeros(C, np.uint32))
    rc = lib.oracle_compress(ct.byref(cfg), C, _ptr(cell_off), _ptr(x), _ptr(v), _ptr(alpha),
                             _ptr(out["K"]), _ptr(out["params"]), _ptr(out["W"]),
                             _ptr(out["rho_target"]), _ptr(out["lnL"]), _ptr(out["sweeps"]),
                             _ptr(out["kwork"]), _ptr(out["status"]),
                             _ptr(None if cell_ids is None else np.ascontiguousarray(cell_ids, dtype=np.int64)),
                             _ptr(None if init_K is None else np.ascontiguousarray(init_K, dtype=np.int32)),
                             _ptr(None if init_params is None else _f64(init_params)),
                             int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_compress failed ({rc})")
    return out


def em_cell(params: dict, vv, alpha, cell: int = 0, init_params=None, init_K: int = 0,
            only_sweeps: int = 0, trace_cap: int = 0) -> dict:
    """One cell: ``vv`` is [N, D].  ``init_params`` [K, P] replaces the
    random initialisation; ``only_sweeps`` > 0 runs that many penalised
    sweeps and skips the final unpenalised step."""
    lib = _load()
    cfg = _cfg(params)
    vv = _f64(vv).reshape(-1, cfg.D)
    N = vv.shape[0]
    alpha = _f64(alpha)
    prm = np.zeros((cfg.Kmax, P_of(cfg.D)))
    ip = None
    if init_params is not None:
        ip = _f64(init_params)
        init_K = ip.shape[0]
    K = np.zeros(1, np.int32); W = np.zeros(1); lnL = np.zeros(1)
    sw = np.zeros(1, np.int32); st = np.zeros(1, np.uint32)
    tr = np.zeros(max(trace_cap, 1)); kt = np.zeros(max(trace_cap, 1), np.int32)
    nt = np.zeros(1, np.int32)
    lib.oracle_em_cell(ct.byref(cfg), int(cell), N, _ptr(vv), _ptr(alpha), _ptr(ip), int(init_K),
                       int(only_sweeps), _ptr(prm), _ptr(K), _ptr(W), _ptr(lnL), _ptr(sw),
                       _ptr(st), _ptr(tr) if trace_cap else None, _ptr(kt) if trace_cap else None,
                       int(trace_cap), _ptr(nt))
    # Ktrace: K after initialisation / after each sweep, negative when the
    # sweep removed a component
    return dict(K=int(K[0]), params=prm, W=float(W[0]), lnL=float(lnL[0]), sweeps=int(sw[0]),
                status=int(st[0]), Ltrace=tr[: int(nt[0])].copy(),
                Ktrace=kt[: int(nt[0])].copy())


def standard(params: dict, cell_off, x, v, alpha, init: int = 0, aa_memory: int = 0,
             kmeans_iters: int = 0, nthreads: int = 1, cell_ids=None, penalised: bool = False) -> dict:
    """Oracle of the standard (non-adaptive) EM of Sec. 4 for every cell:
    ``init`` 0 = random particles, 1 = K-means; ``aa_memory`` > 0 turns on
    Anderson acceleration; ``penalised`` runs the simultaneous EM with the
    penalised weights and annihilation instead (no AA).  Outputs as
    ``compress`` plus iterations, AA steps, AA resets and K-means passes per
    cell."""
    lib = _load()
    cfg = _cfg(params)
    cell_off = np.ascontiguousarray(cell_off, dtype=np.int64)
    C = cell_off.shape[0] - 1
    D = cfg.D
    x = _f64(x); v = _f64(v); alpha = _f64(alpha)
    assert v.shape == (D, int(cell_off[-1]))
    out = dict(K=np.zeros(C, np.int32), params=np.zeros((C, cfg.Kmax, P_of(D))),
               W=np.zeros(C), rho_target=np.zeros(C), lnL=np.zeros(C),
               iters=np.zeros(C, np.int32), aa_steps=np.zeros(C, np.int32),
               aa_resets=np.zeros(C, np.int32), km_passes=np.zeros(C, np.int32),
               status=np.zeros(C, np.uint32))
    rc = lib.oracle_standard(ct.byref(cfg), C, _ptr(cell_off), _ptr(x), _ptr(v), _ptr(alpha),
                             int(init), int(aa_memory), int(kmeans_iters), int(bool(penalised)), _ptr(out["K"]),
                             _ptr(out["params"]), _ptr(out["W"]), _ptr(out["rho_target"]),
                             _ptr(out["lnL"]), _ptr(out["iters"]), _ptr(out["aa_steps"]),
                             _ptr(out["aa_resets"]), _ptr(out["km_passes"]), _ptr(out["status"]),
                             _ptr(None if cell_ids is None else np.ascontiguousarray(cell_ids, dtype=np.int64)),
                             int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_standard failed ({rc})")
    return out


def std_cell(params: dict, vv, alpha, cell: int = 0, init: int = 0, aa_memory: int = 0,
             kmeans_iters: int = 0, trace_cap: int = 0, init_params=None, penalised: bool = False) -> dict:
    """Standard EM of one cell (``vv`` [N, D]) with the trace of L(theta_i)
    (penalised L with ``penalised``); ``init_params`` [K][P] (with ``init``
    = 2) continues from a given fit."""
    lib = _load()
    cfg = _cfg(params)
    vv = _f64(vv).reshape(-1, cfg.D)
    N = vv.shape[0]
    alpha = _f64(alpha)
    prm = np.zeros((cfg.Kmax, P_of(cfg.D)))
    i32 = lambda: np.zeros(1, np.int32)
    K, it, na, nr, km = i32(), i32(), i32(), i32(), i32()
    lnL = np.zeros(1); st = np.zeros(1, np.uint32)
    tr = np.zeros(max(trace_cap, 1)); nt = np.zeros(1, np.int32)
    lib.oracle_std_cell(ct.byref(cfg), int(cell), N, _ptr(vv), _ptr(alpha), int(init),
                        int(aa_memory), int(kmeans_iters), int(bool(penalised)), _ptr(prm), _ptr(K),
                        _ptr(lnL), _ptr(it),
                        _ptr(na), _ptr(nr), _ptr(km), _ptr(st), _ptr(tr) if trace_cap else None,
                        int(trace_cap), _ptr(nt),
                        _ptr(None if init_params is None else _f64(init_params)),
                        0 if init_params is None else int(np.asarray(init_params).shape[0]))
    return dict(K=int(K[0]), params=prm, lnL=float(lnL[0]), iters=int(it[0]), aa_steps=int(na[0]),
                aa_resets=int(nr[0]), km_passes=int(km[0]), status=int(st[0]),
                Ltrace=tr[: int(nt[0])].copy())


def kmeans(vv, ah, picks, iters: int = 100):
    """The oracle's K-means initialisation of one cell (``vv`` [N, D],
    normalised weights ``ah``) from the given centre indices: (K, params
    [K][P], passes)."""
    lib = _load()
    vv = _f64(vv)
    N, D = vv.shape
    ah = _f64(ah)
    picks = np.ascontiguousarray(picks, dtype=np.int64)
    K = picks.shape[0]
    prm = np.zeros((K, P_of(D)))
    Ko = np.zeros(1, np.int32); ps = np.zeros(1, np.int32)
    rc = lib.oracle_kmeans(D, K, N, _ptr(vv), _ptr(ah), _ptr(picks), int(iters), _ptr(prm), _ptr(Ko), _ptr(ps))
    if rc != 0:
        raise ValueError("oracle_kmeans failed")
    return int(Ko[0]), prm[: int(Ko[0])], int(ps[0])


def aa_affine(A, b, x0, memory: int, iters: int):
    """The oracle's Anderson iteration on G(x) = A x + b: (final iterate,
    residual norm ||G(x_i) - x_i|| per step)."""
    lib = _load()
    A = _f64(A); b = _f64(b); x0 = _f64(x0)
    n = b.shape[0]
    x = np.zeros(n); res = np.zeros(iters)
    rc = lib.oracle_aa_affine(n, _ptr(A), _ptr(b), _ptr(x0), int(memory), int(iters), _ptr(x), _ptr(res))
    if rc != 0:
        raise ValueError("oracle_aa_affine failed")
    return x, res


def penalised_L(D: int, prm, vv, ah) -> float:
    lib = _load()
    prm = _f64(prm)
    vv = _f64(vv).reshape(-1, D)
    ah = _f64(ah)
    return lib.oracle_penalised_L(D, prm.shape[0], _ptr(prm), vv.shape[0], _ptr(vv), _ptr(ah))


def cyclic_tridiag(a, b, c, d) -> np.ndarray:
    lib = _load()
    a, b, c, d = (_f64(t) for t in (a, b, c, d))
    x = np.zeros_like(d)
    if lib.oracle_cyclic_tridiag(d.shape[0], _ptr(a), _ptr(b), _ptr(c), _ptr(d), _ptr(x)) != 0:
        raise ValueError("n < 3")
    return x


def reconstruct(params: dict, K, prm, W, rho_target, out_off, nthreads: int = 1,
                want_raw: bool = False) -> dict:
    """Oracle reconstruction (Sec. 2.4): sampling, Gauss'-law weight
    correction, Lemons projection.  Uses ``params['recon_seed']``."""
    lib = _load()
    cfg = _cfg(params, "recon_seed")
    out_off = np.ascontiguousarray(out_off, dtype=np.int64)
    C = out_off.shape[0] - 1
    D = cfg.D
    Nout = int(out_off[-1])
    K = np.ascontiguousarray(K, dtype=np.int32)
    prm = _f64(prm); W = _f64(W); rho_target = _f64(rho_target)
    assert prm.shape == (C, cfg.Kmax, P_of(D))
    out = dict(x=np.zeros(Nout), v=np.zeros((D, Nout)), alpha=np.zeros(Nout),
               status=np.zeros(C, np.uint32), dA=np.zeros(C))
    raw = np.zeros((D, Nout)) if want_raw else None
    rc = lib.oracle_reconstruct(ct.byref(cfg), C, _ptr(K), _ptr(prm), _ptr(W), _ptr(rho_target),
                                _ptr(out_off), _ptr(out["x"]), _ptr(out["v"]), _ptr(out["alpha"]),
                                _ptr(out["status"]), _ptr(out["dA"]), _ptr(raw), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_reconstruct failed ({rc})")
    if want_raw:
        out["v_raw"] = raw
    return out


def deposit2d(params: dict, cell_off, x, y, alpha) -> np.ndarray:
    """Charge density [Cy * Cx] (node j = jy Cx + jx) of particles sorted by
    cell on the 2D periodic mesh of ``params`` (Cx, Cy, Lx, Ly), tensor
    product B-spline of ``shape_order``."""
    lib = _load()
    cfg = _cfg(params)
    m = _mesh(params)
    cell_off = np.ascontiguousarray(cell_off, dtype=np.int64)
    rho = np.zeros(m.Cx * m.Cy)
    rc = lib.oracle_deposit2d(ct.byref(cfg), ct.byref(m), _ptr(cell_off), _ptr(_f64(x)), _ptr(_f64(y)),
                              _ptr(_f64(alpha)), _ptr(rho))
    if rc != 0:
        raise ValueError(f"oracle_deposit2d failed ({rc})")
    return rho


def reconstruct2d(params: dict, K, prm, W, rho_target, out_off, nthreads: int = 1) -> dict:
    """Oracle reconstruction on the 2D periodic mesh (Sec. 2.4 with the
    tensor-product shape function; dense direct solve, at most 2048
    cells).  Uses ``params['recon_seed']``."""
    lib = _load()
    cfg = _cfg(params, "recon_seed")
    m = _mesh(params)
    out_off = np.ascontiguousarray(out_off, dtype=np.int64)
    C = out_off.shape[0] - 1
    assert C == m.Cx * m.Cy
    D = cfg.D
    Nout = int(out_off[-1])
    K = np.ascontiguousarray(K, dtype=np.int32)
    prm = _f64(prm); W = _f64(W); rho_target = _f64(rho_target)
    assert prm.shape == (C, cfg.Kmax, P_of(D))
    xy = np.zeros((2, Nout))
    out = dict(v=np.zeros((D, Nout)), alpha=np.zeros(Nout), status=np.zeros(C, np.uint32), dA=np.zeros(C))
    rc = lib.oracle_reconstruct2d(ct.byref(cfg), ct.byref(m), _ptr(K), _ptr(prm), _ptr(W),
                                  _ptr(rho_target), _ptr(out_off), _ptr(xy), _ptr(out["v"]),
                                  _ptr(out["alpha"]), _ptr(out["status"]), _ptr(out["dA"]), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_reconstruct2d failed ({rc})")
    out["x"], out["y"] = xy[0], xy[1]
    return out


def moments(params: dict, cell_off, x, v, alpha) -> dict:
    lib = _load()
    cfg = _cfg(params)
    cell_off = np.ascontiguousarray(cell_off, dtype=np.int64)
    C = cell_off.shape[0] - 1
    D = cfg.D
    nm = D * (D + 1) // 2
    x = _f64(x); v = _f64(v); alpha = _f64(alpha)
    out = dict(W=np.zeros(C), p=np.zeros((C, D)), M2=np.zeros((C, nm)), E=np.zeros(C),
               rho=np.zeros(C))
    lib.oracle_moments(ct.byref(cfg), C, _ptr(cell_off), _ptr(x), _ptr(v), _ptr(alpha),
                       _ptr(out["W"]), _ptr(out["p"]), _ptr(out["M2"]), _ptr(out["E"]),
                       _ptr(out["rho"]))
    return out


def mixture_moments(params: dict, K, prm, W) -> dict:
    lib = _load()
    cfg = _cfg(params)
    K = np.ascontiguousarray(K, dtype=np.int32)
    C = K.shape[0]
    D = cfg.D
    nm = D * (D + 1) // 2
    prm = _f64(prm); W = _f64(W)
    out = dict(W=np.zeros(C), p=np.zeros((C, D)), M2=np.zeros((C, nm)), E=np.zeros(C))
    lib.oracle_mixture_moments(ct.byref(cfg), C, _ptr(K), _ptr(prm), _ptr(W), _ptr(out["W"]),
                               _ptr(out["p"]), _ptr(out["M2"]), _ptr(out["E"]))
    return out
