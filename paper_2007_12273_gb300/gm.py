"""Thin Python binding of the C ABI in ``include/gm.h`` (argument marshalling
only).  Tensors are torch CUDA tensors; every computation runs in the
library's CUDA kernels on the current (or given) torch stream.

The library is loaded from the package's ``_lib/libgmcr.so``; a missing
library or a missing GPU raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as ct
import os
import threading

import torch

from . import build as _build

GM_OK = 0
GM_ERR_ARG = -1
GM_ERR_CUDA = -2
GM_ERR_NOMEM = -3
GM_ERR_UNSUPPORTED = -4
ST_EM_MAXSWEEPS = 0x01
ST_COV_NOT_PD = 0x02
ST_TOO_FEW = 0x04
ST_EMPTY = 0x08
ST_DEGENERATE = 0x10
ST_PROJ_SKIPPED = 0x100
ST_NEG_WEIGHT = 0x200
ST_MM_EMPTY_COL = 0x400
ST_NO_MIXTURE = 0x800
ST_MM_NOT_CONVERGED = 0x1000
ST_BAD_RANGE = 0x2000
TUNE_CANDIDATES = 15  # GM_TUNE_CANDIDATES

EXPORTED = ("gm_compress", "gm_reconstruct", "gm_moments", "gm_mixture_moments",
            "gm_last_error", "gm_shutdown", "gm_reconstruct_noalloc", "gm_gemm_bf16",
            "gm_compress_from", "gm_features", "gm_mlp_targets", "gm_mlp_sync",
            "gm_mlp_scratch_bytes", "gm_mlp_forward", "gm_mlp_train_step", "gm_mlp_decode",
            "gm_graph_begin", "gm_graph_end", "gm_graph_launch", "gm_graph_destroy", "gm_autotune",
            "gm_compress_standard", "gm_anderson_affine", "gm_deposit_2d", "gm_reconstruct_2d",
            "gm_autotune_from", "gm_noalloc_limits_ok", "gm_trace_begin", "gm_trace_end",
            "gm_trace_get", "gm_convert")


class GMMlp(ct.Structure):
    """Mirror of ``gm_mlp`` (include/gm.h)."""
    _fields_ = [("D", ct.c_int32), ("Kmax", ct.c_int32), ("F", ct.c_int32), ("H", ct.c_int32),
                ("O", ct.c_int32)] + [(nm, ct.c_void_p * 4) for nm in
                                     ("W", "b", "W16", "WT16", "gW", "gb", "mW", "vW", "mb", "vb")]


class GMConfig(ct.Structure):
    """Mirror of ``gm_config`` (include/gm.h)."""
    _fields_ = [("D", ct.c_int32), ("Kmax", ct.c_int32), ("shape_order", ct.c_int32),
                ("max_sweeps", ct.c_int32), ("tol", ct.c_double), ("seed", ct.c_uint64),
                ("L", ct.c_double), ("q", ct.c_double), ("threads_per_cell", ct.c_int32),
                ("smem_particles", ct.c_int32), ("precision", ct.c_int32),
                ("reserved", ct.c_int32)]


class GMMesh2d(ct.Structure):
    """Mirror of ``gm_mesh2d`` (include/gm.h)."""
    _fields_ = [("Cx", ct.c_int64), ("Cy", ct.c_int64), ("Lx", ct.c_double), ("Ly", ct.c_double)]


def mesh2d(params: dict) -> GMMesh2d:
    """gm_mesh2d from a method-parameter dict with Cx, Cy, Lx, Ly."""
    return GMMesh2d(int(params["Cx"]), int(params["Cy"]), float(params["Lx"]), float(params["Ly"]))


class GMStdOpts(ct.Structure):
    """Mirror of ``gm_std_opts`` (include/gm.h)."""
    _fields_ = [("init", ct.c_int32), ("aa_memory", ct.c_int32), ("kmeans_iters", ct.c_int32),
                ("penalised", ct.c_int32)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libgmcr.so (ctypes).  Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB):
            if build_if_missing:
                _build.build()
            else:
                raise RuntimeError(f"CUDA library {_build.LIB} is missing: run "
                                   "__graft_entry__.build() (nvcc, sm_103a) first")
        lib = ct.CDLL(_build.LIB)
        P, I64, I32 = ct.c_void_p, ct.c_int64, ct.c_int32
        lib.gm_compress.argtypes = [P, I64, I64, P, P, P, I32, P, P, P, P, P, P, P, P, P, P]
        lib.gm_reconstruct.argtypes = [P, I64, P, P, P, P, I64, P, P, P, P, P, P, P]
        lib.gm_reconstruct_noalloc.argtypes = [P, I64, P, P, P, P, I64, P, P, P, P, P, P, P]
        lib.gm_moments.argtypes = [P, I64, I64, P, P, P, I32, P, P, P, P, P, P, P]
        lib.gm_mixture_moments.argtypes = [P, I64, P, P, P, P, P, P, P, P]
        lib.gm_gemm_bf16.argtypes = [I32, I32, I32, P, I32, P, I32, P, I32, P, I32, P, P, I32, P, P]
        lib.gm_compress_from.argtypes = [P, I64, I64, P, P, P, I32, P, P, P, P, P, P, P, P, P, P, P, P]
        lib.gm_features.argtypes = [P, I64, I64, P, P, I32, P, P, P, P]
        lib.gm_mlp_targets.argtypes = [P, I64, P, P, P, I32, P, P, P]
        lib.gm_mlp_sync.argtypes = [P, P]
        lib.gm_mlp_scratch_bytes.argtypes = [P, I32]
        lib.gm_mlp_scratch_bytes.restype = ct.c_size_t
        lib.gm_mlp_forward.argtypes = [P, I32, P, P, ct.c_size_t, P, P, P]
        lib.gm_mlp_train_step.argtypes = [P, I32, P, P, P, ct.c_float, I32, P, ct.c_size_t, P, P, P, P]
        lib.gm_mlp_decode.argtypes = [P, I64, P, I32, P, P, ct.c_float, P, P, P]
        lib.gm_graph_begin.argtypes = [P]
        lib.gm_graph_end.argtypes = [P, ct.POINTER(ct.c_void_p)]
        lib.gm_graph_launch.argtypes = [P, P]
        lib.gm_graph_destroy.argtypes = [P]
        lib.gm_autotune.argtypes = [P, I64, I64, P, P, P, I32, P, I32, ct.POINTER(ct.c_float), P]
        lib.gm_autotune_from.argtypes = [P, I64, I64, P, P, P, I32, P, P, P, I32, ct.POINTER(ct.c_float), P]
        lib.gm_compress_standard.argtypes = [P, P, I64, I64, P, P, P, I32, P] + [P] * 10 + [P]
        lib.gm_anderson_affine.argtypes = [I32, P, P, P, I32, I32, P, P, P]
        lib.gm_deposit_2d.argtypes = [P] * 8
        lib.gm_reconstruct_2d.argtypes = [P, P, P, P, P, P, I64] + [P] * 8
        lib.gm_noalloc_limits_ok.argtypes = []
        lib.gm_trace_begin.argtypes = []
        lib.gm_trace_end.argtypes = []
        lib.gm_trace_get.argtypes = [I32, ct.c_char_p, I32, ct.POINTER(ct.c_double), ct.POINTER(I32)]
        lib.gm_convert.argtypes = [I32, I64, P, P, P]
        for f in ("gm_compress", "gm_reconstruct", "gm_moments", "gm_mixture_moments", "gm_shutdown",
                  "gm_reconstruct_noalloc", "gm_gemm_bf16", "gm_compress_from", "gm_features",
                  "gm_mlp_targets", "gm_mlp_sync", "gm_mlp_forward", "gm_mlp_train_step",
                  "gm_mlp_decode", "gm_graph_begin", "gm_graph_end", "gm_graph_launch",
                  "gm_graph_destroy", "gm_autotune", "gm_compress_standard", "gm_anderson_affine",
                  "gm_deposit_2d", "gm_reconstruct_2d", "gm_autotune_from", "gm_noalloc_limits_ok",
                  "gm_trace_begin", "gm_trace_end", "gm_trace_get", "gm_convert"):
            getattr(lib, f).restype = ct.c_int
        lib.gm_last_error.restype = ct.c_char_p
        _lib = lib
        return lib


def config(params: dict, seed_key: str = "seed", **over) -> GMConfig:
    """gm_config from a plain method-parameter dict (see workloads)."""
    c = GMConfig()
    c.D = int(params["D"])
    c.Kmax = int(params["Kmax"])
    c.shape_order = int(params["shape_order"])
    c.max_sweeps = int(params.get("max_sweeps", 1000))
    c.tol = float(params.get("tol", 1e-6))
    c.seed = int(params.get(seed_key, 1))
    c.L = float(params["L"])
    c.q = float(params.get("q", 1.0))
    c.threads_per_cell = int(over.get("threads_per_cell", params.get("threads_per_cell", 0)))
    c.smem_particles = int(over.get("smem_particles", params.get("smem_particles", 0)))
    c.precision = int(over.get("precision", params.get("precision", 0)))
    c.reserved = 0
    return c


def P_of(D: int) -> int:
    return 1 + D + D * (D + 1) // 2


def _ptr(t):
    return ct.c_void_p(t.data_ptr()) if t is not None else None


def _stream_ptr(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ct.c_void_p(s.cuda_stream)


# per-cell status words: int32 or uint32 tensors
_STATUS = (torch.int32,) + ((torch.uint32,) if hasattr(torch, "uint32") else ())


def _check(t, dtype, name, numel: int | None = None):
    """A contiguous CUDA tensor of ``dtype`` (or of one of a tuple of dtypes)
    with at least ``numel`` elements: the C call reads or writes that many
    through its pointer, so a shorter tensor is refused here."""
    if t is None:
        raise ValueError(f"{name} is required")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    dts = dtype if isinstance(dtype, tuple) else (dtype,)
    if t.dtype not in dts:
        raise ValueError(f"{name} must be {' or '.join(map(str, dts))}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} has {t.numel()} elements; the call needs at least {numel}")


def _check_out(out: dict, required: dict, optional: dict | None = None):
    """Caller-supplied outputs: every ``required`` key (name -> (dtype,
    numel)) present and valid, every ``optional`` key valid if present."""
    for k, (dt, ne) in required.items():
        if k not in out:
            raise ValueError(f"out is missing {k!r}")
        _check(out[k], dt, f"out[{k!r}]", ne)
    for k, (dt, ne) in (optional or {}).items():
        if out.get(k) is not None:
            _check(out[k], dt, f"out[{k!r}]", ne)


def _check_particles(cfg: GMConfig, cell_off, x, v, alpha, n: int):
    """Particles in CSR order: cell_off [C+1] int64, x [n] f64 (optional),
    v [D, n] f32 / f64, alpha [n] f64."""
    _check(cell_off, torch.int64, "cell_off")
    if x is not None:
        _check(x, torch.float64, "x", n)
    _check(alpha, torch.float64, "alpha", n)
    if v is None or v.dtype not in (torch.float32, torch.float64) or tuple(v.shape) != (cfg.D, n):
        raise ValueError("v must be [D, n] float32/float64")
    _check(v, v.dtype, "v")


def _rc(lib, rc, what):
    if rc != GM_OK:
        raise RuntimeError(f"{what} failed ({rc}): {lib.gm_last_error().decode()}")


def gm_compress(cfg: GMConfig, cell_off, x, v, alpha, stream=None, out=None, init_K=None,
                init_params=None) -> dict:
    """Per-cell adaptive GM fit.  cell_off [C+1] int64, x [n] f64,
    v [D, n] f32/f64, alpha [n] f64 (all CUDA).  Returns the outputs of
    ``gm_compress`` as CUDA tensors (``out`` may supply them).  With
    ``init_K`` / ``init_params`` the fit starts from those mixtures
    (``gm_compress_from``)."""
    lib = load()
    C = cell_off.shape[0] - 1
    n = alpha.shape[0]
    D = cfg.D
    KP = C * cfg.Kmax * P_of(D)
    _check_particles(cfg, cell_off, x, v, alpha, n)
    dev = alpha.device
    if out is not None:
        req = dict(K=(torch.int32, C), params=(torch.float64, KP), W=(torch.float64, C),
                   lnL=(torch.float64, C), sweeps=(torch.int32, C), kwork=(torch.int32, C),
                   status=(_STATUS, C))
        if x is not None:
            req["rho_target"] = (torch.float64, C)
        _check_out(out, req)
    if out is None:
        out = dict(K=torch.empty(C, dtype=torch.int32, device=dev),
                   params=torch.empty((C, cfg.Kmax, P_of(D)), dtype=torch.float64, device=dev),
                   W=torch.empty(C, dtype=torch.float64, device=dev),
                   rho_target=torch.empty(C, dtype=torch.float64, device=dev) if x is not None else None,
                   lnL=torch.empty(C, dtype=torch.float64, device=dev),
                   sweeps=torch.empty(C, dtype=torch.int32, device=dev),
                   kwork=torch.empty(C, dtype=torch.int32, device=dev),
                   status=torch.empty(C, dtype=torch.int32, device=dev))
    vf = 1 if v.dtype == torch.float64 else 0
    tail = (_ptr(out["K"]), _ptr(out["params"]), _ptr(out["W"]),
            _ptr(out["rho_target"]) if x is not None else None,
            _ptr(out["lnL"]), _ptr(out["sweeps"]), _ptr(out["kwork"]), _ptr(out["status"]),
            _stream_ptr(stream))
    if init_K is None:
        rc = lib.gm_compress(ct.byref(cfg), C, n, _ptr(cell_off), _ptr(x), _ptr(v), vf,
                             _ptr(alpha), *tail)
        _rc(lib, rc, "gm_compress")
    else:
        _check(init_K, torch.int32, "init_K", C)
        _check(init_params, torch.float64, "init_params", KP)
        rc = lib.gm_compress_from(ct.byref(cfg), C, n, _ptr(cell_off), _ptr(x), _ptr(v), vf,
                                  _ptr(alpha), _ptr(init_K), _ptr(init_params), *tail)
        _rc(lib, rc, "gm_compress_from")
    return out


def _check_mixtures(cfg: GMConfig, C: int, K, params, W, rho_target=None):
    """Per-cell mixtures as gm_compress writes them: K [C] int32, params
    [C][Kmax][P] f64, W [C] f64 (and rho_target [C] f64)."""
    _check(K, torch.int32, "K", C)
    _check(params, torch.float64, "params", C * cfg.Kmax * P_of(cfg.D))
    _check(W, torch.float64, "W", C)
    if rho_target is not None:
        _check(rho_target, torch.float64, "rho_target", C)


def _check_recon_out(out: dict, D: int, C: int, n_out: int, two_d: bool = False):
    """Caller-supplied reconstruction outputs (dA optional)."""
    req = dict(x=(torch.float64, n_out), v=(torch.float64, D * n_out),
               alpha=(torch.float64, n_out), status=(_STATUS, C))
    if two_d:
        req["y"] = (torch.float64, n_out)
    _check_out(out, req, dict(dA=(torch.float64, C)))


def gm_reconstruct(cfg: GMConfig, K, params, W, rho_target, out_off, n_out: int | None = None,
                   stream=None, want_dA: bool = False, out=None) -> dict:
    """Resample every cell: returns x [n'], v [D, n'], alpha [n'], status [C]
    (and dA [C] if asked).  ``n_out`` = out_off[-1] (read from the device if
    not given)."""
    lib = load()
    C = out_off.shape[0] - 1
    D = cfg.D
    _check_mixtures(cfg, C, K, params, W, rho_target)
    _check(out_off, torch.int64, "out_off")
    if n_out is None:
        n_out = int(out_off[-1].item())
    dev = W.device
    if out is not None:
        _check_recon_out(out, D, C, n_out)
    if out is None:
        out = dict(x=torch.empty(n_out, dtype=torch.float64, device=dev),
                   v=torch.empty((D, n_out), dtype=torch.float64, device=dev),
                   alpha=torch.empty(n_out, dtype=torch.float64, device=dev),
                   status=torch.empty(C, dtype=torch.int32, device=dev))
        if want_dA:
            out["dA"] = torch.empty(C, dtype=torch.float64, device=dev)
    rc = lib.gm_reconstruct(ct.byref(cfg), C, _ptr(K), _ptr(params), _ptr(W), _ptr(rho_target),
                            n_out, _ptr(out_off), _ptr(out["x"]), _ptr(out["v"]),
                            _ptr(out["alpha"]), _ptr(out["status"]), _ptr(out.get("dA")),
                            _stream_ptr(stream))
    _rc(lib, rc, "gm_reconstruct")
    return out


def gm_reconstruct_noalloc(cfg: GMConfig, K, params, W, rho_target, out_off, out: dict,
                           n_out: int | None = None, stream=None) -> dict:
    """``gm_reconstruct`` without device allocation inside the library: the
    scratch is the library's fixed static array (at most 32768 cells per
    call) and every output tensor is supplied by the caller in ``out``
    (keys x, v, alpha, status, optionally dA).  ``n_out`` = out_off[-1]
    (read from the device if not given); a cell whose out_off range does
    not fit n_out is skipped on the device with GM_ST_BAD_RANGE."""
    lib = load()
    C = out_off.shape[0] - 1
    _check_mixtures(cfg, C, K, params, W, rho_target)
    _check(out_off, torch.int64, "out_off")
    if n_out is None:
        n_out = int(out_off[-1].item()) if C > 0 else 0
    _check_recon_out(out, cfg.D, C, int(n_out))
    rc = lib.gm_reconstruct_noalloc(ct.byref(cfg), C, _ptr(K), _ptr(params), _ptr(W),
                                    _ptr(rho_target), int(n_out), _ptr(out_off), _ptr(out["x"]),
                                    _ptr(out["v"]), _ptr(out["alpha"]), _ptr(out["status"]),
                                    _ptr(out.get("dA")), _stream_ptr(stream))
    _rc(lib, rc, "gm_reconstruct_noalloc")
    return out


def gm_moments(cfg: GMConfig, cell_off, x, v, alpha, stream=None) -> dict:
    lib = load()
    C = cell_off.shape[0] - 1
    n = alpha.shape[0]
    D = cfg.D
    dev = alpha.device
    nm = D * (D + 1) // 2
    _check_particles(cfg, cell_off, x, v, alpha, n)
    out = dict(W=torch.empty(C, dtype=torch.float64, device=dev),
               p=torch.empty((C, D), dtype=torch.float64, device=dev),
               M2=torch.empty((C, nm), dtype=torch.float64, device=dev),
               E=torch.empty(C, dtype=torch.float64, device=dev),
               rho=torch.empty(C, dtype=torch.float64, device=dev))
    rc = lib.gm_moments(ct.byref(cfg), C, n, _ptr(cell_off), _ptr(x), _ptr(v),
                        1 if v.dtype == torch.float64 else 0, _ptr(alpha), _ptr(out["W"]),
                        _ptr(out["p"]), _ptr(out["M2"]), _ptr(out["E"]), _ptr(out["rho"]),
                        _stream_ptr(stream))
    _rc(lib, rc, "gm_moments")
    return out


def gm_mixture_moments(cfg: GMConfig, K, params, W, stream=None) -> dict:
    lib = load()
    C = K.shape[0]
    D = cfg.D
    dev = W.device
    nm = D * (D + 1) // 2
    _check_mixtures(cfg, C, K, params, W)
    out = dict(W=torch.empty(C, dtype=torch.float64, device=dev),
               p=torch.empty((C, D), dtype=torch.float64, device=dev),
               M2=torch.empty((C, nm), dtype=torch.float64, device=dev),
               E=torch.empty(C, dtype=torch.float64, device=dev))
    rc = lib.gm_mixture_moments(ct.byref(cfg), C, _ptr(K), _ptr(params), _ptr(W), _ptr(out["W"]),
                                _ptr(out["p"]), _ptr(out["M2"]), _ptr(out["E"]),
                                _stream_ptr(stream))
    _rc(lib, rc, "gm_mixture_moments")
    return out


def gm_gemm_bf16(A, B, bias=None, relu=False, mask=None, out_f32=None, out_bf16=None,
                 err=None, stream=None):
    """C = A B^T (+bias) (ReLU) (mask) on the tcgen05 tensor cores.  A [M,K],
    B [N,K] bf16 (row-major, K contiguous); returns the FP32 output (or the
    BF16 one if only that is requested)."""
    lib = load()
    M, K = A.shape
    N = B.shape[0]
    for t_, nm_ in ((A, "A"), (B, "B")):
        if not t_.is_cuda or t_.dtype != torch.bfloat16 or t_.stride(1) != 1:
            raise ValueError(f"{nm_} must be a CUDA bf16 matrix with unit column stride")
    if out_f32 is None and out_bf16 is None:
        out_f32 = torch.empty((M, N), dtype=torch.float32, device=A.device)
    ldc = (out_f32 if out_f32 is not None else out_bf16).stride(0)
    rc = lib.gm_gemm_bf16(M, N, K, _ptr(A), A.stride(0), _ptr(B), B.stride(0), _ptr(bias),
                          1 if relu else 0, _ptr(mask), mask.stride(0) if mask is not None else 0,
                          _ptr(out_f32), _ptr(out_bf16), ldc, _ptr(err), _stream_ptr(stream))
    _rc(lib, rc, "gm_gemm_bf16")
    return out_f32 if out_f32 is not None else out_bf16


# ---------------------------------------------------------------------------
# learned initialisation
# ---------------------------------------------------------------------------
def feat_width(D: int) -> int:
    return 128 if D == 1 else 576


def slot_size(D: int) -> int:
    return 2 + 2 * D + D * (D - 1) // 2


def out_width(D: int, Kmax: int) -> int:
    return (Kmax * slot_size(D) + 15) // 16 * 16


def gm_features(cfg: GMConfig, cell_off, v, alpha, stream=None, out=None):
    """Per-cell features (BF16 [C][F]) and whitening statistics
    (FP64 [C][2D]: mean, sd); ``out`` = (feat, wstat) may supply them."""
    lib = load()
    C = cell_off.shape[0] - 1
    n = alpha.shape[0]
    D = cfg.D
    _check_particles(cfg, cell_off, None, v, alpha, n)
    if out is None:
        feat = torch.empty((C, feat_width(D)), dtype=torch.bfloat16, device=alpha.device)
        wstat = torch.empty((C, 2 * D), dtype=torch.float64, device=alpha.device)
    else:
        feat, wstat = out
        _check(feat, torch.bfloat16, "feat", C * feat_width(D))
        _check(wstat, torch.float64, "wstat", C * 2 * D)
    rc = lib.gm_features(ct.byref(cfg), C, n, _ptr(cell_off), _ptr(v),
                         1 if v.dtype == torch.float64 else 0, _ptr(alpha), _ptr(feat),
                         _ptr(wstat), _stream_ptr(stream))
    _rc(lib, rc, "gm_features")
    return feat, wstat


def gm_mlp_targets(cfg: GMConfig, K, params, wstat, stream=None):
    lib = load()
    C = K.shape[0]
    O = out_width(cfg.D, cfg.Kmax)
    _check(K, torch.int32, "K", C)
    _check(params, torch.float64, "params", C * cfg.Kmax * P_of(cfg.D))
    _check(wstat, torch.float64, "wstat", C * 2 * cfg.D)
    T = torch.empty((C, O), dtype=torch.float32, device=K.device)
    Mk = torch.empty((C, O), dtype=torch.float32, device=K.device)
    rc = lib.gm_mlp_targets(ct.byref(cfg), C, _ptr(K), _ptr(params), _ptr(wstat), O, _ptr(T),
                            _ptr(Mk), _stream_ptr(stream))
    _rc(lib, rc, "gm_mlp_targets")
    return T, Mk


def gm_mlp_decode(cfg: GMConfig, out, wstat, cell_off, stream=None, dest=None,
                  presence_logit: float = 0.0):
    """Initial mixtures (K0 [C] int32, params [C][Kmax][P] f64) from the
    network output (slots with presence logit above ``presence_logit``);
    ``dest`` = (K0, params) may supply them."""
    lib = load()
    C = cell_off.shape[0] - 1
    _check(cell_off, torch.int64, "cell_off")
    _check(out, torch.float32, "out")
    if out.dim() != 2 or out.shape[0] < C or out.shape[1] < cfg.Kmax * slot_size(cfg.D):
        raise ValueError(f"out must be [C, >= {cfg.Kmax * slot_size(cfg.D)}] float32")
    _check(wstat, torch.float64, "wstat", C * 2 * cfg.D)
    if dest is None:
        K0 = torch.empty(C, dtype=torch.int32, device=out.device)
        prm = torch.empty((C, cfg.Kmax, P_of(cfg.D)), dtype=torch.float64, device=out.device)
    else:
        K0, prm = dest
        _check(K0, torch.int32, "K0", C)
        _check(prm, torch.float64, "params", C * cfg.Kmax * P_of(cfg.D))
    rc = lib.gm_mlp_decode(ct.byref(cfg), C, _ptr(out), out.shape[1], _ptr(wstat), _ptr(cell_off),
                           float(presence_logit), _ptr(K0), _ptr(prm), _stream_ptr(stream))
    _rc(lib, rc, "gm_mlp_decode")
    return K0, prm


class Net:
    """Device buffers of the learned-initialisation network (FP32 masters,
    BF16 copies and transposes, gradients, Adam moments) and the gm_mlp
    struct that points at them."""

    def __init__(self, D: int, Kmax: int, device="cuda"):
        self.D, self.Kmax = D, Kmax
        self.F, self.H, self.O = feat_width(D), 256, out_width(D, Kmax)
        self.device = torch.device(device)
        shapes = [(self.H, self.F), (self.H, self.H), (self.H, self.H), (self.O, self.H)]
        z = lambda *sh, dt=torch.float32: torch.zeros(sh, dtype=dt, device=self.device)
        self.W = [z(*sh) for sh in shapes]
        self.b = [z(sh[0]) for sh in shapes]
        self.W16 = [z(*sh, dt=torch.bfloat16) for sh in shapes]
        self.WT16 = [z(sh[1], sh[0], dt=torch.bfloat16) for sh in shapes]
        self.gW = [z(*sh) for sh in shapes]
        self.gb = [z(sh[0]) for sh in shapes]
        self.mW = [z(*sh) for sh in shapes]
        self.vW = [z(*sh) for sh in shapes]
        self.mb = [z(sh[0]) for sh in shapes]
        self.vb = [z(sh[0]) for sh in shapes]
        self.step = 0
        self._scratch = None
        self.err = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.s = GMMlp()
        self.s.D, self.s.Kmax, self.s.F, self.s.H, self.s.O = D, Kmax, self.F, self.H, self.O
        for nm in ("W", "b", "W16", "WT16", "gW", "gb", "mW", "vW", "mb", "vb"):
            arr = getattr(self.s, nm)
            for i, t in enumerate(getattr(self, nm)):
                arr[i] = t.data_ptr()

    def init_weights(self, seed: int = 0):
        """He-normal weights, zero biases (seeded on the host)."""
        g = torch.Generator().manual_seed(seed)
        for W in self.W:
            n, k = W.shape
            W.copy_(torch.randn((n, k), generator=g, dtype=torch.float64).mul_((2.0 / k) ** 0.5))
        for b in self.b:
            b.zero_()
        self.sync()

    def load(self, Ws, bs):
        for W, w in zip(self.W, Ws):
            W.copy_(torch.as_tensor(w, dtype=torch.float32))
        for b, bb in zip(self.b, bs):
            b.copy_(torch.as_tensor(bb, dtype=torch.float32))
        self.sync()

    def sync(self, stream=None):
        lib = load()
        _rc(lib, lib.gm_mlp_sync(ct.byref(self.s), _stream_ptr(stream)), "gm_mlp_sync")

    def scratch(self, M: int):
        lib = load()
        need = lib.gm_mlp_scratch_bytes(ct.byref(self.s), M)
        if self._scratch is None or self._scratch.numel() < need:
            self._scratch = torch.empty(need, dtype=torch.uint8, device=self.device)
        return self._scratch

    def _check_rows(self, X):
        _check(X, torch.bfloat16, "X")
        if X.dim() != 2 or X.shape[1] != self.F:
            raise ValueError(f"X must be [M, {self.F}] bfloat16")
        return X.shape[0]

    def forward(self, X, out=None, stream=None):
        lib = load()
        M = self._check_rows(X)
        if out is None:
            out = torch.empty((M, self.O), dtype=torch.float32, device=self.device)
        _check(out, torch.float32, "out", M * self.O)
        sc = self.scratch(M)
        rc = lib.gm_mlp_forward(ct.byref(self.s), M, _ptr(X), _ptr(sc), sc.numel(), _ptr(out),
                                _ptr(self.err), _stream_ptr(stream))
        _rc(lib, rc, "gm_mlp_forward")
        return out

    def train_step(self, X, T, Mk, lr: float, loss=None, out=None, stream=None):
        """One step; returns the device loss accumulator.  lr <= 0 computes
        gradients only."""
        lib = load()
        M = self._check_rows(X)
        _check(T, torch.float32, "T", M * self.O)
        _check(Mk, torch.float32, "Mk", M * self.O)
        if out is None:
            out = torch.empty((M, self.O), dtype=torch.float32, device=self.device)
        if loss is None:
            loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        _check(out, torch.float32, "out", M * self.O)
        _check(loss, torch.float64, "loss", 1)
        if lr > 0:
            self.step += 1
        sc = self.scratch(M)
        rc = lib.gm_mlp_train_step(ct.byref(self.s), M, _ptr(X), _ptr(T), _ptr(Mk), float(lr),
                                   self.step, _ptr(sc), sc.numel(), _ptr(out), _ptr(loss),
                                   _ptr(self.err), _stream_ptr(stream))
        _rc(lib, rc, "gm_mlp_train_step")
        return loss


def gm_autotune(cfg: GMConfig, cell_off, x, v, alpha, sweeps_per_trial: int = 0, stream=None,
                init_K=None, init_params=None):
    """Times the EM launch shapes on a sample of the batch and writes the
    fastest into ``cfg`` (threads_per_cell, smem_particles).  Returns the
    trial times in ms (TUNE_CANDIDATES entries, -1 = not run; candidate i
    has threads_per_cell (64, 128, 256)[i % 3] and tile i // 3)."""
    lib = load()
    C = cell_off.shape[0] - 1
    n = x.shape[0]
    _check_particles(cfg, cell_off, x, v, alpha, n)
    t = (ct.c_float * TUNE_CANDIDATES)()
    vf = 1 if v.dtype == torch.float64 else 0
    if init_K is None:
        rc = lib.gm_autotune(ct.byref(cfg), C, n, _ptr(cell_off), _ptr(x), _ptr(v), vf, _ptr(alpha),
                             int(sweeps_per_trial), t, _stream_ptr(stream))
        _rc(lib, rc, "gm_autotune")
    else:  # trials from the supplied initial mixtures (gm_autotune_from)
        _check(init_K, torch.int32, "init_K", C)
        _check(init_params, torch.float64, "init_params", C * cfg.Kmax * P_of(cfg.D))
        rc = lib.gm_autotune_from(ct.byref(cfg), C, n, _ptr(cell_off), _ptr(x), _ptr(v), vf,
                                  _ptr(alpha), _ptr(init_K), _ptr(init_params), int(sweeps_per_trial),
                                  t, _stream_ptr(stream))
        _rc(lib, rc, "gm_autotune_from")
    return list(t)


class Graph:
    """A CUDA graph of library calls, captured natively (gm_graph_begin /
    gm_graph_end).  Use as a context manager on a non-default stream; every
    library call inside must target that stream and write into buffers that
    exist before the capture (``keep`` holds references to them for the
    graph's lifetime).  ``launch`` replays the calls."""

    def __init__(self, stream=None):
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle = None
        self._keep = []

    def keep(self, *objs):
        self._keep.extend(objs)
        return objs[0] if len(objs) == 1 else objs

    def __enter__(self):
        lib = load()
        _rc(lib, lib.gm_graph_begin(_stream_ptr(self.stream)), "gm_graph_begin")
        return self

    def __exit__(self, exc_type, exc, tb):
        lib = load()
        h = ct.c_void_p()
        rc = lib.gm_graph_end(_stream_ptr(self.stream), ct.byref(h))
        if exc_type is not None:
            if rc == GM_OK:
                lib.gm_graph_destroy(h)
            return False
        _rc(lib, rc, "gm_graph_end")
        self.handle = h
        return False

    def launch(self, stream=None):
        lib = load()
        _rc(lib, lib.gm_graph_launch(self.handle, _stream_ptr(stream if stream is not None else self.stream)),
            "gm_graph_launch")

    def close(self):
        if self.handle is not None:
            lib = load()
            lib.gm_graph_destroy(self.handle)
            self.handle = None
        self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gm_compress_standard(cfg: GMConfig, cell_off, x, v, alpha, init: int = 0, aa_memory: int = 0,
                         kmeans_iters: int = 0, stream=None, out=None, penalised: bool = False) -> dict:
    """Standard (non-adaptive) EM with optional K-means initialisation
    (``init`` = 1) and Anderson acceleration (``aa_memory`` > 0): the
    acceleration study of Sec. 4; ``penalised`` runs the simultaneous EM
    with the penalised weights and annihilation instead.  Returns the
    outputs of ``gm_compress_standard`` as CUDA tensors (``out`` may supply
    them)."""
    lib = load()
    C = cell_off.shape[0] - 1
    n = x.shape[0]
    D = cfg.D
    _check_particles(cfg, cell_off, x, v, alpha, n)
    dev = x.device
    if out is not None:
        _check_out(out, dict(K=(torch.int32, C), params=(torch.float64, C * cfg.Kmax * P_of(D)),
                             W=(torch.float64, C), rho_target=(torch.float64, C),
                             lnL=(torch.float64, C), iters=(torch.int32, C),
                             aa_steps=(torch.int32, C), aa_resets=(torch.int32, C),
                             km_passes=(torch.int32, C), status=(_STATUS, C)))
    if out is None:
        i32 = lambda: torch.empty(C, dtype=torch.int32, device=dev)
        out = dict(K=i32(), params=torch.empty((C, cfg.Kmax, P_of(D)), dtype=torch.float64, device=dev),
                   W=torch.empty(C, dtype=torch.float64, device=dev),
                   rho_target=torch.empty(C, dtype=torch.float64, device=dev),
                   lnL=torch.empty(C, dtype=torch.float64, device=dev),
                   iters=i32(), aa_steps=i32(), aa_resets=i32(), km_passes=i32(), status=i32())
    opts = GMStdOpts(int(init), int(aa_memory), int(kmeans_iters), int(bool(penalised)))
    rc = lib.gm_compress_standard(ct.byref(cfg), ct.byref(opts), C, n, _ptr(cell_off), _ptr(x), _ptr(v),
                                  1 if v.dtype == torch.float64 else 0, _ptr(alpha), _ptr(out["K"]),
                                  _ptr(out["params"]), _ptr(out["W"]), _ptr(out["rho_target"]),
                                  _ptr(out["lnL"]), _ptr(out["iters"]), _ptr(out["aa_steps"]),
                                  _ptr(out["aa_resets"]), _ptr(out["km_passes"]), _ptr(out["status"]),
                                  _stream_ptr(stream))
    _rc(lib, rc, "gm_compress_standard")
    return out


def gm_deposit_2d(cfg: GMConfig, mesh: GMMesh2d, cell_off, x, y, alpha=None, stream=None, out=None):
    """Charge density [Cy * Cx] on the 2D mesh (node jy * Cx + jx) of
    particles sorted by cell; ``alpha`` None = unit weights."""
    lib = load()
    C = mesh.Cx * mesh.Cy
    if cell_off.shape[0] != C + 1:
        raise ValueError("cell_off must have Cx * Cy + 1 entries")
    _check(cell_off, torch.int64, "cell_off")
    _check(x, torch.float64, "x")
    _check(y, torch.float64, "y")
    if alpha is not None:
        _check(alpha, torch.float64, "alpha")
    if out is None:
        out = torch.empty(C, dtype=torch.float64, device=x.device)
    else:
        _check(out, torch.float64, "out", C)
    rc = lib.gm_deposit_2d(ct.byref(cfg), ct.byref(mesh), _ptr(cell_off), _ptr(x), _ptr(y), _ptr(alpha),
                           _ptr(out), _stream_ptr(stream))
    _rc(lib, rc, "gm_deposit_2d")
    return out


def gm_reconstruct_2d(cfg: GMConfig, mesh: GMMesh2d, K, params, W, rho_target, out_off,
                      n_out: int | None = None, stream=None, want_dA: bool = False, out=None) -> dict:
    """Resample every cell of the 2D mesh: x, y [n'], v [D, n'], alpha [n'],
    status [C] (and dA [C] if asked)."""
    lib = load()
    C = mesh.Cx * mesh.Cy
    D = cfg.D
    if out_off.shape[0] != C + 1:
        raise ValueError("out_off must have Cx * Cy + 1 entries")
    _check_mixtures(cfg, C, K, params, W, rho_target)
    _check(out_off, torch.int64, "out_off")
    if n_out is None:
        n_out = int(out_off[-1].item())
    dev = W.device
    if out is not None:
        _check_recon_out(out, D, C, n_out, two_d=True)
    if out is None:
        out = dict(x=torch.empty(n_out, dtype=torch.float64, device=dev),
                   y=torch.empty(n_out, dtype=torch.float64, device=dev),
                   v=torch.empty((D, n_out), dtype=torch.float64, device=dev),
                   alpha=torch.empty(n_out, dtype=torch.float64, device=dev),
                   status=torch.empty(C, dtype=torch.int32, device=dev))
        if want_dA:
            out["dA"] = torch.empty(C, dtype=torch.float64, device=dev)
    rc = lib.gm_reconstruct_2d(ct.byref(cfg), ct.byref(mesh), _ptr(K), _ptr(params), _ptr(W),
                               _ptr(rho_target), n_out, _ptr(out_off), _ptr(out["x"]), _ptr(out["y"]),
                               _ptr(out["v"]), _ptr(out["alpha"]), _ptr(out["status"]),
                               _ptr(out.get("dA")), _stream_ptr(stream))
    _rc(lib, rc, "gm_reconstruct_2d")
    return out


def gm_anderson_affine(A, b, x0, memory: int, iters: int, stream=None):
    """The standard-EM kernel's Anderson step on G(x) = A x + b (FP64 CUDA
    tensors): (last iterate, residual norm per step)."""
    lib = load()
    n = b.shape[0]
    for t, nm in ((A, "A"), (b, "b"), (x0, "x0")):
        _check(t, torch.float64, nm)
    x = torch.empty(n, dtype=torch.float64, device=b.device)
    res = torch.empty(max(iters, 1), dtype=torch.float64, device=b.device)
    rc = lib.gm_anderson_affine(n, _ptr(A), _ptr(b), _ptr(x0), int(memory), int(iters), _ptr(x), _ptr(res),
                                _stream_ptr(stream))
    _rc(lib, rc, "gm_anderson_affine")
    return x, res[:iters]


def gm_convert(x, stream=None):
    """The library's integer-pipe conversions: an FP32 CUDA tensor to FP64
    (exact), an FP64 one to FP32 (mantissa truncated toward zero)."""
    lib = load()
    if not x.is_cuda or not x.is_contiguous() or x.dtype not in (torch.float32, torch.float64):
        raise ValueError("x must be a contiguous CUDA float32 or float64 tensor")
    d = 0 if x.dtype == torch.float32 else 1
    out = torch.empty(x.shape, dtype=torch.float64 if d == 0 else torch.float32, device=x.device)
    _rc(lib, lib.gm_convert(d, x.numel(), _ptr(x), _ptr(out), _stream_ptr(stream)), "gm_convert")
    return out


class Trace:
    """Per-kernel device times of the library's calls inside a ``with``
    block (``gm_trace_begin`` / ``gm_trace_end``): ``.times`` maps kernel
    name -> (milliseconds, launches) after the block."""

    def __enter__(self):
        lib = load()
        _rc(lib, lib.gm_trace_begin(), "gm_trace_begin")
        self.times = {}
        return self

    def __exit__(self, exc_type, exc, tb):
        lib = load()
        n = lib.gm_trace_end()
        if n < 0:
            _rc(lib, n, "gm_trace_end")
        buf = ct.create_string_buffer(128)
        ms = ct.c_double()
        cnt = ct.c_int32()
        for i in range(n):
            _rc(lib, lib.gm_trace_get(i, buf, 128, ct.byref(ms), ct.byref(cnt)), "gm_trace_get")
            self.times[buf.value.decode()] = (ms.value, cnt.value)
        return False
