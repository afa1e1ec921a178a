"""ORACLE -- test infrastructure only.

A plain FP64 CPU implementation of EPLL / fast-EPLL (the C file
``epll_oracle.c`` next to this one) with a ctypes wrapper.  Only the tests,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg use it; the
CUDA library never imports, links or calls anything here, and this package
imports nothing from the library.

Functions follow the paper's steps (see the C file's header for the
equation numbering and the readings taken where the paper is silent).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "epll_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libepll_oracle.so")
_lock = threading.Lock()
_lib = None

P = 64
FULL, FRACTION, JITTER, REGULAR, VALID = 0, 1, 2, 3, 4
DENOISE, PIXELWISE, CONV, SR = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (strict IEEE: no fast-math, no -march)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_SO)
            d, i, u64, vp = C.c_double, C.c_int, C.c_uint64, C.c_void_p
            lib.or_rng_u64.restype = u64
            lib.or_rng_u64.argtypes = [u64, u64, u64]
            lib.or_splitmix64_nth.restype = u64
            lib.or_splitmix64_nth.argtypes = [u64, u64]
            lib.or_flat_tail.argtypes = [i, vp, i, d, vp, vp]
            lib.or_sample_full.argtypes = [i, i, vp]
            lib.or_sample_fraction.argtypes = [i, i, d, u64, i, vp]
            lib.or_sample_jitter.argtypes = [i, i, i, u64, i, vp]
            lib.or_sample_regular.argtypes = [i, i, i, vp]
            lib.or_sample_valid.argtypes = [i, i, vp]
            lib.or_valid_weights.argtypes = [i, i, vp]
            lib.or_valid_weights.restype = None
            lib.or_xupdate_weighted.argtypes = [i, vp, vp, i, i, vp, vp, vp, i, i, d, i, vp]
            lib.or_xupdate_weighted.restype = None
            lib.or_scores.argtypes = [i, vp, vp, vp, vp, vp, d, vp, i, i, vp, i, vp]
            lib.or_scores.restype = None
            lib.or_patch_step.argtypes = [i, vp, vp, vp, vp, vp, d, vp, i, i, vp, i, vp,
                                          vp, vp, vp, vp]
            lib.or_dft2_real.argtypes = [vp, i, i, vp, vp]
            lib.or_dft2_real.restype = None
            lib.or_lambda.restype = d
            lib.or_lambda.argtypes = [i, vp, vp, i, i, i, i, d]
            lib.or_xupdate_pixelwise.argtypes = [vp, vp, vp, i, d, vp]
            lib.or_xupdate_pixelwise.restype = None
            lib.or_xupdate_conv.argtypes = [vp, i, i, vp, vp, i, i, d, vp]
            lib.or_xupdate_conv.restype = None
            lib.or_init_conv.argtypes = [vp, i, i, vp, i, i, d, vp]
            lib.or_init_conv.restype = None
            lib.or_init_cg.argtypes = [vp, vp, i, i, d, i, vp]
            lib.or_init_cg.restype = None
            lib.or_restore.argtypes = [i, vp, vp, vp, vp, vp, vp, i, i, i, vp, vp, i, i, i, d,
                                       vp, i, i, d, u64, i, vp, vp, vp, vp]
            lib.or_sr_apply.argtypes = [vp, i, i, vp, i, i, i, vp]
            lib.or_sr_apply.restype = None
            lib.or_sr_adjoint.argtypes = [vp, i, i, vp, i, i, i, vp]
            lib.or_sr_adjoint.restype = None
            lib.or_xupdate_sr.argtypes = [vp, i, i, vp, vp, i, i, i, d, vp]
            lib.or_init_sr.argtypes = [vp, i, i, vp, i, i, i, d, vp]
            lib.or_lambda_sr.restype = d
            lib.or_lambda_sr.argtypes = [vp, i, i, i, i, i, d]
            _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a):
    return None if a is None else a.ctypes.data


# --------------------------------------------------------------------------
def rng_u64(seed: int, stream: int, idx: int) -> int:
    return int(_L().or_rng_u64(seed, stream, idx))


def splitmix64_nth(state: int, n: int) -> int:
    return int(_L().or_splitmix64_nth(state, n))


def flat_tail(S, mode: str = "fixed", param: float = 64):
    """(r[K] int32, lam[K]) for the flat-tail approximation of spectra S[K,P]."""
    S = _f64(S)
    K = S.shape[0]
    r = np.zeros(K, np.int32)
    lam = np.zeros(K)
    rc = _L().or_flat_tail(K, _p(S), 0 if mode == "fixed" else 1, float(param), _p(r), _p(lam))
    if rc:
        raise ValueError("bad flat-tail parameter")
    return r, lam


def sample(H: int, W: int, kind: int = FULL, param: float = 0.0, seed: int = 0, t: int = 0):
    out = np.zeros(H * W, np.int32)
    L = _L()
    if kind == FULL:
        n = L.or_sample_full(H, W, _p(out))
    elif kind == FRACTION:
        n = L.or_sample_fraction(H, W, float(param), seed, t, _p(out))
    elif kind == JITTER:
        n = L.or_sample_jitter(H, W, int(param), seed, t, _p(out))
    elif kind == REGULAR:
        n = L.or_sample_regular(H, W, int(param), _p(out))
    elif kind == VALID:
        n = L.or_sample_valid(H, W, _p(out))
    else:
        raise ValueError("unknown sampler kind")
    if n < 0:
        raise ValueError("sampler failed")
    return out[:n].copy()


class Model:
    """Eigen-form GMM plus its flat-tail truncation (oracle side)."""

    def __init__(self, w, U, S, mode: str = "fixed", param: float = 64):
        self.w, self.U, self.S = _f64(w), _f64(U), _f64(S)
        self.K = self.w.shape[0]
        self.r, self.lam = flat_tail(self.S, mode, param)

    def _args(self):
        return (self.K, _p(self.w), _p(self.U), _p(self.S), _p(self.r), _p(self.lam))


def scores(m: Model, beta: float, x, anchors):
    x = _f64(x)
    H, W = x.shape
    a = _i32(anchors)
    out = np.zeros((a.shape[0], m.K))
    _L().or_scores(*m._args(), float(beta), _p(x), H, W, _p(a), a.shape[0], _p(out))
    return out


def patch_step(m: Model, beta: float, x, anchors=None, forced_k=None):
    """(xtilde, kstar, gap, best) of Algorithm 1's first four steps."""
    x = _f64(x)
    H, W = x.shape
    a = _i32(np.arange(H * W) if anchors is None else anchors)
    n = a.shape[0]
    fk = None if forced_k is None else _i32(forced_k)
    xt = np.zeros((H, W))
    ks = np.zeros(n, np.int32)
    gap = np.zeros(n)
    best = np.zeros(n)
    rc = _L().or_patch_step(*m._args(), float(beta), _p(x), H, W, _p(a), n, _p(fk),
                            _p(xt), _p(ks), _p(gap), _p(best))
    if rc:
        raise MemoryError("oracle patch step")
    return xt, ks, gap, best


def dft2(x):
    x = _f64(x)
    H, W = x.shape
    re = np.zeros((H, W))
    im = np.zeros((H, W))
    _L().or_dft2_real(_p(x), H, W, _p(re), _p(im))
    return re + 1j * im


def lam(kind: int, H: int, W: int, sigma: float, a=None, kernel=None):
    a = None if a is None else _f64(a)
    k = None if kernel is None else _f64(kernel)
    kh, kw = (0, 0) if k is None else k.shape
    return float(_L().or_lambda(kind, _p(a), _p(k), kh, kw, H, W, float(sigma)))


def xupdate_pixelwise(y, xtilde, bs: float, a=None):
    y, xt = _f64(y), _f64(xtilde)
    a = None if a is None else _f64(a)
    out = np.zeros_like(y)
    _L().or_xupdate_pixelwise(_p(a), _p(y), _p(xt), y.size, float(bs), _p(out))
    return out


def xupdate_conv(kernel, y, xtilde, bs: float):
    k, y, xt = _f64(kernel), _f64(y), _f64(xtilde)
    H, W = y.shape
    out = np.zeros_like(y)
    _L().or_xupdate_conv(_p(k), k.shape[0], k.shape[1], _p(y), _p(xt), H, W, float(bs), _p(out))
    return out


def init_conv(kernel, y, c: float):
    k, y = _f64(kernel), _f64(y)
    H, W = y.shape
    out = np.zeros_like(y)
    _L().or_init_conv(_p(k), k.shape[0], k.shape[1], _p(y), H, W, float(c), _p(out))
    return out


def init_cg(a, y, c: float, iters: int):
    a, y = _f64(a), _f64(y)
    H, W = y.shape
    out = np.zeros_like(y)
    _L().or_init_cg(_p(a), _p(y), H, W, float(c), int(iters), _p(out))
    return out


def valid_weights(H: int, W: int):
    """Per-pixel count of the patches lying inside the image, divided by P."""
    out = np.zeros((H, W))
    _L().or_valid_weights(H, W, _p(out))
    return out


def xupdate_weighted(deg: int, y, xtilde, wgt, bs: float, a=None, kernel=None, iters: int = 100):
    """Image update of Eq. 6 with the per-pixel overlap weights wgt."""
    y, xt, w = _f64(y), _f64(xtilde), _f64(wgt)
    H, W = y.shape
    a = None if a is None else _f64(a)
    k = None if kernel is None else _f64(kernel)
    kh, kw = (0, 0) if k is None else k.shape
    out = np.zeros_like(y)
    _L().or_xupdate_weighted(deg, _p(a), _p(k), kh, kw, _p(y), _p(xt), _p(w), H, W, float(bs), int(iters),
                             _p(out))
    return out


def sr_apply(kernel, x, d: int):
    """A x = decimation by d (keep pixel (d i, d j)) of the periodic blur of x."""
    k, x = _f64(kernel), _f64(x)
    H, W = x.shape
    out = np.zeros((H // d, W // d))
    _L().or_sr_apply(_p(k), k.shape[0], k.shape[1], _p(x), H, W, int(d), _p(out))
    return out


def sr_adjoint(kernel, ylow, d: int):
    """A^T y: zero insertion to (d h) x (d w), then correlation with the kernel."""
    k, y = _f64(kernel), _f64(ylow)
    H, W = y.shape[0] * d, y.shape[1] * d
    out = np.zeros((H, W))
    _L().or_sr_adjoint(_p(k), k.shape[0], k.shape[1], _p(y), H, W, int(d), _p(out))
    return out


def lam_sr(kernel, H: int, W: int, d: int, sigma: float) -> float:
    k = _f64(kernel)
    return float(_L().or_lambda_sr(_p(k), k.shape[0], k.shape[1], H, W, int(d), float(sigma)))


def xupdate_sr(kernel, ylow, xtilde, d: int, bs: float):
    k, y, xt = _f64(kernel), _f64(ylow), _f64(xtilde)
    H, W = xt.shape
    out = np.zeros_like(xt)
    _L().or_xupdate_sr(_p(k), k.shape[0], k.shape[1], _p(y), _p(xt), H, W, int(d), float(bs), _p(out))
    return out


def init_sr(kernel, ylow, d: int, c: float):
    k, y = _f64(kernel), _f64(ylow)
    H, W = y.shape[0] * d, y.shape[1] * d
    out = np.zeros((H, W))
    _L().or_init_sr(_p(k), k.shape[0], k.shape[1], _p(y), H, W, int(d), float(c), _p(out))
    return out


def restore(m: Model, y, sigma: float, beta_mult=(1, 4, 8, 16, 32), deg: int = DENOISE,
            a=None, kernel=None, subset: int = FULL, subset_param: float = 0.0,
            seed: int = 0, cg_iters: int = 100, record: bool = False, factor: int = 1):
    """Full restoration.  With record=True also returns per-iteration
    (kstar list, gap list) in sampling order.  deg=SR: y is the
    (H/factor) x (W/factor) observation and the result is H x W."""
    y = _f64(y)
    H, W = y.shape
    if deg == SR:
        H, W = H * factor, W * factor
    a = None if a is None else _f64(a)
    k = None if kernel is None else _f64(kernel)
    kh, kw = (0, 0) if k is None else k.shape
    bm = _f64(beta_mult)
    T = bm.shape[0]
    x = np.zeros((H, W))
    ks = np.zeros((T, H * W), np.int32) if record else None
    gp = np.zeros((T, H * W)) if record else None
    ns = np.zeros(T, np.int32)
    rc = _L().or_restore(*m._args(), _p(y), H, W, deg, _p(a), _p(k), kh, kw, int(factor), float(sigma),
                         _p(bm), T, subset, float(subset_param), seed, cg_iters, _p(x),
                         _p(ks), _p(gp), _p(ns))
    if rc:
        raise RuntimeError("oracle restore failed")
    if record:
        return x, [ks[t, :ns[t]] for t in range(T)], [gp[t, :ns[t]] for t in range(T)]
    return x
