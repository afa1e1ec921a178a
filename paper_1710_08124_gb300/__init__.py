"""Python binding of libepll (argument marshalling only).

Every computation happens in the CUDA library built from ``csrc/`` (see
``include/epll.h`` for the C ABI).  PyTorch supplies device memory and
streams; numpy arrays are accepted for the host-buffer entry point.  The
binding raises if the library is missing -- there is no CPU fallback.

Names mirror the C ABI without the ``epll_`` prefix: ``gmm_load``,
``restore``, ``restore_host``, ``patch_step``, ``sample``, ``last_counters``.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libepll.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED = 0, -1, -2, -3, -4, -5
RANK_FIXED, RANK_RHO = 0, 1
DENOISE, PIXELWISE, CONV_PERIODIC, CONV_DECIMATE = 0, 1, 2, 3
SUBSET_ALL, SUBSET_FRACTION, SUBSET_JITTER, SUBSET_REGULAR, SUBSET_VALID = 0, 1, 2, 3, 4
FP32, BF16, FP16, BF16X3, FP8, AUTO = 0, 1, 2, 3, 4, 5
SELECT_EXHAUSTIVE, SELECT_PROPOSAL, SELECT_TREE = 0, 1, 2
PAPER_BETA = (1.0, 4.0, 8.0, 16.0, 32.0)


class EpllError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"epll status {status}: {msg}")
        self.status = status


class _Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("tie_gap", C.c_float), ("subset", C.c_int),
                ("subset_param", C.c_double), ("seed", C.c_uint64), ("cg_iters", C.c_int),
                ("select", C.c_int)]


class _Job(C.Structure):
    _fields_ = [("y", C.c_void_p), ("x_out", C.c_void_p), ("a", C.c_void_p), ("H", C.c_int),
                ("W", C.c_int), ("kind", C.c_int), ("sigma", C.c_float), ("kernel", C.c_void_p),
                ("kh", C.c_int), ("kw", C.c_int)]


BATCH_SEQUENTIAL, BATCH_GRAPH = 0, 1


class _Degradation(C.Structure):
    _fields_ = [("kind", C.c_int), ("a", C.c_void_p), ("kernel", C.c_void_p),
                ("kh", C.c_int), ("kw", C.c_int), ("factor", C.c_int)]


@dataclass
class Options:
    """Mirror of ``epll_options``."""
    precision: int = FP32
    tie_gap: float = -1.0
    subset: int = SUBSET_ALL
    subset_param: float = 0.0
    seed: int = 0
    cg_iters: int = 100
    select: int = SELECT_EXHAUSTIVE

    def _c(self) -> _Options:
        return _Options(self.precision, self.tie_gap, self.subset, self.subset_param,
                        self.seed, self.cg_iters, self.select)


_lib = None


def build(force: bool = False) -> str:
    from . import buildlib as _b
    return _b.build(force=force)


def lib():
    """The loaded libepll (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libepll is not built ({LIB_PATH} missing); run build()")
        L = C.CDLL(LIB_PATH)
        i, d, vp = C.c_int, C.c_double, C.c_void_p
        L.epll_last_error.restype = C.c_char_p
        L.epll_gmm_load.argtypes = [i, i, vp, vp, vp, i, d, C.POINTER(vp)]
        L.epll_gmm_free.argtypes = [vp]
        L.epll_gmm_free.restype = None
        L.epll_gmm_ranks.argtypes = [vp, vp, vp]
        L.epll_restore.argtypes = [vp, vp, i, i, C.POINTER(_Degradation), C.c_float, vp, i,
                                   C.POINTER(_Options), vp, vp]
        L.epll_restore_host.argtypes = L.epll_restore.argtypes
        L.epll_image_update.argtypes = [vp, vp, vp, i, i, C.POINTER(_Degradation), C.c_float, d, vp, vp]
        L.epll_patch_step.argtypes = [vp, vp, i, i, d, C.POINTER(_Options), i, vp, vp, vp, vp,
                                      vp, C.POINTER(C.c_int), vp]
        L.epll_sample.argtypes = [i, i, C.POINTER(_Options), i, vp, C.POINTER(C.c_int), vp]
        L.epll_sample_noalloc.argtypes = L.epll_sample.argtypes
        L.epll_restore_batch.argtypes = [vp, i, C.POINTER(_Job), vp, i, C.POINTER(_Options), i, i, vp]
        L.epll_set_tiles.argtypes = [vp, i, i]
        L.epll_set_cta_pairs.argtypes = [vp, i]
        L.epll_batch_config.argtypes = [vp, vp, vp, vp]
        L.epll_last_counters.argtypes = [vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                         C.POINTER(C.c_longlong)]
        L.epll_profile_enable.argtypes = [vp, i]
        L.epll_profile_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong),
                                        C.POINTER(C.c_double)]
        L.epll_options_default.argtypes = [C.POINTER(_Options)]
        L.epll_options_default.restype = None
        L.epll_proposal_size.argtypes = [i]
        L.epll_proposal_size.restype = C.c_size_t
        L.epll_proposal_create.argtypes = [i, C.c_uint64, C.POINTER(vp)]
        L.epll_proposal_free.argtypes = [vp]
        L.epll_proposal_free.restype = None
        L.epll_proposal_get.argtypes = [vp, vp]
        L.epll_proposal_set.argtypes = [vp, vp]
        L.epll_proposal_grad.argtypes = [vp, vp, i, i, i, vp, vp, vp, vp, vp, i, i, vp, vp, vp]
        L.epll_proposal_train.argtypes = [vp, vp, i, i, i, vp, vp, vp, vp, vp, i, i, C.c_float, C.c_float,
                                          vp, vp]
        L.epll_gmm_attach_proposal.argtypes = [vp, vp, i, C.c_float]
        L.epll_proposal_topm.argtypes = [vp, vp, i, i, vp, i, d, vp, vp, vp]
        L.epll_last_fallbacks.argtypes = [vp, C.POINTER(C.c_longlong)]
        L.epll_gmm_attach_tree.argtypes = [vp, i, vp, vp, vp, vp, vp]
        _lib = L
    return _lib


def last_error() -> str:
    return lib().epll_last_error().decode()


def _check(status: int):
    if status != OK:
        raise EpllError(status, last_error())


def _dptr(t, dtype=None):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected dtype {dtype}, got {t.dtype}")
    return t.data_ptr()


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


class GMM:
    """A loaded GMM patch prior (``epll_gmm_load``)."""

    def __init__(self, w, U, S, rank_mode: int = RANK_FIXED, rank_param: float = 64):
        self.w = np.ascontiguousarray(w, np.float64)
        self.U = np.ascontiguousarray(U, np.float64)
        self.S = np.ascontiguousarray(S, np.float64)
        self.K = int(self.w.shape[0])
        h = C.c_void_p()
        _check(lib().epll_gmm_load(self.K, int(self.U.shape[1]), self.w.ctypes.data,
                                   self.U.ctypes.data, self.S.ctypes.data, int(rank_mode),
                                   float(rank_param), C.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def ranks(self):
        r = np.zeros(self.K, np.int32)
        lam = np.zeros(self.K)
        _check(lib().epll_gmm_ranks(self._h, r.ctypes.data, lam.ctypes.data))
        return r, lam

    def free(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().epll_gmm_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def gmm_load(w, U, S, rank_mode: int = RANK_FIXED, rank_param: float = 64) -> GMM:
    return GMM(w, U, S, rank_mode, rank_param)


def _degradation(kind, a_ptr, kernel, factor: int = 1):
    if kernel is not None:
        k = np.ascontiguousarray(kernel, np.float32)
        deg = _Degradation(kind, a_ptr, k.ctypes.data, k.shape[0], k.shape[1], int(factor))
        return deg, k
    return _Degradation(kind, a_ptr, None, 0, 0, int(factor)), None


def restore(g: GMM, y, sigma: float, beta_mult=PAPER_BETA, kind: int = DENOISE, a=None,
            kernel=None, options: Options | None = None, out=None, stream=None, factor: int = 1):
    """Device-buffer restoration; y (and a) are float32 CUDA tensors [H, W]
    (kind=CONV_DECIMATE: y is [H/factor, W/factor] and the result [H, W])."""
    import torch
    H, W = y.shape
    if kind == CONV_DECIMATE:
        H, W = H * factor, W * factor
    out = torch.empty((H, W), dtype=torch.float32, device=y.device) if out is None else out
    deg, keep = _degradation(kind, _dptr(a, torch.float32), kernel, factor)
    bm = np.ascontiguousarray(beta_mult, np.float64)
    opt = (options or Options())._c()
    _check(lib().epll_restore(g.handle, _dptr(y, torch.float32), H, W, C.byref(deg), float(sigma),
                              bm.ctypes.data, bm.shape[0], C.byref(opt), _dptr(out, torch.float32),
                              _stream(stream)))
    del keep
    return out


def image_update(g: GMM, y, xtilde, sigma: float, beta_mult: float, kind: int = DENOISE, a=None,
                 kernel=None, out=None, stream=None, factor: int = 1):
    """The image estimation step alone (``epll_image_update``); float32 CUDA tensors."""
    import torch
    H, W = xtilde.shape
    out = torch.empty_like(xtilde) if out is None else out
    deg, keep = _degradation(kind, _dptr(a, torch.float32), kernel, factor)
    _check(lib().epll_image_update(g.handle, _dptr(y, torch.float32), _dptr(xtilde, torch.float32), H, W,
                                   C.byref(deg), float(sigma), float(beta_mult), _dptr(out, torch.float32),
                                   _stream(stream)))
    del keep
    return out


def restore_batch(g: GMM, jobs, beta_mult=PAPER_BETA, options: Options | None = None,
                  mode: int = BATCH_GRAPH, lanes: int = 0, stream=None):
    """Batched restoration (``epll_restore_batch``).  ``jobs`` is a list of
    (y, x_out, a_or_None, kind, sigma) or (y, x_out, a_or_None, kind, sigma,
    kernel) with float32 CUDA tensors (kernel: a host array for
    CONV_PERIODIC jobs)."""
    import torch
    arr = (_Job * len(jobs))()
    keep = []
    for i, job in enumerate(jobs):
        y, xo, a, kind, sigma = job[:5]
        kern = job[5] if len(job) > 5 else None
        H, W = y.shape
        kp, kh, kw = None, 0, 0
        if kern is not None:
            k = np.ascontiguousarray(kern, np.float32)
            keep.append(k)
            kp, kh, kw = k.ctypes.data, k.shape[0], k.shape[1]
        arr[i] = _Job(_dptr(y, torch.float32), _dptr(xo, torch.float32), _dptr(a, torch.float32), H, W,
                      int(kind), float(sigma), kp, kh, kw)
    bm = np.ascontiguousarray(beta_mult, np.float64)
    opt = (options or Options())._c()
    _check(lib().epll_restore_batch(g.handle, len(jobs), arr, bm.ctypes.data, bm.shape[0], C.byref(opt),
                                    int(mode), int(lanes), _stream(stream)))
    del keep


def set_tiles(g: GMM, tile_bn: int = 256, tile_agg: int = 1):
    """Tile shapes of the handle's selection and reprojection kernels (``epll_set_tiles``)."""
    _check(lib().epll_set_tiles(g.handle, int(tile_bn), int(tile_agg)))


def set_cta_pairs(g: GMM, enable: bool = True):
    """Selection's first pass in clusters of two CTAs sharing each tensor-core
    product (``epll_set_cta_pairs``)."""
    _check(lib().epll_set_cta_pairs(g.handle, int(bool(enable))))


def batch_config(g: GMM):
    """(lanes, tile_bn, tile_agg) the batch autotuner chose (``epll_batch_config``)."""
    l, b, a = C.c_int(0), C.c_int(0), C.c_int(0)
    _check(lib().epll_batch_config(g.handle, C.byref(l), C.byref(b), C.byref(a)))
    return l.value, b.value, a.value


def restore_host(g: GMM, y: np.ndarray, sigma: float, beta_mult=PAPER_BETA, kind: int = DENOISE,
                 a=None, kernel=None, options: Options | None = None, out=None, stream=None, factor: int = 1):
    """Host-buffer restoration (copies inside the call); y, a, out are float32 arrays
    (pinned torch CPU tensors are accepted too)."""
    def hptr(v):
        if v is None:
            return None
        if isinstance(v, np.ndarray):
            if v.dtype != np.float32 or not v.flags.c_contiguous:
                raise ValueError("host arrays must be C-contiguous float32")
            return v.ctypes.data
        return v.data_ptr()

    H, W = y.shape
    if kind == CONV_DECIMATE:
        H, W = H * factor, W * factor
    if out is None:
        out = np.empty((H, W), np.float32)
    deg, keep = _degradation(kind, hptr(a), kernel, factor)
    bm = np.ascontiguousarray(beta_mult, np.float64)
    opt = (options or Options())._c()
    _check(lib().epll_restore_host(g.handle, hptr(y), H, W, C.byref(deg), float(sigma),
                                   bm.ctypes.data, bm.shape[0], C.byref(opt), hptr(out),
                                   _stream(stream)))
    del keep
    return out


def patch_step(g: GMM, xhat, beta: float, options: Options | None = None, t: int = 0,
               forced_k=None, stream=None):
    """One patch step; returns (xtilde, anchors, kstar, gap) as CUDA tensors."""
    import torch
    H, W = xhat.shape
    dev = xhat.device
    xt = torch.empty_like(xhat)
    an = torch.empty(H * W, dtype=torch.int32, device=dev)
    ks = torch.empty(H * W, dtype=torch.int32, device=dev)
    gp = torch.empty(H * W, dtype=torch.float32, device=dev)
    n = C.c_int(0)
    opt = (options or Options())._c()
    _check(lib().epll_patch_step(g.handle, _dptr(xhat, torch.float32), H, W, float(beta),
                                 C.byref(opt), int(t), _dptr(xt), _dptr(an), _dptr(ks), _dptr(gp),
                                 _dptr(forced_k, torch.int32), C.byref(n), _stream(stream)))
    m = n.value
    return xt, an[:m], ks[:m], gp[:m]


def sample(H: int, W: int, options: Options | None = None, t: int = 0, device="cuda", stream=None):
    import torch
    an = torch.empty(H * W, dtype=torch.int32, device=device)
    n = C.c_int(0)
    opt = (options or Options())._c()
    _check(lib().epll_sample(H, W, C.byref(opt), int(t), _dptr(an), C.byref(n), _stream(stream)))
    return an[:n.value]


def sample_noalloc(H: int, W: int, options: Options | None = None, t: int = 0, out=None, stream=None):
    """Patch sampling that allocates no device memory inside the library
    (``epll_sample_noalloc``); ``out`` is a caller-provided int32 CUDA tensor of
    at least H*W entries.  Returns the filled prefix of ``out``."""
    import torch
    if out is None:
        an = torch.empty(H * W, dtype=torch.int32, device="cuda")
    else:
        an = out
        if an.device.type != "cuda" or an.device.index != torch.cuda.current_device():
            raise ValueError("out must be on the current CUDA device (the static scratch is per device)")
        if not an.is_contiguous() or an.numel() < H * W:
            raise ValueError(f"out must be a contiguous int32 tensor of at least H*W = {H * W} entries")
    n = C.c_int(0)
    opt = (options or Options())._c()
    _check(lib().epll_sample_noalloc(H, W, C.byref(opt), int(t), _dptr(an, torch.int32), C.byref(n),
                                     _stream(stream)))
    return an[:n.value]


def last_counters(g: GMM):
    """(patch evaluations, near-tie rescored patches, kernel launches) of the last call."""
    a, b, c = C.c_longlong(), C.c_longlong(), C.c_longlong()
    _check(lib().epll_last_counters(g.handle, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def last_fallbacks(g: GMM) -> int:
    """Patches the last proposal-selection call sent to the exhaustive pass."""
    v = C.c_longlong()
    _check(lib().epll_last_fallbacks(g.handle, C.byref(v)))
    return v.value


def profile_enable(g: GMM, enable: bool = True):
    _check(lib().epll_profile_enable(g.handle, int(enable)))


def profile_read(g: GMM):
    """(selection-kernel device ms, launches, algorithmic FLOPs) since the last read."""
    ms, n, fl = C.c_double(), C.c_longlong(), C.c_double()
    _check(lib().epll_profile_read(g.handle, C.byref(ms), C.byref(n), C.byref(fl)))
    return ms.value, n.value, fl.value


class Proposal:
    """Learned top-m proposal network (``epll_proposal_*``): 64 -> 256 -> 256 -> K."""

    def __init__(self, K: int, seed: int = 0):
        h = C.c_void_p()
        _check(lib().epll_proposal_create(int(K), int(seed), C.byref(h)))
        self._h = h
        self.K = int(K)
        self.size = int(lib().epll_proposal_size(self.K))

    @property
    def handle(self):
        return self._h

    def get(self) -> np.ndarray:
        out = np.empty(self.size, np.float32)
        _check(lib().epll_proposal_get(self._h, out.ctypes.data))
        return out

    def set(self, params):
        v = np.ascontiguousarray(params, np.float32)
        if v.shape != (self.size,):
            raise ValueError(f"expected {self.size} parameters")
        _check(lib().epll_proposal_set(self._h, v.ctypes.data))

    @staticmethod
    def _batch(images, img_idx, anchors, log_ib, labels, sel):
        import torch
        if images.dim() == 2:
            images = images[None]
        n_img, H, W = images.shape
        n_all = int(labels.numel())
        B = n_all if sel is None else int(sel.numel())
        return (_dptr(images, torch.float32), n_img, H, W, _dptr(img_idx, torch.int32),
                _dptr(anchors, torch.int32), _dptr(log_ib, torch.float32), _dptr(labels, torch.int32),
                _dptr(sel, torch.int32), n_all, B)

    def grad(self, images, img_idx, anchors, log_ib, labels, sel=None, stream=None):
        """(gradient as a CUDA float32 tensor, mean cross-entropy) of one batch."""
        import torch
        g = torch.empty(self.size, dtype=torch.float32, device=images.device)
        loss = C.c_float(0.0)
        _check(lib().epll_proposal_grad(self._h, *self._batch(images, img_idx, anchors, log_ib, labels, sel),
                                        _dptr(g), C.byref(loss), _stream(stream)))
        return g, loss.value

    def train_step(self, images, img_idx, anchors, log_ib, labels, sel=None, lr: float = 1e-3,
                   weight_decay: float = 0.0, want_loss: bool = True, stream=None):
        """One AdamW step on the samples ``sel`` (None: all); returns the batch
        loss (before the step) when want_loss."""
        loss = C.c_float(0.0)
        _check(lib().epll_proposal_train(self._h, *self._batch(images, img_idx, anchors, log_ib, labels, sel),
                                         float(lr), float(weight_decay),
                                         C.byref(loss) if want_loss else None, _stream(stream)))
        return loss.value if want_loss else None

    def free(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().epll_proposal_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def attach_proposal(g: GMM, p: Proposal | None, topm: int = 4, pmin: float = 0.0):
    """Attaches (or, with None, detaches) a proposal network to a model."""
    _check(lib().epll_gmm_attach_proposal(g.handle, p.handle if p is not None else None, int(topm),
                                          float(pmin)))
    g._proposal = p
    g._topm = int(topm)


def proposal_topm(g: GMM, xhat, beta: float, anchors=None, stream=None):
    """Runs the attached network: (cand int32 [n][topm], pmass float32 [n]) as CUDA tensors."""
    import torch
    H, W = xhat.shape
    n = H * W if anchors is None else int(anchors.numel())
    topm = g._topm
    cand = torch.empty((n, topm), dtype=torch.int32, device=xhat.device)
    pmass = torch.empty(n, dtype=torch.float32, device=xhat.device)
    _check(lib().epll_proposal_topm(g.handle, _dptr(xhat, torch.float32), H, W, _dptr(anchors, torch.int32), n,
                                    float(beta), _dptr(cand), _dptr(pmass), _stream(stream)))
    return cand, pmass


def attach_tree(g: GMM, tree):
    """Attaches a search tree (``tree.build_tree``'s result) to a model, or
    detaches it with None."""
    if tree is None:
        _check(lib().epll_gmm_attach_tree(g.handle, 0, None, None, None, None, None))
        g._tree = None
        return
    w = np.ascontiguousarray(tree.weights, np.float64)
    U = np.ascontiguousarray(tree.eigvecs, np.float64)
    S = np.ascontiguousarray(tree.eigvals, np.float64)
    cb = np.ascontiguousarray(tree.child_begin, np.int32)
    lf = np.ascontiguousarray(tree.leaf_component, np.int32)
    _check(lib().epll_gmm_attach_tree(g.handle, int(w.shape[0]), w.ctypes.data, U.ctypes.data, S.ctypes.data,
                                      cb.ctypes.data, lf.ctypes.data))
    g._tree = tree
