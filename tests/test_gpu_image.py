"""Image-domain steps of the CUDA path against the FP64 oracle, through the
C ABI: the initialisation of the inverse problems (Sec. "Parameter settings":
x0 = (A^T A + c L)^-1 A^T y, c = 0.2 sigma^2 / lambda; an FFT solve for a
periodic blur, conjugate gradients for a pixelwise A) and the image
estimation step alone (last step of Algorithm 1, Eq. 6), for periodic
deblurring, pixelwise operators and super-resolution (blur then decimation,
solved per aliasing block of frequencies).

Every bound here is derived from the conditioning of the step and FP32
arithmetic (unit roundoff u = 2^-24), not chosen:

* conjugate gradients: the forward error of a linear solve whose backward
  error is of the order of u is at most kappa_2(A) u |x|_inf (kappa from the
  extreme eigenvalues of the system matrix); for a converged run the backward
  error itself, |b - A x|_inf / (|A|_inf |x|_inf + |b|_inf), is at most 16 u
  (5 products per stencil row plus the recurrence's drift);
* FFT solves x = F^-1 G F v: each FP32 transform is within ceil(log2 N) u of
  its exact result (Higham, Accuracy and Stability of Numerical Algorithms,
  Sec. 24.1), amplified by the operator norm max |G| of the diagonal
  multiplier; the bound is that sum over the inputs;
* the pixelwise update is a handful of FP32 operations per pixel: 8 u |x|;
* super-resolution: the same FFT rounding at both resolutions, amplified by
  the gain of the per-block solve (computed in FP64 from numpy's transform).
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)
sp = pytest.importorskip("scipy.sparse")
sla = pytest.importorskip("scipy.sparse.linalg")

import paper_1710_08124_gb300 as ep  # noqa: E402

U = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _built():
    ep.build()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")


def model(K=12, r=8):
    g = synth.synthetic_gmm(K)
    return ep.gmm_load(g.w, g.U, g.S, ep.RANK_FIXED, r)


def pixelwise_matrix(a, c):
    """diag(a^2) + c L, L the periodic 5-point negative Laplacian (sparse)."""
    H, W = a.shape
    N = H * W
    idx = np.arange(N).reshape(H, W)
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [(a * a).ravel() + 4 * c]
    for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
        nb = np.roll(np.roll(idx, -di, 0), -dj, 1)
        rows.append(idx.ravel())
        cols.append(nb.ravel())
        vals.append(np.full(N, -c))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))


def otf(kernel, H, W):
    """Transfer function of the periodic blur (centre (kh/2, kw/2) at (0, 0))."""
    kh, kw = kernel.shape
    h = np.zeros((H, W))
    for u in range(kh):
        for v in range(kw):
            h[(u - kh // 2) % H, (v - kw // 2) % W] += kernel[u, v]
    return np.fft.fft2(h)


def laplacian_symbol(H, W):
    u = np.arange(H)[:, None]
    v = np.arange(W)[None, :]
    return 4 - 2 * np.cos(2 * np.pi * u / H) - 2 * np.cos(2 * np.pi * v / W)


# ---------------------------------------------------------------- initialisation
@pytest.mark.parametrize("H,W,sigma,i,iters", [
    (40, 48, 10 / 255, 7, 100),    # the restoration test's problem, converged
    (97, 131, 10 / 255, 3, 100),   # ragged split over the cluster's CTAs
    (128, 128, 25 / 255, 5, 100),
    (97, 131, 10 / 255, 3, 7),     # far from converged: the iteration itself is compared
    (40, 48, 10 / 255, 7, 1),
    (40, 48, 10 / 255, 7, 0),      # x0 = a y
])
def test_init_cg(H, W, sigma, i, iters):
    x, a, y = synth.inpaint_problem(i, H, sigma, W=W)
    y32 = y.astype(np.float32).astype(np.float64)
    lam = oracle.lam(oracle.PIXELWISE, H, W, sigma, a=a)
    c = 0.2 * sigma ** 2 / lam
    xo = oracle.init_cg(a, y32, c, iters)
    gm = model()
    xg = ep.restore(gm, dev(y), sigma, beta_mult=(), kind=ep.PIXELWISE, a=dev(a),
                    options=ep.Options(cg_iters=iters)).cpu().numpy().astype(np.float64)
    A = pixelwise_matrix(a, c)
    lmin = sla.eigsh(A, k=1, sigma=0, which="LM", return_eigenvectors=False)[0]
    lmax = sla.eigsh(A, k=1, which="LA", return_eigenvectors=False)[0]
    kappa = lmax / lmin
    err = np.abs(xg - xo).max()
    assert err <= kappa * U * np.abs(xo).max(), (err, kappa)
    if iters == 100:
        b = (a * y32).ravel()
        xs = sla.spsolve(A.tocsc(), b)
        assert np.abs(xo.ravel() - xs).max() <= 1e-12  # the oracle has converged
        rho = np.abs(b - A @ xg.ravel()).max()
        a_inf = abs(A).sum(axis=1).max()
        assert rho <= 16 * U * (a_inf * np.abs(xg).max() + np.abs(b).max()), rho


@pytest.mark.parametrize("H,W,sigma,i", [(48, 40, 2 / 255, 6), (61, 77, 5 / 255, 3), (128, 128, 2 / 255, 2)])
def test_init_fft(H, W, sigma, i):
    x, k, y = synth.deblur_problem(i, H, sigma, W=W)
    k64 = k.astype(np.float32).astype(np.float64)
    y32 = y.astype(np.float32).astype(np.float64)
    lam = oracle.lam(oracle.CONV, H, W, sigma, kernel=k64)
    c = 0.2 * sigma ** 2 / lam
    xo = oracle.init_conv(k64, y32, c)
    gm = model()
    xg = ep.restore(gm, dev(y), sigma, beta_mult=(), kind=ep.CONV_PERIODIC, kernel=k).cpu().numpy()
    Hh = otf(k64, H, W)
    G = np.abs(Hh) / (np.abs(Hh) ** 2 + c * laplacian_symbol(H, W))
    bound = G.max() * math.ceil(math.log2(H * W)) * U * np.abs(y32).max()
    err = np.abs(xg - xo).max()
    assert err <= bound, (err, bound)


# ---------------------------------------------------------------- image estimation step
@pytest.mark.parametrize("mult", [1.0, 8.0, 32.0])
def test_image_update_fft(mult):
    H, W, sigma = 48, 40, 2 / 255
    x, k, y = synth.deblur_problem(6, H, sigma, W=W)
    k64 = k.astype(np.float32).astype(np.float64)
    y32 = y.astype(np.float32).astype(np.float64)
    xt = (x + 0.02 * np.random.default_rng(1).standard_normal(x.shape)).astype(np.float32)
    lam = oracle.lam(oracle.CONV, H, W, sigma, kernel=k64)
    bs = lam * mult
    xo = oracle.xupdate_conv(k64, y32, xt.astype(np.float64), bs)
    gm = model()
    xg = ep.image_update(gm, dev(y), dev(xt), sigma, mult, kind=ep.CONV_PERIODIC, kernel=k).cpu().numpy()
    Hh = np.abs(otf(k64, H, W))
    gy = (Hh / (Hh ** 2 + bs)).max()
    gx = (bs / (Hh ** 2 + bs)).max()
    bound = math.ceil(math.log2(H * W)) * U * (gy * np.abs(y32).max() + gx * np.abs(xt).max())
    err = np.abs(xg - xo).max()
    assert err <= bound, (err, bound)


@pytest.mark.parametrize("kind", ["denoise", "mask", "vignette"])
def test_image_update_pixelwise(kind):
    H, W, sigma = 37, 53, 15 / 255
    x, y = synth.denoise_problem(2, H, sigma, W=W)
    rng = np.random.default_rng(3)
    xt = (x + 0.01 * rng.standard_normal(x.shape)).astype(np.float32)
    if kind == "denoise":
        a = None
        deg = oracle.DENOISE
    elif kind == "mask":
        a = synth.observed_mask(2, H, W, 0.7)
        deg = oracle.PIXELWISE
    else:
        a = (0.3 + 0.7 * rng.random((H, W))).astype(np.float32)
        deg = oracle.PIXELWISE
    y32 = y.astype(np.float32).astype(np.float64)
    a64 = None if a is None else a.astype(np.float32).astype(np.float64)
    if a64 is not None:
        y32 = a64 * y32
    lam = oracle.lam(deg, H, W, sigma, a=a64)
    xo = oracle.xupdate_pixelwise(y32, xt.astype(np.float64), lam * 4.0, a=a64)
    gm = model()
    xg = ep.image_update(gm, dev(y32), dev(xt), sigma, 4.0, kind=ep.DENOISE if a is None else ep.PIXELWISE,
                         a=None if a is None else dev(a)).cpu().numpy()
    err = np.abs(xg - xo).max()
    assert err <= 8 * U * max(np.abs(xo).max(), 1.0), err


# ---------------------------------------------------------------- super-resolution
def sr_problem(i, H, W, d, sigma, ks=9, sb=1.0):
    x = synth.image(i, H, W)
    k = synth.gaussian_kernel(ks, sb)
    yl = synth.blur_periodic(x, k)[::d, ::d] + synth.noise(i, H // d, W // d, sigma)
    return x, k, yl.astype(np.float32)


def sr_blocks(k, H, W, d):
    """Transfer function at the d^2 aliases of every low-resolution frequency:
    array [d^2, H/d, W/d] (numpy FP64 FFT, independent of both paths)."""
    Hh = otf(k, H, W)
    h, w = H // d, W // d
    return np.stack([Hh[a * h:(a + 1) * h, b * w:(b + 1) * w] for a in range(d) for b in range(d)])


@pytest.mark.parametrize("H,W,d,sigma", [(48, 48, 3, 2 / 255), (48, 36, 2, 5 / 255), (40, 40, 1, 2 / 255)])
def test_init_sr(H, W, d, sigma):
    """Initialisation of super-resolution (one solve per aliasing block
    between FP32 FFTs) against the oracle's FP64 conjugate gradients; bound:
    the FFT rounding of both transforms amplified by the block solve's gain
    Gamma / d, Gamma^2 = max over blocks of sum_k |X_k / Y|^2."""
    x, k, yl = sr_problem(3, H, W, d, sigma)
    k64 = k.astype(np.float32).astype(np.float64)
    y64 = yl.astype(np.float64)
    lam = oracle.lam_sr(k64, H, W, d, sigma)
    c = 0.2 * sigma ** 2 / lam
    xo = oracle.init_sr(k64, y64, d, c)
    gm = model()
    xg = ep.restore(gm, dev(yl), sigma, beta_mult=(), kind=ep.CONV_DECIMATE, kernel=k, factor=d).cpu().numpy()
    assert xg.shape == (H, W)
    Hb = sr_blocks(k64, H, W, d)
    h, w = H // d, W // d
    L = np.stack([laplacian_symbol(H, W)[a * h:(a + 1) * h, b * w:(b + 1) * w] for a in range(d) for b in range(d)])
    # X = (D + s g g^H)^-1 g Y per block: gain of each entry relative to Y
    s = 1.0 / d ** 2
    G = np.zeros_like(Hb, dtype=np.float64)
    for u in range(h):
        for v in range(w):
            g = np.conj(Hb[:, u, v])
            M = np.diag(c * L[:, u, v]) + s * np.outer(g, np.conj(g))
            G[:, u, v] = np.abs(np.linalg.solve(M, g))
    gamma = np.sqrt((G ** 2).sum(axis=0).max())
    bound = gamma / d * (math.ceil(math.log2(h * w)) + math.ceil(math.log2(H * W))) * U * np.abs(y64).max()
    err = np.abs(xg - xo).max()
    assert err <= bound, (err, bound)


@pytest.mark.parametrize("H,W,d", [(48, 48, 3), (48, 36, 2)])
def test_image_update_sr(H, W, d):
    sigma = 2 / 255
    x, k, yl = sr_problem(4, H, W, d, sigma)
    k64 = k.astype(np.float32).astype(np.float64)
    xt = (x + 0.02 * np.random.default_rng(5).standard_normal(x.shape)).astype(np.float32)
    lam = oracle.lam_sr(k64, H, W, d, sigma)
    mult = 4.0
    bs = lam * mult
    xo = oracle.xupdate_sr(k64, yl.astype(np.float64), xt.astype(np.float64), d, bs)
    gm = model()
    xg = ep.image_update(gm, dev(yl), dev(xt), sigma, mult, kind=ep.CONV_DECIMATE, kernel=k,
                         factor=d).cpu().numpy()
    Hb = np.abs(sr_blocks(k64, H, W, d))
    s = 1.0 / d ** 2
    ng = (Hb ** 2).sum(axis=0)
    gamma_y = np.sqrt(((Hb / (bs + s * ng)) ** 2).sum(axis=0).max())
    n_lo, n_hi = math.ceil(math.log2(H * W / d ** 2)), math.ceil(math.log2(H * W))
    bound = U * (gamma_y / d * (n_lo + n_hi) * np.abs(yl).max() + 2 * n_hi * np.abs(xt).max())
    err = np.abs(xg - xo).max()
    assert err <= bound, (err, bound)


def test_sr_factor_one_equals_deconvolution_path():
    """CONV_DECIMATE with factor 1 solves the deconvolution through the
    aliasing-block kernels and C2C transforms; it must agree with the
    CONV_PERIODIC path (R2C transforms, pointwise kernels) to FP32 rounding."""
    sigma = 2 / 255
    x, k, y = synth.deblur_problem(6, 48, sigma, W=40)
    gm = model()
    a = ep.restore(gm, dev(y), sigma, kind=ep.CONV_PERIODIC, kernel=k).cpu().numpy()
    b = ep.restore(gm, dev(y), sigma, kind=ep.CONV_DECIMATE, kernel=k, factor=1).cpu().numpy()
    assert np.abs(a - b).max() <= 1e-4
