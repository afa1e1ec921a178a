"""Pins of the FP64 oracle against things other than itself.

Each test checks the oracle (oracle/epll_oracle.c) against a closed form, a
published value, brute force, or an independent dense formulation of the
paper's equations, so that a dropped term, a wrong sign, index or transposed
operand in the oracle fails at least one of them:

* Algorithm 1 written literally in covariance form (dense solves and
  log-determinants, explicit extraction matrices P_i) vs the oracle's
  eigenspace (Eqs. 7-10) and flat-tail (Eqs. 13-16) forms;
* exact ties and brute-force argmin on tiny inputs;
* K = 1: the whole denoising restoration is a linear shift-invariant filter
  whose Fourier-domain recursion is computed by a separate route;
* beta -> infinity: patch extraction + reprojection is the identity;
* the FFT image update / initialisation vs dense N x N solves (Eq. 6);
* conjugate gradients vs a dense solve;
* lambda's closed forms (Sec. "Parameter settings");
* the samplers' coverage / count invariants and the published splitmix64
  outputs.
"""
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# dense literal Algorithm 1 (covariance form), numpy
# --------------------------------------------------------------------------
def flat_cov(U, S, r, lam):
    """Sigma_k with the eigenvalues after r replaced by lam (Sec. flat tail)."""
    s = S.copy()
    if r < len(S):
        s[r:] = lam
    return (U * s[None, :]) @ U.T


def extraction_matrix(H, W, a):
    Pm = np.zeros((64, H * W))
    ai, aj = divmod(int(a), W)
    for u in range(8):
        for v in range(8):
            Pm[u * 8 + v, ((ai + u) % H) * W + (aj + v) % W] = 1.0
    return Pm


def dense_patch_step(g, r, lam, beta, x, anchors, forced=None):
    H, W = x.shape
    K = g.K
    covs = [flat_cov(g.U[k], g.S[k], int(r[k]), lam[k]) for k in range(K)]
    I = np.eye(64)
    num = np.zeros(H * W)
    den = np.zeros((H * W, H * W))
    ks, gaps, allsc = [], [], []
    for n, a in enumerate(anchors):
        Pm = extraction_matrix(H, W, a)
        z = Pm @ x.ravel()
        mu = z.mean()
        zt = z - mu
        sc = np.array([-2 * np.log(g.w[k]) + np.linalg.slogdet(covs[k] + I / beta)[1]
                       + zt @ np.linalg.solve(covs[k] + I / beta, zt) for k in range(K)])
        k = int(np.argmin(sc)) if forced is None else int(forced[n])
        srt = np.sort(sc)
        ks.append(k)
        gaps.append(srt[1] - srt[0] if K > 1 else np.inf)
        allsc.append(sc)
        zh = np.linalg.solve(covs[k] + I / beta, covs[k] @ zt) + mu
        num += Pm.T @ zh
        den += Pm.T @ Pm
    d = np.diag(den)
    xt = np.where(d > 0, num / np.where(d > 0, d, 1), x.ravel())
    return xt.reshape(H, W), np.array(ks), np.array(gaps), np.array(allsc)


@pytest.mark.parametrize("mode,param", [("fixed", 64), ("fixed", 8), ("fixed", 3), ("rho", 0.9)])
def test_patch_step_matches_dense_literal(mode, param):
    g = synth.tiny_gmm(4, seed=11)
    m = oracle.Model(g.w, g.U, g.S, mode, param)
    rng = np.random.default_rng(5)
    x = rng.random((10, 11))
    beta = 1.0 / 0.004
    anchors = np.arange(110)
    xt, ks, gap, best = oracle.patch_step(m, beta, x, anchors)
    dxt, dks, dgap, dsc = dense_patch_step(g, m.r, m.lam, beta, x, anchors)
    assert np.array_equal(ks, dks)
    np.testing.assert_allclose(best, dsc.min(axis=1), rtol=0, atol=1e-9)
    np.testing.assert_allclose(gap, dgap, rtol=0, atol=1e-9)
    np.testing.assert_allclose(xt, dxt, rtol=0, atol=1e-12)
    sc = oracle.scores(m, beta, x, anchors)
    np.testing.assert_allclose(sc, dsc, rtol=0, atol=1e-9)


def test_patch_step_subset_and_forced():
    g = synth.tiny_gmm(3, seed=12)
    m = oracle.Model(g.w, g.U, g.S, "fixed", 5)
    x = np.random.default_rng(6).random((12, 9))
    anchors = np.array([0, 7, 13, 50, 51, 99, 107])
    forced = np.array([2, 0, 1, 1, 0, 2, 2])
    xt, ks, _, _ = oracle.patch_step(m, 300.0, x, anchors, forced)
    dxt, _, _, _ = dense_patch_step(g, m.r, m.lam, 300.0, x, anchors, forced)
    assert np.array_equal(ks, forced)
    np.testing.assert_allclose(xt, dxt, atol=1e-12)


def test_flat_tail_full_rank_is_exact_form():
    """r = P in the fixed mode reproduces the exact (covariance) form."""
    g = synth.tiny_gmm(3, seed=13)
    m = oracle.Model(g.w, g.U, g.S, "fixed", 64)
    assert np.all(m.r == 64) and np.all(m.lam == 0)
    x = np.random.default_rng(7).random((9, 9))
    covs = [(g.U[k] * g.S[k]) @ g.U[k].T for k in range(3)]
    beta = 80.0
    sc = oracle.scores(m, beta, x, [0, 40])
    for n, a in enumerate([0, 40]):
        z = extraction_matrix(9, 9, a) @ x.ravel()
        zt = z - z.mean()
        for k in range(3):
            C = covs[k] + np.eye(64) / beta
            ref = -2 * np.log(g.w[k]) + np.linalg.slogdet(C)[1] + zt @ np.linalg.solve(C, zt)
            assert abs(sc[n, k] - ref) < 1e-9


def test_flat_tail_ranks():
    S = synth.spectrum()[None, :]
    r, lam = oracle.flat_tail(S, "rho", 0.95)
    cum = np.cumsum(S[0])
    assert r[0] == int(np.searchsorted(cum, 0.95 * cum[-1]) + 1)
    assert r[0] == 10
    np.testing.assert_allclose(lam[0], S[0, 10:].mean(), rtol=1e-15)
    r8, lam8 = oracle.flat_tail(S, "fixed", 8)
    assert r8[0] == 8 and abs(lam8[0] - S[0, 8:].mean()) < 1e-18
    with pytest.raises(ValueError):
        oracle.flat_tail(S, "fixed", 0)


def test_exact_tie_goes_to_lowest_index():
    g = synth.tiny_gmm(2, seed=14)
    # components 1, 2 and 3 identical (same weight, basis, spectrum)
    w = np.array([g.w[0], 0.3, 0.3, 0.3])
    U = np.stack([g.U[0], g.U[1], g.U[1], g.U[1]])
    S = np.stack([g.S[0], g.S[1], g.S[1], g.S[1]])
    m = oracle.Model(w / w.sum(), U, S, "fixed", 64)
    x = np.random.default_rng(8).random((8, 8)) * 0.05
    sc = oracle.scores(m, 500.0, x, np.arange(64))
    _, ks, gap, _ = oracle.patch_step(m, 500.0, x)
    for n in range(64):
        assert sc[n, 1] == sc[n, 2] == sc[n, 3]
        assert ks[n] == int(np.argmin(sc[n]))  # numpy: first minimum
        if ks[n] in (1, 2, 3):
            assert ks[n] == 1 and gap[n] == 0.0


def test_brute_force_argmin_tiny():
    g = synth.tiny_gmm(4, seed=15)
    m = oracle.Model(g.w, g.U, g.S, "fixed", 6)
    x = np.random.default_rng(9).random((8, 12))
    sc = oracle.scores(m, 1000.0, x, np.arange(96))
    _, ks, gap, best = oracle.patch_step(m, 1000.0, x)
    for n in range(96):
        order = sorted(range(4), key=lambda k: (sc[n, k], k))
        assert ks[n] == order[0]
        assert gap[n] == sc[n, order[1]] - sc[n, order[0]]
        assert best[n] == sc[n, order[0]]


def test_identity_when_beta_is_infinite():
    """gamma -> 1: the patch step reproduces the image (extraction followed by
    reprojection is the identity, Sec. Algorithm)."""
    g = synth.synthetic_gmm(5)
    m = oracle.Model(g.w, g.U, g.S, "fixed", 8)
    x = synth.image(3, 24, 20)
    xt, _, _, _ = oracle.patch_step(m, 1e13, x)
    np.testing.assert_allclose(xt, x, atol=1e-9)
    sub = oracle.sample(24, 20, oracle.JITTER, 6, seed=3, t=1)
    xt2, _, _, _ = oracle.patch_step(m, 1e13, x, sub)
    np.testing.assert_allclose(xt2, x, atol=1e-9)


# --------------------------------------------------------------------------
# K = 1: a linear shift-invariant filter (Fourier-domain recursion)
# --------------------------------------------------------------------------
def k1_fourier_restore(U, S, r, lam, y, sigma, mults):
    H, W = y.shape
    s = S.copy()
    if r < 64:
        s[r:] = lam
    Y = np.fft.fft2(y)
    X = Y.copy()
    for mt in mults:
        beta = mt / sigma ** 2            # lambda = 1 for denoising
        gam = s / (s + 1.0 / beta)
        Wm = (U * gam[None, :]) @ U.T
        Cm = np.eye(64) - np.ones((64, 64)) / 64
        G = Wm @ Cm + np.ones((64, 64)) / 64
        # xtilde(p) = sum_delta h(delta) x(p + delta), delta = b - a
        h = np.zeros((H, W))
        for a in range(64):
            for b in range(64):
                du = b // 8 - a // 8
                dv = b % 8 - a % 8
                h[du % H, dv % W] += G[a, b] / 64.0
        # DFT of x(p + delta) is exp(+2 pi i omega delta) X
        Hh = np.conj(np.fft.fft2(h))
        X = (Y + mt * Hh * X) / (1.0 + mt)
    return np.real(np.fft.ifft2(X))


@pytest.mark.parametrize("r", [64, 8])
def test_k1_reduces_to_wiener_filter_recursion(r):
    g = synth.synthetic_gmm(1)
    w1 = np.array([1.0])
    m = oracle.Model(w1, g.U, g.S, "fixed", r)
    sigma = 20 / 255
    _, y = synth.denoise_problem(0, 32, sigma)
    xo = oracle.restore(m, y, sigma)
    xf = k1_fourier_restore(g.U[0], g.S[0], r, m.lam[0], y, sigma, [1, 4, 8, 16, 32])
    np.testing.assert_allclose(xo, xf, atol=1e-10)


# --------------------------------------------------------------------------
# image estimation and initialisation vs dense solves (Eq. 6)
# --------------------------------------------------------------------------
def circulant_blur(kernel, H, W):
    A = np.zeros((H * W, H * W))
    kh, kw = kernel.shape
    for i in range(H):
        for j in range(W):
            for u in range(kh):
                for v in range(kw):
                    q = ((i - (u - kh // 2)) % H) * W + (j - (v - kw // 2)) % W
                    A[i * W + j, q] += kernel[u, v]
    return A


def neg_laplacian(H, W):
    L = np.zeros((H * W, H * W))
    for i in range(H):
        for j in range(W):
            p = i * W + j
            L[p, p] += 4
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                L[p, ((i + di) % H) * W + (j + dj) % W] -= 1
    return L


def test_dft_matches_numpy():
    rng = np.random.default_rng(1)
    for H, W in [(16, 16), (12, 18), (7, 5), (24, 9)]:
        x = rng.standard_normal((H, W))
        np.testing.assert_allclose(oracle.dft2(x), np.fft.fft2(x), atol=1e-9)


def test_conv_update_matches_dense_solve():
    H = W = 16
    k = synth.gaussian_kernel(7, 1.2)
    A = circulant_blur(k, H, W)
    rng = np.random.default_rng(2)
    x = rng.random((H, W))
    y = (A @ x.ravel()).reshape(H, W) + 0.01 * rng.standard_normal((H, W))
    np.testing.assert_allclose(synth.blur_periodic(x, k).ravel(), A @ x.ravel(), atol=1e-12)
    xt = rng.random((H, W))
    bs = 0.37
    ref = np.linalg.solve(A.T @ A + bs * np.eye(H * W), A.T @ y.ravel() + bs * xt.ravel())
    np.testing.assert_allclose(oracle.xupdate_conv(k, y, xt, bs).ravel(), ref, atol=1e-10)
    c = 0.013
    ref0 = np.linalg.solve(A.T @ A + c * neg_laplacian(H, W), A.T @ y.ravel())
    np.testing.assert_allclose(oracle.init_conv(k, y, c).ravel(), ref0, atol=1e-9)


def test_pixelwise_update_and_cg_match_dense_solve():
    H, W = 12, 10
    rng = np.random.default_rng(3)
    a = (rng.random((H, W)) < 0.7).astype(float)
    y = a * rng.random((H, W))
    xt = rng.random((H, W))
    bs = 2.5
    ref = np.linalg.solve(np.diag(a.ravel() ** 2) + bs * np.eye(H * W),
                          a.ravel() * y.ravel() + bs * xt.ravel())
    np.testing.assert_allclose(oracle.xupdate_pixelwise(y, xt, bs, a).ravel(), ref, atol=1e-13)
    c = 0.05
    ref0 = np.linalg.solve(np.diag(a.ravel() ** 2) + c * neg_laplacian(H, W), a.ravel() * y.ravel())
    np.testing.assert_allclose(oracle.init_cg(a, y, c, 600).ravel(), ref0, atol=1e-9)


def _dense_sr(k, H, W, d):
    """Dense matrix of A = decimation after the periodic blur, built column by
    column from unit images with the input generator's blur."""
    cols = []
    for p in range(H * W):
        e = np.zeros(H * W)
        e[p] = 1.0
        cols.append(synth.blur_periodic(e.reshape(H, W), k)[::d, ::d].ravel())
    return np.array(cols).T


@pytest.mark.parametrize("H,W,d", [(12, 12, 3), (12, 18, 2), (10, 10, 1)])
def test_sr_operator_lambda_and_solves_match_dense(H, W, d):
    """Super-resolution A = S B: the oracle's A and A^T are the dense matrix
    and its transpose; lambda = N^-1 ||A^T A||_F^2 / ||A||_2^2 computed from
    the dense matrix; the image update and the initialisation equal dense
    solves of (A^T A + bs I) x = A^T y + bs xt and (A^T A + c L) x = A^T y."""
    k = synth.gaussian_kernel(7, 1.1)
    A = _dense_sr(k, H, W, d)
    rng = np.random.default_rng(H + W + d)
    x = rng.random((H, W))
    yl = rng.random((H // d, W // d))
    np.testing.assert_allclose(oracle.sr_apply(k, x, d).ravel(), A @ x.ravel(), atol=1e-13)
    np.testing.assert_allclose(oracle.sr_adjoint(k, yl, d).ravel(), A.T @ yl.ravel(), atol=1e-13)
    AtA = A.T @ A
    lam_dense = (np.sum(AtA ** 2) / (H * W)) / np.linalg.norm(A, 2) ** 2
    sigma = 40 / 255  # cap 250 (40)^2 far above
    assert abs(oracle.lam_sr(k, H, W, d, sigma) - lam_dense) <= 1e-12 * lam_dense
    xt = rng.random((H, W))
    bs = 0.21
    ref = np.linalg.solve(AtA + bs * np.eye(H * W), A.T @ yl.ravel() + bs * xt.ravel())
    np.testing.assert_allclose(oracle.xupdate_sr(k, yl, xt, d, bs).ravel(), ref, atol=1e-11)
    c = 0.017
    ref0 = np.linalg.solve(AtA + c * neg_laplacian(H, W), A.T @ yl.ravel())
    np.testing.assert_allclose(oracle.init_sr(k, yl, d, c).ravel(), ref0, atol=1e-9)


def test_sr_factor_one_is_the_deconvolution():
    """With d = 1 the super-resolution operator is the periodic blur: lambda,
    the initialisation, the image update and a whole restoration equal those
    of the deconvolution (a Fourier-domain route)."""
    H, W = 24, 20
    k = synth.gaussian_kernel(9, 1.3)
    rng = np.random.default_rng(4)
    y = synth.blur_periodic(synth.image(3, H, W), k) + 0.01 * rng.standard_normal((H, W))
    sigma = 0.01
    assert abs(oracle.lam_sr(k, H, W, 1, sigma) - oracle.lam(oracle.CONV, H, W, sigma, kernel=k)) < 1e-14
    c = 0.2 * sigma ** 2 / oracle.lam(oracle.CONV, H, W, sigma, kernel=k)
    np.testing.assert_allclose(oracle.init_sr(k, y, 1, c), oracle.init_conv(k, y, c), atol=1e-8)
    xt = rng.random((H, W))
    np.testing.assert_allclose(oracle.xupdate_sr(k, y, xt, 1, 0.05), oracle.xupdate_conv(k, y, xt, 0.05),
                               atol=1e-11)
    g = synth.tiny_gmm(3, seed=2)
    m = oracle.Model(g.w, g.U, g.S, "fixed", 8)
    a = oracle.restore(m, y, sigma, (1, 4), deg=oracle.SR, kernel=k, factor=1)
    b = oracle.restore(m, y, sigma, (1, 4), deg=oracle.CONV, kernel=k)
    np.testing.assert_allclose(a, b, atol=1e-8)


def test_valid_boundary_sampler_and_weights():
    """`valid` boundary: exactly the (H-7)(W-7) patches inside the image, in
    raster order; the weights are the brute-force patch count over P."""
    for H, W in ((8, 8), (10, 12), (17, 9)):
        an = oracle.sample(H, W, oracle.VALID)
        assert len(an) == (H - 7) * (W - 7)
        i, j = np.divmod(an, W)
        assert (i <= H - 8).all() and (j <= W - 8).all() and np.all(np.diff(an) > 0)
        cnt = np.zeros((H, W))
        for a in an:
            r, c = divmod(int(a), W)
            cnt[r:r + 8, c:c + 8] += 1
        np.testing.assert_array_equal(oracle.valid_weights(H, W), cnt / 64)


@pytest.mark.parametrize("deg", ["denoise", "mask", "blur"])
def test_weighted_update_is_eq6_with_valid_patches(deg):
    """The image update with the `valid` boundary equals Eq. 6 written with
    the literal patch extraction matrices P_i of the valid patches:
    x = (A^T A + b' sum P_i^T P_i)^-1 (A^T y + b' sum P_i^T zhat_i), b' = bs / P,
    for random patch estimates zhat_i (the blur's conjugate gradients run to
    convergence here)."""
    H, W = 11, 13
    rng = np.random.default_rng(3)
    an = oracle.sample(H, W, oracle.VALID)
    Ps = []
    for a in an:
        r, c = divmod(int(a), W)
        P = np.zeros((64, H * W))
        for e in range(64):
            P[e, (r + e // 8) * W + c + e % 8] = 1.0
        Ps.append(P)
    zh = rng.standard_normal((len(an), 64)) * 0.1 + 0.5
    S = sum(P.T @ P for P in Ps)
    Z = sum(P.T @ z for P, z in zip(Ps, zh))
    cnt = np.diag(S)
    xt = (Z / cnt).reshape(H, W)
    wgt = oracle.valid_weights(H, W)
    y = rng.random((H, W))
    bs = 0.37
    a = kern = None
    if deg == "denoise":
        A, kind = np.eye(H * W), oracle.DENOISE
    elif deg == "mask":
        a = (rng.random((H, W)) < 0.7).astype(float)
        A, kind = np.diag(a.ravel()), oracle.PIXELWISE
    else:
        kern = synth.gaussian_kernel(5, 1.0)
        A, kind = circulant_blur(kern, H, W), oracle.CONV
    ref = np.linalg.solve(A.T @ A + bs / 64 * S, A.T @ y.ravel() + bs / 64 * Z)
    got = oracle.xupdate_weighted(kind, y, xt, wgt, bs, a=a, kernel=kern, iters=5000)
    np.testing.assert_allclose(got.ravel(), ref, atol=1e-10)
    if deg == "blur":
        # with uniform weights the conjugate gradients reach the Fourier solve
        got1 = oracle.xupdate_weighted(kind, y, xt, np.ones((H, W)), bs, kernel=kern, iters=5000)
        np.testing.assert_allclose(got1, oracle.xupdate_conv(kern, y, xt, bs), atol=1e-10)


def test_lambda_closed_forms():
    H = W = 16
    assert oracle.lam(oracle.DENOISE, H, W, 20 / 255) == 1.0
    a = synth.observed_mask(0, H, W, 0.7)
    assert abs(oracle.lam(oracle.PIXELWISE, H, W, 20 / 255, a=a) - a.mean()) < 1e-15
    k = synth.gaussian_kernel(25, 1.6)
    A = circulant_blur(k, H, W)
    AtA = A.T @ A
    ref = np.linalg.norm(AtA, "fro") ** 2 / (H * W) / np.linalg.norm(A, 2) ** 2
    assert abs(oracle.lam(oracle.CONV, H, W, 2 / 255, kernel=k) - ref) < 1e-12
    assert abs(oracle.lam(oracle.CONV, 512, 512, 2 / 255, kernel=k) - 0.01554) < 5e-6
    # the 250 sigma^2 cap, sigma in grey levels
    assert abs(oracle.lam(oracle.DENOISE, H, W, 0.01 / 255) - 250 * 0.01 ** 2) < 1e-15


# --------------------------------------------------------------------------
# whole restorations vs a dense literal restoration (tiny)
# --------------------------------------------------------------------------
def dense_restore(g, r, lam_k, y, sigma, mults, deg, a=None, kernel=None, anchors_fn=None,
                  cg_exact=True):
    H, W = y.shape
    N = H * W
    if deg == oracle.DENOISE:
        A = np.eye(N)
    elif deg == oracle.PIXELWISE:
        A = np.diag(a.ravel())
    else:
        A = circulant_blur(kernel, H, W)
    AtA = A.T @ A
    lm = min(np.linalg.norm(AtA, "fro") ** 2 / N / np.linalg.norm(A, 2) ** 2, 250 * (255 * sigma) ** 2)
    c = 0.2 * sigma ** 2 / lm
    if deg == oracle.DENOISE:
        x = y.ravel().copy()
    else:
        x = np.linalg.solve(AtA + c * neg_laplacian(H, W), A.T @ y.ravel())
    for t, mt in enumerate(mults):
        bs = lm * mt
        beta = bs / sigma ** 2
        anchors = np.arange(N) if anchors_fn is None else anchors_fn(t)
        xt, _, _, _ = dense_patch_step(g, r, lam_k, beta, x.reshape(H, W), anchors)
        x = np.linalg.solve(AtA + bs * np.eye(N), A.T @ y.ravel() + bs * xt.ravel())
    return x.reshape(H, W), lm


def test_restore_deblur_matches_dense():
    g = synth.tiny_gmm(2, seed=21)
    m = oracle.Model(g.w, g.U, g.S, "fixed", 6)
    k = synth.gaussian_kernel(5, 1.0)
    x = synth.image(5, 10, 10)
    sigma = 5 / 255
    y = synth.blur_periodic(x, k) + synth.noise(5, 10, 10, sigma)
    xo = oracle.restore(m, y, sigma, [1, 4, 8], deg=oracle.CONV, kernel=k)
    xd, _ = dense_restore(g, m.r, m.lam, y, sigma, [1, 4, 8], oracle.CONV, kernel=k)
    np.testing.assert_allclose(xo, xd, atol=1e-8)


def test_restore_inpaint_subset_matches_dense():
    g = synth.tiny_gmm(2, seed=22)
    m = oracle.Model(g.w, g.U, g.S, "fixed", 64)
    H, W = 10, 9
    x = synth.image(6, H, W)
    a = synth.observed_mask(6, H, W, 0.7)
    sigma = 10 / 255
    y = a * x + synth.noise(6, H, W, sigma)
    xo = oracle.restore(m, y, sigma, [1, 4], deg=oracle.PIXELWISE, a=a,
                        subset=oracle.FRACTION, subset_param=1 / 3, seed=9, cg_iters=400)
    fn = lambda t: oracle.sample(H, W, oracle.FRACTION, 1 / 3, seed=9, t=t)
    xd, lm = dense_restore(g, m.r, m.lam, y, sigma, [1, 4], oracle.PIXELWISE, a=a, anchors_fn=fn)
    assert abs(lm - a.mean()) < 1e-15
    np.testing.assert_allclose(xo, xd, atol=1e-8)


# --------------------------------------------------------------------------
# samplers and random numbers
# --------------------------------------------------------------------------
def test_splitmix64_published_values():
    vals = [int(l, 16) for l in open(os.path.join(GOLD, "splitmix64.txt")) if l.startswith("0x")]
    assert [oracle.splitmix64_nth(0, n) for n in (1, 2, 3)] == vals


@pytest.mark.parametrize("H,W,s", [(64, 64, 6), (50, 37, 6), (33, 40, 4), (20, 20, 8), (17, 23, 5)])
def test_jitter_covers_every_pixel(H, W, s):
    J = (8 - s) // 2
    for t in range(4):
        an = oracle.sample(H, W, oracle.JITTER, s, seed=123, t=t)
        ni, nj = -(-H // s), -(-W // s)
        assert an.shape[0] == ni * nj
        cov = np.zeros((H, W), int)
        for a in an:
            i, j = divmod(int(a), W)
            for u in range(8):
                for v in range(8):
                    cov[(i + u) % H, (j + v) % W] += 1
        assert cov.min() >= 1
        # offsets from the shifted grid stay within [-J, J]
        gi = [oracle.rng_u64(123, t, 0) >> 32, oracle.rng_u64(123, t, 1) >> 32]
        gi = [(v * s) >> 32 for v in gi]
        for g_, a in enumerate(an):
            n, mm = divmod(g_, nj)
            i, j = divmod(int(a), W)
            di = (i - (gi[0] + s * n)) % H
            dj = (j - (gi[1] + s * mm)) % W
            assert min(di, H - di) <= J and min(dj, W - dj) <= J


@pytest.mark.parametrize("H,W,s", [(64, 64, 8), (50, 37, 3), (17, 23, 5), (8, 8, 8), (20, 13, 2)])
def test_regular_grid_pins(H, W, s):
    """Regular patch subsampling (Sec. on the random subset of patches): |I| =
    N / s^2 when s divides both sides (ceil otherwise), every pixel covered for
    s <= 8, the same list at every iteration; at s = 8 it is the jittered grid
    (J = 0 there) without its random shift; at s = 1 it is the full set."""
    an = oracle.sample(H, W, oracle.REGULAR, s)
    assert an.shape[0] == -(-H // s) * -(-W // s)
    if H % s == 0 and W % s == 0:
        assert an.shape[0] * s * s == H * W
    assert len(set(an.tolist())) == an.shape[0]
    cov = np.zeros((H, W), int)
    for a in an:
        i, j = divmod(int(a), W)
        cov[np.ix_((np.arange(8) + i) % H, (np.arange(8) + j) % W)] += 1
    assert cov.min() >= 1
    assert np.array_equal(an, oracle.sample(H, W, oracle.REGULAR, s, seed=9, t=3))
    if s == 8:
        for t in range(3):
            jit = oracle.sample(H, W, oracle.JITTER, 8, seed=77, t=t)
            gi = ((oracle.rng_u64(77, t, 0) >> 32) * 8) >> 32
            gj = ((oracle.rng_u64(77, t, 1) >> 32) * 8) >> 32
            ji, jj = np.divmod(jit, W)
            unshifted = ((ji - gi) % H) * W + (jj - gj) % W
            assert np.array_equal(unshifted, an)
    assert np.array_equal(oracle.sample(H, W, oracle.REGULAR, 1), oracle.sample(H, W, oracle.FULL))


def test_jitter_expected_coverage_is_uniform():
    """The random global shift makes every pixel's expected coverage equal
    (Sec. on the random subset of patches)."""
    H = W = 24
    acc = np.zeros((H, W))
    T = 600
    for t in range(T):
        for a in oracle.sample(H, W, oracle.JITTER, 6, seed=5, t=t):
            i, j = divmod(int(a), W)
            acc[np.ix_((np.arange(8) + i) % H, (np.arange(8) + j) % W)] += 1
    acc /= T
    expect = 64 * (H // 6) * (W // 6) / (H * W)
    assert abs(acc.mean() - expect) < 1e-12
    assert acc.std() / acc.mean() < 0.05


def test_fraction_sampler_count_and_order():
    H, W = 40, 37
    for t in range(3):
        an = oracle.sample(H, W, oracle.FRACTION, 1 / 3, seed=77, t=t)
        M = math.ceil(H * W / 3)
        assert an.shape[0] == M
        assert np.all(np.diff(an) > 0)
        keys = np.array([oracle.rng_u64(77, t, a) >> 32 for a in range(H * W)], dtype=np.uint64)
        order = np.lexsort((np.arange(H * W), keys))
        assert np.array_equal(np.sort(order[:M]), an)


# --------------------------------------------------------------------------
# proposal network (oracle/mlp.py): gradient pinned by central differences
# --------------------------------------------------------------------------
def test_mlp_gradient_matches_central_differences():
    from oracle import mlp
    K = 7
    rng = np.random.default_rng(3)
    theta = rng.standard_normal(mlp.n_params(K)) * 0.1
    p = mlp.unpack(theta, K)
    X = rng.standard_normal((5, 64))
    cond = rng.standard_normal(5)
    labels = rng.integers(0, K, 5)
    L, g = mlp.loss_and_grad(p, X, cond, labels)
    assert abs(L - mlp.loss(p, X, cond, labels)) < 1e-12
    gv = mlp.pack(g, K)
    idx = rng.choice(theta.size, 60, replace=False)
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        num = (mlp.loss(mlp.unpack(tp, K), X, cond, labels) - mlp.loss(mlp.unpack(tm, K), X, cond, labels)) / (2 * h)
        assert abs(num - gv[i]) < 1e-7 + 1e-5 * abs(num), (i, num, gv[i])


def test_mlp_gelu_and_softmax_closed_forms():
    from oracle import mlp
    from scipy.stats import norm
    # the tanh form is within 5e-4 of the exact GELU x Phi(x) (its published
    # accuracy); a wrong constant (0.04 for 0.044715, 0.8 for sqrt(2/pi)) is not
    x = np.linspace(-10, 10, 20001)
    assert np.abs(mlp.gelu(x) - x * norm.cdf(x)).max() < 5e-4
    assert np.abs(mlp.gelu_grad(x) - (norm.cdf(x) + x * norm.pdf(x))).max() < 2e-3
    # derivative against central differences of the function itself
    h = 1e-5
    np.testing.assert_allclose(mlp.gelu_grad(x), (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h), atol=1e-8)
    # uniform logits: loss = log K
    K = 5
    p = mlp.unpack(np.zeros(mlp.n_params(K)), K)
    assert abs(mlp.loss(p, np.ones((3, 64)), np.zeros(3), np.array([0, 2, 4])) - np.log(K)) < 1e-14


def _adamw_variant(p, g, m, v, step, lr, wd, bias_correction=True, coupled=False):
    """AdamW with a planted mistake (test of the pins' and the GPU test's
    sensitivity): no bias correction, or the decay folded into the gradient
    (Adam with L2 regularisation instead of decoupled decay)."""
    from oracle import mlp
    c1 = 1.0 - mlp.ADAM_B1 ** step if bias_correction else 1.0
    c2 = 1.0 - mlp.ADAM_B2 ** step if bias_correction else 1.0
    p2, m2, v2 = {}, {}, {}
    for k in p:
        gk = g[k] + (wd * p[k] if coupled and k in mlp.DECAYED else 0.0)
        m2[k] = mlp.ADAM_B1 * m[k] + (1 - mlp.ADAM_B1) * gk
        v2[k] = mlp.ADAM_B2 * v[k] + (1 - mlp.ADAM_B2) * gk * gk
        u = (m2[k] / c1) / (np.sqrt(v2[k] / c2) + mlp.ADAM_EPS)
        if k in mlp.DECAYED and not coupled:
            u = u + wd * p[k]
        p2[k] = p[k] - lr * u
    return p2, m2, v2


def test_adamw_matches_torch_and_closed_form():
    """The AdamW oracle against an independent implementation (torch.optim.AdamW
    on the weight matrices, torch.optim.Adam without decay on the biases and wb,
    float64) over several steps; the first step in closed form (m_hat = g,
    v_hat = g^2: the update is lr (g / (|g| + eps) + wd theta)); and planted
    mistakes (no bias correction, decay coupled into the gradient) are far off."""
    import torch
    from oracle import mlp
    K = 6
    rng = np.random.default_rng(21)
    p = mlp.unpack(rng.standard_normal(mlp.n_params(K)) * 0.3, K)
    grads = [mlp.unpack(rng.standard_normal(mlp.n_params(K)) * 10.0 ** rng.uniform(-4, 0), K) for _ in range(5)]
    lr, wd = 1e-2, 0.5
    tp = {k: torch.tensor(p[k], dtype=torch.float64, requires_grad=True) for k in p}
    opt_w = torch.optim.AdamW([tp[k] for k in mlp.DECAYED], lr=lr, betas=(mlp.ADAM_B1, mlp.ADAM_B2),
                              eps=mlp.ADAM_EPS, weight_decay=wd)
    opt_b = torch.optim.Adam([tp[k] for k in p if k not in mlp.DECAYED], lr=lr,
                             betas=(mlp.ADAM_B1, mlp.ADAM_B2), eps=mlp.ADAM_EPS, weight_decay=0.0)
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(x) for k, x in p.items()}
    q = dict(p)
    for t, g in enumerate(grads, start=1):
        if t == 1:
            q1, _, _ = mlp.adamw_step(q, g, m, v, 1, lr, wd)
            for k in q:
                ref = q[k] - lr * (g[k] / (np.abs(g[k]) + mlp.ADAM_EPS) + (wd * q[k] if k in mlp.DECAYED else 0.0))
                np.testing.assert_allclose(q1[k], ref, rtol=0, atol=1e-15)
        q, m, v = mlp.adamw_step(q, g, m, v, t, lr, wd)
        for k in tp:
            tp[k].grad = torch.tensor(g[k], dtype=torch.float64)
        opt_w.step()
        opt_b.step()
        for k in q:
            np.testing.assert_allclose(q[k], tp[k].detach().numpy(), rtol=0, atol=1e-14)
    # planted mistakes, three steps from the same start: the moved parameters
    # differ from the oracle's by a sizeable fraction of the step length
    # (also at the GPU test's lr = 1e-3, wd = 2)
    for lr_, wd_ in ((lr, wd), (1e-3, 2.0)):
        for kw in (dict(bias_correction=False), dict(coupled=True)):
            a, am, av = dict(p), {k: np.zeros_like(x) for k, x in p.items()}, {k: np.zeros_like(x) for k, x in p.items()}
            b, bm, bv = dict(p), dict(am), dict(av)
            for t, g in enumerate(grads[:3], start=1):
                a, am, av = mlp.adamw_step(a, g, am, av, t, lr_, wd_)
                b, bm, bv = _adamw_variant(b, g, bm, bv, t, lr_, wd_, **kw)
            d = max(np.abs(a[k] - b[k]).max() for k in mlp.DECAYED)
            assert d > 0.1 * lr_, (kw, lr_, d)


def test_bf16_rounding_matches_torch_and_ties_to_even():
    import torch
    from oracle import mlp
    rng = np.random.default_rng(11)
    x = rng.standard_normal(20000) * np.exp(rng.uniform(-30, 30, 20000))
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).double().numpy()
    np.testing.assert_array_equal(mlp.bf16(x), ref)
    # halfway cases round to the even mantissa
    np.testing.assert_array_equal(mlp.bf16(np.array([1 + 2.0**-8, 1 + 3 * 2.0**-8, -(1 + 2.0**-8), 2.0**-133])),
                                  np.array([1.0, 1 + 2.0**-6, -1.0, 2.0**-133]))


def test_mlp_inference_form_scaling_and_topm():
    """The inference form is the training forward at X = sqrt(beta) z, cond =
    log(1/beta) up to the BF16 roundings of z and of the hidden activations;
    top-m takes the lowest index first on equal logits."""
    from oracle import mlp
    K = 9
    rng = np.random.default_rng(5)
    p = mlp.unpack(rng.standard_normal(mlp.n_params(K)) * 0.1, K)
    Z = rng.standard_normal((40, 64)) * 0.05
    ibeta = 0.01
    li = mlp.forward_infer(p, Z, ibeta)
    lt, _ = mlp.forward(mlp.round_weights(p), Z / np.sqrt(ibeta), np.full(40, np.log(ibeta)))
    scale = np.abs(lt).max()
    assert np.abs(li - lt).max() < 2e-2 * scale
    # a wrong scaling convention (z / sqrt(beta)) is far off
    lw, _ = mlp.forward(mlp.round_weights(p), Z * np.sqrt(ibeta), np.full(40, np.log(ibeta)))
    assert np.abs(lw - lt).max() > 0.2 * scale
    logits = np.array([[0.0, 2.0, 2.0, 1.0], [3.0, 3.0, 3.0, 3.0]])
    idx, mass = mlp.topm(logits, 2)
    np.testing.assert_array_equal(idx, [[1, 2], [0, 1]])
    e = np.exp(logits[0] - 2.0)
    np.testing.assert_allclose(mass, [2 / e.sum(), 0.5], rtol=1e-15)


def test_tree_kl_closed_forms():
    """Eq. 17: for diagonal covariances 1/2 sum(a/b + b/a - 2); zero for equal
    covariances; symmetric; invariant under a common rotation."""
    from oracle import tree
    rng = np.random.default_rng(8)
    a, b = rng.uniform(0.1, 2.0, 64), rng.uniform(0.1, 2.0, 64)
    assert abs(tree.sym_kl(np.diag(a), np.diag(b)) - 0.5 * np.sum(a / b + b / a - 2)) < 1e-10
    A = rng.standard_normal((64, 64))
    A = A @ A.T + 64 * np.eye(64)
    B = rng.standard_normal((64, 64))
    B = B @ B.T + 64 * np.eye(64)
    assert abs(tree.sym_kl(A, A)) < 1e-10
    assert abs(tree.sym_kl(A, B) - tree.sym_kl(B, A)) < 1e-10
    Q, _ = np.linalg.qr(rng.standard_normal((64, 64)))
    assert abs(tree.sym_kl(Q @ A @ Q.T, Q @ B @ Q.T) - tree.sym_kl(A, B)) < 1e-8 * tree.sym_kl(A, B)


def test_tree_collapse_is_the_mixture_second_moment():
    """Eq. 19: the collapsed covariance is the second moment of samples drawn
    from the cluster's zero-mean mixture (Monte Carlo, 400k samples)."""
    from oracle import tree
    rng = np.random.default_rng(9)
    P = 4
    covs = []
    for _ in range(3):
        M = rng.standard_normal((P, P))
        covs.append(M @ M.T + 0.5 * np.eye(P))
    w = np.array([0.2, 0.5, 0.3])
    wl, cl = tree.collapse(w, covs, [[0, 1, 2]])
    assert abs(wl[0] - 1.0) < 1e-15
    n = 400_000
    comp = rng.choice(3, n, p=w)
    x = np.empty((n, P))
    for k in range(3):
        sel = comp == k
        x[sel] = rng.multivariate_normal(np.zeros(P), covs[k], sel.sum())
    emp = x.T @ x / n
    assert np.abs(emp - cl[0]).max() < 0.03 * np.abs(cl[0]).max()


def test_tree_partition_balanced_and_swap_optimal():
    """Clusters partition the components with sizes floor(n/L) or ceil(n/L),
    no single swap lowers Eq. 18, and the cost beats random balanced partitions;
    on 8 components in 2 clusters it is compared with brute force."""
    import itertools
    from oracle import tree
    import synth
    g = synth.synthetic_gmm(23)
    covs = [g.U[k] @ np.diag(g.S[k]) @ g.U[k].T for k in range(23)]
    D = tree.kl_matrix(covs)
    parts = tree.partition(D, g.w, 8)
    assert sorted(sum(parts, [])) == list(range(23))
    assert sorted(len(p) for p in parts) == [2] + [3] * 7
    c = tree.cost(D, parts)
    for a, b in itertools.combinations(range(23), 2):
        la = next(i for i, p in enumerate(parts) if a in p)
        lb = next(i for i, p in enumerate(parts) if b in p)
        if la == lb:
            continue
        q = [list(p) for p in parts]
        q[la][q[la].index(a)] = b
        q[lb][q[lb].index(b)] = a
        assert tree.cost(D, q) >= c - 1e-9
    rng = np.random.default_rng(1)
    for _ in range(20):
        perm = rng.permutation(23)
        sizes = [len(p) for p in parts]
        q, o = [], 0
        for s_ in sizes:
            q.append(perm[o:o + s_].tolist())
            o += s_
        assert tree.cost(D, q) >= c
    D8 = D[:8, :8]
    p8 = tree.partition(D8, g.w[:8], 2)
    best = min(tree.cost(D8, [list(s_), [x for x in range(8) if x not in s_]])
               for s_ in itertools.combinations(range(8), 4))
    assert tree.cost(D8, p8) <= best * 1.10


def test_tree_descent_special_cases():
    """A root with every component as a child is the exhaustive argmin (lowest
    index on ties); a hand-built two-level tree follows the cheaper branch even
    when a leaf of the other branch is cheaper."""
    from oracle import tree
    rng = np.random.default_rng(4)
    sc = rng.standard_normal((50, 6))
    sc[3, 2] = sc[3, 4] = sc[3].min() - 1.0
    cb = np.array([1, 7, 7, 7, 7, 7, 7, 7])   # root 0 -> nodes 1..6 (leaves)
    leaf, gap = tree.descend(np.concatenate([np.zeros((50, 1)), sc], axis=1), cb)
    assert np.array_equal(leaf - 1, np.argmin(sc, axis=1))
    assert leaf[3] == 3 and gap[3] == 0.0
    # root 0 -> {1, 2}; 1 -> {3, 4}; 2 -> {5, 6}
    cb2 = np.array([1, 3, 5, 7, 7, 7, 7, 7])
    s2 = np.array([[0, 1.0, 2.0, 5.0, 4.0, 0.5, 3.0]])
    leaf2, gap2 = tree.descend(s2, cb2)
    assert leaf2[0] == 4 and abs(gap2[0] - 1.0) < 1e-15


def test_tree_level_sizes_follow_the_paper():
    """K = 200 collapses to 64, 32, 16, 8, 4, 2 and 1 components (327 nodes)."""
    from oracle import tree
    s = tree.level_sizes(200)
    assert s == [64, 32, 16, 8, 4, 2, 1] and 200 + sum(s) == 327
