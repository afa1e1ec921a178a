"""Parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (FP32 mode): component selection identical to the oracle's outside
near-ties (oracle top-2 gap < 1e-4), patch averages within 1e-5 on the same
input, restored images within 1e-4 max abs error and 0.05 dB PSNR.
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

import paper_1710_08124_gb300 as ep  # noqa: E402

TIE = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    ep.build()


def psnr(x, ref):
    return -10 * math.log10(float(np.mean((np.asarray(x, np.float64) - ref) ** 2)))


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")


def models(K, mode="fixed", param=64, gmm=None):
    g = gmm or synth.synthetic_gmm(K)
    rm = ep.RANK_FIXED if mode == "fixed" else ep.RANK_RHO
    return ep.gmm_load(g.w, g.U, g.S, rm, param), oracle.Model(g.w, g.U, g.S, mode, param)


def agree(ks_gpu, ks_or, gap_or):
    ok = (ks_gpu == ks_or) | (gap_or < TIE)
    return ok


# ---------------------------------------------------------------- sampler
@pytest.mark.parametrize("H,W", [(64, 64), (50, 37), (8, 8), (129, 200)])
def test_sampler_bit_identical(H, W):
    for t in range(3):
        for kind, param in [(ep.SUBSET_FRACTION, 1 / 3), (ep.SUBSET_FRACTION, 0.05),
                            (ep.SUBSET_JITTER, 6), (ep.SUBSET_JITTER, 3),
                            (ep.SUBSET_REGULAR, 3), (ep.SUBSET_REGULAR, 8), (ep.SUBSET_VALID, 0)]:
            o = ep.Options(subset=kind, subset_param=param, seed=1234 + t)
            g = ep.sample(H, W, o, t).cpu().numpy()
            r = oracle.sample(H, W, kind, param, seed=1234 + t, t=t)
            assert np.array_equal(g, r), (H, W, kind, param, t)
    a = ep.sample(H, W, ep.Options(), 0).cpu().numpy()
    assert np.array_equal(a, np.arange(H * W))


# ---------------------------------------------------------------- patch step
def _check_step(gm, om, x, beta, opts, t=0, xt_tol=1e-5):
    xt, an, ks, gp = ep.patch_step(gm, dev(x), beta, opts, t)
    xt, an, ks, gp = (v.cpu().numpy() for v in (xt, an, ks, gp))
    oxt, oks, ogap, _ = oracle.patch_step(om, beta, x.astype(np.float32).astype(np.float64), an)
    ok = agree(ks, oks, ogap)
    assert ok.all(), f"{(~ok).sum()} disagreements, oracle gaps {ogap[~ok][:5]}"
    if np.array_equal(ks, oks):
        np.testing.assert_allclose(xt, oxt, atol=xt_tol, rtol=0)
    # teacher forcing with the oracle's selection reproduces its patch average
    fxt, _, fks, _ = ep.patch_step(gm, dev(x), beta, opts, t, forced_k=torch.as_tensor(oks, device="cuda"))
    assert np.array_equal(fks.cpu().numpy(), oks)
    np.testing.assert_allclose(fxt.cpu().numpy(), oxt, atol=xt_tol, rtol=0)
    return ks, gp, oks, ogap


def test_patch_step_config1_all_betas():
    """64x64, K=20, full rank, sigma=20/255, every beta of the schedule."""
    gm, om = models(20)
    sigma = 20 / 255
    _, y = synth.denoise_problem(0, 64, sigma)
    xs = oracle.restore(om, y, sigma, [1, 4])
    for x in (y, xs):
        for m in ep.PAPER_BETA:
            _check_step(gm, om, x, m / sigma ** 2, ep.Options())


@pytest.mark.parametrize("r", [8, 64])
@pytest.mark.parametrize("subset,param", [(ep.SUBSET_FRACTION, 1 / 3), (ep.SUBSET_JITTER, 6)])
def test_patch_step_subsets_ragged(r, subset, param):
    gm, om = models(37, "fixed", r)
    sigma = 25 / 255
    _, y = synth.denoise_problem(1, 50, sigma, W=37)
    for t in range(2):
        _check_step(gm, om, y, 8 / sigma ** 2, ep.Options(subset=subset, subset_param=param, seed=5), t)


@pytest.mark.parametrize("prec", [ep.AUTO, ep.FP32])
@pytest.mark.parametrize("r", [8, 64])
def test_reprojection_with_duplicate_anchors(r, prec):
    """The jittered grid on a side its spacing does not divide places some
    anchors twice across the wrap seam, and such an anchor counts twice.  The
    reprojection reads one estimate per anchor through its index in the subset
    and weighs it by the multiplicity: patch averages within 1e-5 of the
    oracle's, and the whole restoration within 1e-4."""
    H, W, seed = 50, 37, 1
    an = oracle.sample(H, W, oracle.JITTER, 6, seed, 0)
    _, cnt = np.unique(an, return_counts=True)
    assert (cnt > 1).any()
    gm, om = models(37, "fixed", r)
    sigma = 25 / 255
    x, y = synth.denoise_problem(1, H, sigma, W=W)
    o = ep.Options(precision=prec, subset=ep.SUBSET_JITTER, subset_param=6, seed=seed)
    _check_step(gm, om, y, 8 / sigma ** 2, o, 0)
    xo = oracle.restore(om, y.astype(np.float32).astype(np.float64), sigma, subset=oracle.JITTER,
                        subset_param=6, seed=seed)
    xg = ep.restore(gm, dev(y), sigma, options=o).cpu().numpy()
    assert np.abs(xg - xo).max() <= 1e-4


def test_patch_step_rho_ranks():
    g = synth.tiny_gmm(9, seed=31)
    gm, om = models(9, "rho", 0.9, gmm=g)
    r, lam = gm.ranks()
    assert np.array_equal(r, om.r) and np.allclose(lam, om.lam, rtol=1e-15)
    x = synth.image(2, 40, 24) + synth.noise(2, 40, 24, 0.05)
    _check_step(gm, om, x, 1 / 0.001, ep.Options())


def test_patch_step_k1_and_min_size():
    gm, om = models(1)
    x = synth.image(4, 8, 8)
    _check_step(gm, om, x, 400.0, ep.Options())
    gm2, om2 = models(3, "fixed", 8)
    _check_step(gm2, om2, synth.image(5, 9, 13), 900.0, ep.Options())


def test_exact_ties_lowest_index():
    g = synth.tiny_gmm(2, seed=14)
    w = np.array([g.w[0], 0.3, 0.3, 0.3])
    U = np.stack([g.U[0], g.U[1], g.U[1], g.U[1]])
    S = np.stack([g.S[0], g.S[1], g.S[1], g.S[1]])
    gm = ep.gmm_load(w / w.sum(), U, S)
    x = (np.random.default_rng(8).random((8, 8)) * 0.05).astype(np.float32)
    _, _, ks, _ = ep.patch_step(gm, dev(x), 500.0)
    ks = ks.cpu().numpy()
    assert not np.isin(ks, [2, 3]).any()


# ---------------------------------------------------------------- restores
def test_restore_config1():
    """The small EPLL denoising case: 64x64, K=20, sigma=20/255, five iterations."""
    gm, om = models(20)
    sigma = 20 / 255
    x, y = synth.denoise_problem(0, 64, sigma)
    xo = oracle.restore(om, y.astype(np.float32).astype(np.float64), sigma)
    xg = ep.restore(gm, dev(y), sigma).cpu().numpy()
    err = np.abs(xg - xo).max()
    assert err <= 1e-4, err
    assert abs(psnr(xg, x) - psnr(xo, x)) <= 0.05
    xh = ep.restore_host(gm, y.astype(np.float32), sigma)
    assert np.array_equal(xh, xg)


def test_restore_subset_jitter():
    gm, om = models(30, "fixed", 8)
    sigma = 25 / 255
    x, y = synth.denoise_problem(3, 72, sigma, W=56)
    o = ep.Options(subset=ep.SUBSET_JITTER, subset_param=6, seed=11)
    xo = oracle.restore(om, y.astype(np.float32).astype(np.float64), sigma, subset=oracle.JITTER,
                        subset_param=6, seed=11)
    xg = ep.restore(gm, dev(y), sigma, options=o).cpu().numpy()
    assert abs(psnr(xg, x) - psnr(xo, x)) <= 0.05
    assert np.abs(xg - xo).max() <= 1e-4


def test_restore_subset_regular():
    """Regular patch subsampling with spacing 3 (the paper's 9x setting)."""
    gm, om = models(30, "fixed", 8)
    sigma = 25 / 255
    x, y = synth.denoise_problem(3, 72, sigma, W=56)
    o = ep.Options(subset=ep.SUBSET_REGULAR, subset_param=3)
    xo = oracle.restore(om, y.astype(np.float32).astype(np.float64), sigma, subset=oracle.REGULAR,
                        subset_param=3)
    xg = ep.restore(gm, dev(y), sigma, options=o).cpu().numpy()
    assert abs(psnr(xg, x) - psnr(xo, x)) <= 0.05
    assert np.abs(xg - xo).max() <= 1e-4


@pytest.mark.parametrize("prec", [ep.FP32, ep.BF16X3])
def test_restore_deblur(prec):
    """Periodic deblurring (FFT initialisation and FFT image update): the
    restoration matches the oracle's within the image tolerance 1e-4."""
    gm, om = models(12, "fixed", 8)
    sigma = 2 / 255
    x, k, y = synth.deblur_problem(6, 48, sigma, W=40)
    xo = oracle.restore(om, y.astype(np.float32).astype(np.float64), sigma, deg=oracle.CONV,
                        kernel=k.astype(np.float32).astype(np.float64))
    xg = ep.restore(gm, dev(y), sigma, kind=ep.CONV_PERIODIC, kernel=k,
                    options=ep.Options(precision=prec)).cpu().numpy()
    assert abs(psnr(xg, x) - psnr(xo, x)) <= 0.05
    assert np.abs(xg - xo).max() <= 1e-4


@pytest.mark.parametrize("prec", [ep.FP32, ep.BF16X3])
def test_restore_inpaint(prec):
    """Inpainting (conjugate-gradient initialisation, pixelwise update) on a
    random 1/3 patch subset: within the image tolerance 1e-4 of the oracle."""
    gm, om = models(12, "fixed", 8)
    sigma = 10 / 255
    x, a, y = synth.inpaint_problem(7, 40, sigma, W=48)
    o = ep.Options(cg_iters=100, subset=ep.SUBSET_FRACTION, subset_param=1 / 3, seed=3, precision=prec)
    xo = oracle.restore(om, y.astype(np.float32).astype(np.float64), sigma, deg=oracle.PIXELWISE,
                        a=a, cg_iters=100, subset=oracle.FRACTION, subset_param=1 / 3, seed=3)
    xg = ep.restore(gm, dev(y), sigma, kind=ep.PIXELWISE, a=dev(a), options=o).cpu().numpy()
    assert abs(psnr(xg, x) - psnr(xo, x)) <= 0.05
    assert np.abs(xg - xo).max() <= 1e-4


@pytest.mark.parametrize("H,W,d,sub", [(48, 48, 3, False), (64, 48, 2, True)])
def test_restore_super_resolution(H, W, d, sub):
    """Super-resolution (blur then decimation by d; Sec. "Complexity via
    eigenspace implementation", Fig. 8): the whole restoration, from the
    low-resolution observation, within 1e-4 of the oracle's."""
    gm, om = models(12, "fixed", 8)
    sigma = 2 / 255
    x = synth.image(8, H, W)
    k = synth.gaussian_kernel(9, 1.0)
    yl = (synth.blur_periodic(x, k)[::d, ::d] + synth.noise(8, H // d, W // d, sigma)).astype(np.float32)
    kw = dict(subset=oracle.FRACTION, subset_param=1 / 3, seed=4) if sub else {}
    o = ep.Options(subset=ep.SUBSET_FRACTION, subset_param=1 / 3, seed=4) if sub else ep.Options()
    xo = oracle.restore(om, yl.astype(np.float64), sigma, deg=oracle.SR, kernel=k.astype(np.float32).astype(np.float64),
                        factor=d, **kw)
    xg = ep.restore(gm, dev(yl), sigma, kind=ep.CONV_DECIMATE, kernel=k, factor=d, options=o).cpu().numpy()
    assert xg.shape == (H, W)
    assert abs(psnr(xg, x) - psnr(xo, x)) <= 0.05
    assert np.abs(xg - xo).max() <= 1e-4
    xh = ep.restore_host(gm, yl, sigma, kind=ep.CONV_DECIMATE, kernel=k, factor=d, options=o)
    assert np.abs(xh - xg).max() == 0.0


@pytest.mark.parametrize("kind", ["denoise", "inpaint", "deblur"])
def test_restore_valid_boundary(kind):
    """`valid` boundary (only the patches inside the image; Eq. 6 with the
    per-pixel patch count): denoising and inpainting update pixel by pixel
    with the count weights, deblurring by conjugate gradients on the weighted
    system; within 1e-4 of the oracle."""
    gm, om = models(12, "fixed", 8)
    o = ep.Options(subset=ep.SUBSET_VALID, cg_iters=60)
    kw = dict(subset=oracle.VALID, cg_iters=60)
    if kind == "denoise":
        sigma = 20 / 255
        x, y = synth.denoise_problem(12, 44, sigma, W=37)
        xo = oracle.restore(om, y.astype(np.float32).astype(np.float64), sigma, **kw)
        xg = ep.restore(gm, dev(y), sigma, options=o).cpu().numpy()
    elif kind == "inpaint":
        sigma = 10 / 255
        x, a, y = synth.inpaint_problem(13, 40, sigma, W=33)
        xo = oracle.restore(om, y.astype(np.float32).astype(np.float64), sigma, deg=oracle.PIXELWISE, a=a, **kw)
        xg = ep.restore(gm, dev(y), sigma, kind=ep.PIXELWISE, a=dev(a), options=o).cpu().numpy()
    else:
        sigma = 5 / 255
        x, k, y = synth.deblur_problem(14, 40, sigma, W=36, size=9, sigma_b=1.0)
        k = k.astype(np.float32)
        xo = oracle.restore(om, y.astype(np.float32).astype(np.float64), sigma, deg=oracle.CONV,
                            kernel=k.astype(np.float64), **kw)
        xg = ep.restore(gm, dev(y), sigma, kind=ep.CONV_PERIODIC, kernel=k, options=o).cpu().numpy()
    assert abs(psnr(xg, x) - psnr(xo, x)) <= 0.05
    assert np.abs(xg - xo).max() <= 1e-4


def test_restore_inpaint_ragged_large():
    """A larger, ragged inpainting problem (the CG splits unevenly over its
    CTAs), K = 20 at full rank, every patch."""
    gm, om = models(20)
    sigma = 15 / 255
    x, a, y = synth.inpaint_problem(9, 97, sigma, W=131)
    xo = oracle.restore(om, y.astype(np.float32).astype(np.float64), sigma, beta_mult=(1, 4, 8),
                        deg=oracle.PIXELWISE, a=a, cg_iters=100)
    xg = ep.restore(gm, dev(y), sigma, beta_mult=(1, 4, 8), kind=ep.PIXELWISE, a=dev(a),
                    options=ep.Options(cg_iters=100)).cpu().numpy()
    assert np.abs(xg - xo).max() <= 1e-4


def test_invalid_arguments():
    gm, _ = models(3)
    y = dev(np.zeros((16, 16)))
    with pytest.raises(ep.EpllError) as e:
        ep.restore(gm, dev(np.zeros((4, 16))), 0.1)
    assert e.value.status == ep.EINVAL
    with pytest.raises(ep.EpllError):
        ep.restore(gm, y, -1.0)
    with pytest.raises(ep.EpllError):
        ep.restore(gm, y, 0.1, options=ep.Options(subset=ep.SUBSET_JITTER, subset_param=9))
    with pytest.raises(ep.EpllError):
        ep.restore(gm, y, 0.1, kind=ep.PIXELWISE)
