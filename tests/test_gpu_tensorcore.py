"""Parity of the tcgen05 selection path (BF16, FP16, split BF16) against the
FP64 oracle, through the C ABI.

Selection must match the oracle wherever the oracle's top-2 gap is >= 1e-4
(near-ties in the reduced precision are rescored in compensated FP32), and
the reported gap of every patch must be within the precision's error bound
of the oracle's gap.
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
REL = {ep.BF16: 1e-2, ep.FP16: 1.5e-3, ep.BF16X3: 1e-4, ep.FP8: 1e-1, ep.AUTO: 1.5e-3}
PRECS = [ep.BF16X3, ep.FP16, ep.BF16, ep.FP8, ep.AUTO]


@pytest.fixture(scope="module", autouse=True)
def _built():
    ep.build()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")


def tmax(S, r, lam, beta):
    ib = 1.0 / beta
    return max((1.0 / (lam[k] + ib)) if r[k] < 64 else 1.0 / (S[k, -1] + ib) for k in range(len(r)))


def check(gm, om, g, x, beta, prec, subset=ep.SUBSET_ALL, param=0.0, t=0):
    o = ep.Options(precision=prec, subset=subset, subset_param=param, seed=17)
    xt, an, ks, gp = ep.patch_step(gm, dev(x), beta, o, t)
    xt, an, ks, gp = (v.cpu().numpy() for v in (xt, an, ks, gp))
    x64 = x.astype(np.float32).astype(np.float64)
    oxt, oks, ogap, _ = oracle.patch_step(om, beta, x64, an)
    bad = (ks != oks) & (ogap >= TIE)
    assert not bad.any(), f"prec {prec}: {bad.sum()} disagreements, oracle gaps {ogap[bad][:5]}"
    # gaps: within the error bound of the arithmetic (rescored patches are exact)
    H, W = x.shape
    zz = np.array([np.var(x64[np.ix_((np.arange(8) + a // W) % H, (np.arange(8) + a % W) % W)]) * 64
                   for a in an])
    bound = 2e-3 + 2 * REL[prec] * zz * tmax(g.S, om.r, om.lam, beta)
    fin = np.isfinite(ogap) & (ogap < 1e30)
    assert np.all(np.abs(gp[fin] - ogap[fin]) <= bound[fin] + 1e-4 * np.abs(ogap[fin]))
    if np.array_equal(ks, oks):
        np.testing.assert_allclose(xt, oxt, atol=1e-5, rtol=0)
    return ks, oks


@pytest.mark.parametrize("prec", PRECS)
def test_single_tile_full_rank(prec):
    """One CTA (< 128 patches), K = 20 full rank: the smallest tensor-core case."""
    g = synth.synthetic_gmm(20)
    gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_FIXED, 64)
    om = oracle.Model(g.w, g.U, g.S, "fixed", 64)
    sigma = 20 / 255
    x = synth.image(0, 8, 12) + synth.noise(0, 8, 12, sigma)
    check(gm, om, g, x, 1 / sigma ** 2, prec)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("r", [64, 8, 16])
def test_many_tiles_ragged_tail(prec, r):
    """Several M tiles plus a ragged last tile; K*r not a multiple of the N tile."""
    K = 37
    g = synth.synthetic_gmm(K)
    gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_FIXED, r)
    om = oracle.Model(g.w, g.U, g.S, "fixed", r)
    sigma = 25 / 255
    x = synth.image(1, 40, 29) + synth.noise(1, 40, 29, sigma)
    for m in (1, 32):
        check(gm, om, g, x, m / sigma ** 2, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_ragged_ranks_rho(prec):
    g = synth.tiny_gmm(23, seed=41)
    gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_RHO, 0.9)
    om = oracle.Model(g.w, g.U, g.S, "rho", 0.9)
    assert len(set(om.r.tolist())) > 1
    x = synth.image(2, 33, 35) + synth.noise(2, 33, 35, 0.05)
    check(gm, om, g, x, 1 / 0.0004, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_k200_subset(prec):
    """The FEPLL configuration's model (K = 200) on a 1/3 subset of a 96x96 image."""
    g = synth.synthetic_gmm(200)
    for r in (8, 64):
        gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_FIXED, r)
        om = oracle.Model(g.w, g.U, g.S, "fixed", r)
        sigma = 25 / 255
        x = synth.image(3, 96) + synth.noise(3, 96, 96, sigma)
        check(gm, om, g, x, 8 / sigma ** 2, prec, ep.SUBSET_FRACTION, 1 / 3)


@pytest.mark.parametrize("prec", PRECS)
def test_restore_matches_oracle_psnr(prec):
    g = synth.synthetic_gmm(200)
    gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_FIXED, 8)
    om = oracle.Model(g.w, g.U, g.S, "fixed", 8)
    sigma = 25 / 255
    x, y = synth.denoise_problem(4, 64, sigma)
    o = ep.Options(precision=prec, subset=ep.SUBSET_FRACTION, subset_param=1 / 3, seed=2)
    xo = oracle.restore(om, y.astype(np.float32).astype(np.float64), sigma, subset=oracle.FRACTION,
                        subset_param=1 / 3, seed=2)
    xg = ep.restore(gm, dev(y), sigma, options=o).cpu().numpy()
    ep.last_counters(gm)  # raises if a bounded device wait gave up
    ps = lambda a: -10 * math.log10(np.mean((a - x) ** 2))
    assert abs(ps(xg) - ps(xo)) <= 0.05
    evals, rescored, launches = ep.last_counters(gm)
    assert evals == 5 * math.ceil(64 * 64 / 3) and launches > 0


def test_fp8_deblur_matches_oracle_psnr():
    """The FEPLL deblurring configuration in miniature: periodic 25x25 Gaussian
    blur (sigma_b = 1.6), sigma = 2/255, K = 200, r = 8, E4M3 selection."""
    g = synth.synthetic_gmm(200)
    gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_FIXED, 8)
    om = oracle.Model(g.w, g.U, g.S, "fixed", 8)
    sigma = 2 / 255
    x, k, y = synth.deblur_problem(8, 64, sigma)
    xo = oracle.restore(om, y.astype(np.float32).astype(np.float64), sigma, deg=oracle.CONV,
                        kernel=k.astype(np.float32).astype(np.float64))
    xg = ep.restore(gm, dev(y), sigma, kind=ep.CONV_PERIODIC, kernel=k,
                    options=ep.Options(precision=ep.FP8)).cpu().numpy()
    ep.last_counters(gm)
    ps = lambda a: -10 * math.log10(np.mean((a - x) ** 2))
    assert abs(ps(xg) - ps(xo)) <= 0.05
