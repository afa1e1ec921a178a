"""The candidate step of the FP16 selection form (FP16, and AUTO at rank 64),
through the C ABI; BF16 (one-term pass, then the split pass) alongside.

The FP16 pass keeps each patch's four best components; a patch it cannot
decide has the components within its error bound rescored in the split form
(grouped by component), and a patch whose band may hold more than four
components goes to the compensated rescoring.  Models with exact duplicates force both branches on every patch:
the selected component must then be one of the minimisers of the oracle's
scores (Eq. 14), and the patch estimate the oracle's for that component.
"""
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
FORMS = [ep.FP16, ep.BF16, ep.AUTO]


@pytest.fixture(scope="module", autouse=True)
def _built():
    ep.build()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")


def duplicated(K, copies, seed=11):
    """A synthetic GMM whose components 1 .. copies-1 repeat component 0."""
    g = synth.synthetic_gmm(K, seed=seed)
    w, U, S = g.w.copy(), g.U.copy(), g.S.copy()
    for c in range(1, copies):
        U[c], S[c], w[c] = U[0], S[0], w[0]
    return w / w.sum(), U, S


def check_minimisers(w, U, S, r, prec, beta, x):
    gm = ep.gmm_load(w, U, S, ep.RANK_FIXED, r)
    om = oracle.Model(w, U, S, "fixed", r)
    o = ep.Options(precision=prec, subset=ep.SUBSET_FRACTION, subset_param=0.5, seed=5)
    xt, an, ks, gp = ep.patch_step(gm, dev(x), beta, o, 0)
    ep.last_counters(gm)
    an, ks = an.cpu().numpy(), ks.cpu().numpy()
    x64 = x.astype(np.float32).astype(np.float64)
    sc = oracle.scores(om, beta, x64, an)
    best = sc.min(1)
    mine = sc[np.arange(len(an)), ks]
    assert np.all(mine - best <= TIE + 1e-9 * np.abs(best)), np.max(mine - best)
    # the estimate of each patch is the oracle's for the selected component
    oxt, _, _, _ = oracle.patch_step(om, beta, x64, an, forced_k=ks)
    np.testing.assert_allclose(xt.cpu().numpy(), oxt, atol=1e-5, rtol=0)
    return ks


@pytest.mark.parametrize("prec", FORMS)
def test_exact_ties_within_four(prec):
    """Three copies of one component: every patch that prefers it has an
    exact three-way tie, inside the four candidates."""
    w, U, S = duplicated(12, 3)
    sigma = 25 / 255
    x = synth.image(21, 48) + synth.noise(21, 48, 48, sigma)
    ks = check_minimisers(w, U, S, 64, prec, 4 / sigma ** 2, x)
    # among exact copies the lowest index wins
    assert not np.isin(ks, [1, 2]).any()


@pytest.mark.parametrize("prec", FORMS)
def test_band_overflow(prec):
    """Six copies of one component: the band holds more than four components
    and those patches go to the compensated rescoring."""
    w, U, S = duplicated(16, 6)
    sigma = 25 / 255
    x = synth.image(22, 40, 56) + synth.noise(22, 40, 56, sigma)
    ks = check_minimisers(w, U, S, 64, prec, 8 / sigma ** 2, x)
    assert (ks == 0).any() and not np.isin(ks, [1, 2, 3, 4, 5]).any()


@pytest.mark.parametrize("K", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("prec", [ep.FP16, ep.BF16])
def test_few_components(K, prec):
    """K <= 4 leaves empty candidate slots; K = 5 just fills them."""
    g = synth.synthetic_gmm(K, seed=3)
    sigma = 20 / 255
    x = synth.image(23, 24, 40) + synth.noise(23, 24, 40, sigma)
    check_minimisers(g.w, g.U, g.S, 64, prec, 2 / sigma ** 2, x)


@pytest.mark.parametrize("r", [64, 8, 16])
def test_one_term_ranks_match_split(r):
    """At every uniform rank the FP16 form selects what the split form does
    wherever the oracle's top-2 gap is clear."""
    g = synth.synthetic_gmm(200)
    gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_FIXED, r)
    om = oracle.Model(g.w, g.U, g.S, "fixed", r)
    sigma = 25 / 255
    x = synth.image(24, 64) + synth.noise(24, 64, 64, sigma)
    beta = 16 / sigma ** 2
    out = {}
    for prec in (ep.BF16X3, ep.FP16):
        o = ep.Options(precision=prec, subset=ep.SUBSET_FRACTION, subset_param=1 / 3, seed=9)
        _, an, ks, _ = ep.patch_step(gm, dev(x), beta, o, 2)
        out[prec] = (an.cpu().numpy(), ks.cpu().numpy())
    assert np.array_equal(out[ep.BF16X3][0], out[ep.FP16][0])
    an = out[ep.FP16][0]
    _, oks, ogap, _ = oracle.patch_step(om, beta, x.astype(np.float32).astype(np.float64), an)
    clear = ogap >= TIE
    assert np.array_equal(out[ep.FP16][1][clear], oks[clear])
    assert np.array_equal(out[ep.BF16X3][1][clear], oks[clear])


@pytest.mark.parametrize("prec", [ep.FP16, ep.AUTO])
def test_many_tiles_per_cta(prec):
    """Every patch of a 256x256 image: 512 tiles of 128 patches, so each
    persistent CTA of the FP16 pass takes three or four tiles; the selection
    must match the oracle's."""
    g = synth.synthetic_gmm(12, seed=5)
    gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_FIXED, 64)
    om = oracle.Model(g.w, g.U, g.S, "fixed", 64)
    sigma = 15 / 255
    x = synth.image(25, 256) + synth.noise(25, 256, 256, sigma)
    beta = 4 / sigma ** 2
    xt, an, ks, gp = ep.patch_step(gm, dev(x), beta, ep.Options(precision=prec), 0)
    ep.last_counters(gm)
    an, ks = an.cpu().numpy(), ks.cpu().numpy()
    assert len(an) == 256 * 256
    x64 = x.astype(np.float32).astype(np.float64)
    oxt, oks, ogap, _ = oracle.patch_step(om, beta, x64, an)
    bad = (ks != oks) & (ogap >= TIE)
    assert not bad.any(), f"{bad.sum()} disagreements"
    if np.array_equal(ks, oks):
        np.testing.assert_allclose(xt.cpu().numpy(), oxt, atol=1e-5, rtol=0)
