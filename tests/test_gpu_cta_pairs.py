"""The selection's first pass in its other launch forms against the default
one (one CTA per MMA, 256-column basis tiles) and the FP64 oracle, through
the C ABI: CTA pairs (tcgen05 cta_group::2: 256 patch rows per pair, each CTA
holding half of every basis tile) and 128-column basis tiles (four
accumulator buffers; at rank 64 two sets of epilogue warps on alternate
buffers).

Neither form changes the sums: each accumulator of Eq. 14's projections is
the same products added in the same order.  So the selections, gaps and
patch estimates must equal those of the default form, and the selection must
match the oracle wherever the oracle's top-2 gap is >= 1e-4.  The shapes cover one pair whose second CTA holds no
patch (n < 128), one partly filled pair, several 256-row tiles with a ragged
tail, ragged ranks (flat tail, rho rule), and the FEPLL size (512 x 512,
K = 200, 1/3 subset: 87,382 patches, several tiles per pair).
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
PRECS = [ep.BF16X3, ep.FP16, ep.BF16, ep.AUTO]


@pytest.fixture(scope="module", autouse=True)
def _built():
    ep.build()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")


def step(gm, x, beta, prec, pair, subset=ep.SUBSET_ALL, param=0.0, bn=256):
    ep.set_cta_pairs(gm, pair)
    ep.set_tiles(gm, bn, 1)
    o = ep.Options(precision=prec, subset=subset, subset_param=param, seed=17)
    out = [v.cpu().numpy() for v in ep.patch_step(gm, dev(x), beta, o, 0)]
    ep.last_counters(gm)  # raises if a bounded device wait gave up
    return out


def compare(gm, om, x, beta, prec, subset=ep.SUBSET_ALL, param=0.0, bn=256):
    """The default form against pairs (bn = 256) or 128-column tiles (bn = 128)."""
    xt1, an1, ks1, gp1 = step(gm, x, beta, prec, False, subset, param)
    xt2, an2, ks2, gp2 = step(gm, x, beta, prec, bn == 256, subset, param, bn)
    assert np.array_equal(an1, an2)
    assert np.array_equal(ks1, ks2), f"{(ks1 != ks2).sum()} selections differ"
    assert np.array_equal(gp1, gp2)
    assert np.array_equal(xt1, xt2)
    if om is not None:
        x64 = x.astype(np.float32).astype(np.float64)
        _, oks, ogap, _ = oracle.patch_step(om, beta, x64, an2)
        bad = (ks2 != oks) & (ogap >= TIE)
        assert not bad.any(), f"{bad.sum()} disagreements with the oracle, gaps {ogap[bad][:5]}"


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", [(8, 12), (13, 15), (40, 29)])
@pytest.mark.parametrize("r", [64, 8])
def test_pairs_equal_single_cta(prec, shape, r):
    """96 patches (the pair's second CTA reads only out-of-range rows), 195
    (a partly filled pair), 1160 (five 256-row tiles, the last ragged)."""
    g = synth.synthetic_gmm(37)
    gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_FIXED, r)
    om = oracle.Model(g.w, g.U, g.S, "fixed", r)
    sigma = 25 / 255
    H, W = shape
    x = synth.image(1, H, W) + synth.noise(1, H, W, sigma)
    compare(gm, om, x, 4 / sigma ** 2, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_pairs_ragged_ranks(prec):
    g = synth.tiny_gmm(23, seed=41)
    gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_RHO, 0.9)
    om = oracle.Model(g.w, g.U, g.S, "rho", 0.9)
    assert len(set(om.r.tolist())) > 1
    x = synth.image(2, 33, 35) + synth.noise(2, 33, 35, 0.05)
    compare(gm, om, x, 1 / 0.0004, prec)


@pytest.mark.parametrize("r", [64, 8])
def test_pairs_fepll_size(r):
    """512 x 512, K = 200, 1/3 subset, AUTO (FP16 pass at r = 64, split BF16 at
    r = 8): every pair takes several tiles of the persistent loop."""
    g = synth.synthetic_gmm(200)
    gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_FIXED, r)
    sigma = 25 / 255
    x = synth.image(3, 512) + synth.noise(3, 512, 512, sigma)
    compare(gm, None, x, 8 / sigma ** 2, ep.AUTO, ep.SUBSET_FRACTION, 1 / 3)


def test_pairs_restore_and_batch():
    """Whole restorations: pairs on and off give the same image, and a batch
    of uneven images under the captured graph equals the per-image calls."""
    g = synth.synthetic_gmm(37)
    gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_FIXED, 64)
    o = ep.Options(precision=ep.AUTO, subset=ep.SUBSET_FRACTION, subset_param=1 / 3, seed=4)
    probs = [synth.denoise_problem(30 + i, H, s, W=W)
             for i, (H, W, s) in enumerate([(64, 48, 0.1), (40, 72, 0.05), (96, 96, 0.2)])]
    outs = {}
    for pair in (False, True):
        ep.set_cta_pairs(gm, pair)
        outs[pair] = [ep.restore(gm, dev(y), s, options=o).cpu().numpy()
                      for (_, y), s in zip(probs, (0.1, 0.05, 0.2))]
        ep.last_counters(gm)
    for a, b in zip(outs[False], outs[True]):
        assert np.array_equal(a, b)
    jobs = [(dev(y), torch.empty(y.shape, device="cuda"), None, ep.DENOISE, s)
            for (_, y), s in zip(probs, (0.1, 0.05, 0.2))]
    for rep in range(2):  # capture, then replay
        ep.restore_batch(gm, jobs, options=o, mode=ep.BATCH_GRAPH, lanes=2)
        torch.cuda.synchronize()
        for j, ref in zip(jobs, outs[True]):
            assert np.array_equal(j[1].cpu().numpy(), ref), rep
    ep.last_counters(gm)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("r", [64, 8])
def test_tiles_128_equal_256(prec, r):
    """128-column basis tiles (at r = 64 two epilogue warp sets on alternate
    accumulator buffers) on several tiles with a ragged tail, and at the FEPLL
    size."""
    g = synth.synthetic_gmm(37)
    gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_FIXED, r)
    om = oracle.Model(g.w, g.U, g.S, "fixed", r)
    sigma = 25 / 255
    x = synth.image(1, 40, 29) + synth.noise(1, 40, 29, sigma)
    compare(gm, om, x, 4 / sigma ** 2, prec, bn=128)
    g = synth.synthetic_gmm(200)
    gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_FIXED, r)
    x = synth.image(3, 512) + synth.noise(3, 512, 512, sigma)
    compare(gm, None, x, 8 / sigma ** 2, prec, ep.SUBSET_FRACTION, 1 / 3, bn=128)
