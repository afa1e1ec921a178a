"""Selection down the balanced search tree through the C ABI, against the
FP64 tree oracle (descent over the same node Gaussians)."""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import tree as otree

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1710_08124_gb300 as ep  # noqa: E402
from paper_1710_08124_gb300 import tree as ptree  # noqa: E402

TIE = 1e-4
SPLIT_REL = 4e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    ep.build()


def dev(a, dtype=np.float32):
    return torch.as_tensor(np.ascontiguousarray(a, dtype), device="cuda")


def setup(K, r):
    g = synth.synthetic_gmm(K)
    T = ptree.build_tree(g.w, g.U, g.S)
    gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_FIXED, r)
    ep.attach_tree(gm, T)
    om_nodes = oracle.Model(T.weights, T.eigvecs, T.eigvals, "fixed", r)
    om = oracle.Model(g.w, g.U, g.S, "fixed", r)
    return g, T, gm, om, om_nodes


def oracle_descent(om_nodes, T, beta, x, anchors):
    sc = oracle.scores(om_nodes, beta, x.astype(np.float64), anchors)
    leaf, gap = otree.descend(sc, T.child_begin)
    return T.leaf_component[leaf], gap


def node_tmax(om_nodes, beta):
    ib = 1.0 / beta
    return max((1.0 / (om_nodes.lam[k] + ib)) if om_nodes.r[k] < 64 else 1.0 / (om_nodes.S[k, -1] + ib)
               for k in range(len(om_nodes.r)))


def check_descent(gm, om, om_nodes, T, x, beta, opts):
    xt, an, ks, gp = ep.patch_step(gm, dev(x), beta, opts)
    ep.last_counters(gm)
    xt, an, ks, gp = (v.cpu().numpy() for v in (xt, an, ks, gp))
    ko, go = oracle_descent(om_nodes, T, beta, x, an)
    H, W = x.shape
    x64 = x.astype(np.float64)
    zz = np.array([np.var(x64[np.ix_((np.arange(8) + a // W) % H, (np.arange(8) + a % W) % W)]) * 64 for a in an])
    band = TIE + 2 * SPLIT_REL * zz * node_tmax(om_nodes, beta)
    bad = (ks != ko) & (go >= band)
    assert not bad.any(), f"{bad.sum()} disagreements outside the split-BF16 band, oracle gaps {go[bad][:5]}"
    # the estimates are those of the oracle forced to the same selection
    oxt, _, _, _ = oracle.patch_step(om, beta, x64, an, forced_k=ks)
    np.testing.assert_allclose(xt, oxt, atol=1e-5, rtol=0)
    return ks, ko


@pytest.mark.parametrize("r", [64, 8])
def test_descent_matches_oracle_k40(r):
    g, T, gm, om, om_nodes = setup(40, r)
    sigma = 25 / 255
    x = (synth.image(20, 48, 56) + synth.noise(20, 48, 56, sigma)).astype(np.float32)
    for m in (1, 16):
        ks, ko = check_descent(gm, om, om_nodes, T, x, m / sigma ** 2, ep.Options(select=ep.SELECT_TREE))
        assert np.mean(ks == ko) > 0.99


def test_descent_matches_oracle_k200_subset():
    """The paper's tree shape (327 nodes, 7 levels) on a 1/3 subset."""
    g, T, gm, om, om_nodes = setup(200, 64)
    assert T.n_nodes == 327
    sigma = 25 / 255
    x = (synth.image(21, 96) + synth.noise(21, 96, 96, sigma)).astype(np.float32)
    opts = ep.Options(select=ep.SELECT_TREE, subset=ep.SUBSET_FRACTION, subset_param=1 / 3, seed=5)
    check_descent(gm, om, om_nodes, T, x, 8 / sigma ** 2, opts)


def test_single_level_tree_is_exhaustive():
    """A root whose children are all the components is the exhaustive argmin."""
    g = synth.synthetic_gmm(4)
    T = ptree.build_tree(g.w, g.U, g.S)
    assert T.depth == 1 and T.n_nodes == 5
    gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_FIXED, 64)
    ep.attach_tree(gm, T)
    om = oracle.Model(g.w, g.U, g.S, "fixed", 64)
    sigma = 20 / 255
    x = (synth.image(22, 40) + synth.noise(22, 40, 40, sigma)).astype(np.float32)
    beta = 4 / sigma ** 2
    _, an, ks, _ = ep.patch_step(gm, dev(x), beta, ep.Options(select=ep.SELECT_TREE))
    _, oks, ogap, _ = oracle.patch_step(om, beta, x.astype(np.float64), an.cpu().numpy())
    ks = ks.cpu().numpy()
    assert np.all((ks == oks) | (ogap < TIE + 1e-2))
    assert np.mean(ks == oks) > 0.999


def test_tree_restore_matches_oracle():
    g, T, gm, om, om_nodes = setup(40, 8)
    sigma = 25 / 255
    x, y = synth.denoise_problem(23, 64, sigma)
    y32 = y.astype(np.float32)
    beta_mult = (1.0, 4.0, 8.0, 16.0, 32.0)
    lam = oracle.lam(oracle.DENOISE, 64, 64, sigma)
    xo = y32.astype(np.float64)
    for t, m in enumerate(beta_mult):
        beta = lam * m / sigma ** 2
        an = oracle.sample(64, 64, oracle.FRACTION, 1 / 3, seed=3, t=t)
        k, _ = oracle_descent(om_nodes, T, beta, xo, an)
        xt, _, _, _ = oracle.patch_step(om, beta, xo, an, forced_k=k)
        xo = oracle.xupdate_pixelwise(y32.astype(np.float64), xt, lam * m)
    opts = ep.Options(select=ep.SELECT_TREE, subset=ep.SUBSET_FRACTION, subset_param=1 / 3, seed=3)
    xg = ep.restore(gm, dev(y32), sigma, beta_mult, options=opts).cpu().numpy()
    ep.last_counters(gm)
    ps = lambda a: -10 * math.log10(np.mean((a - x) ** 2))
    assert abs(ps(xg) - ps(xo)) <= 0.05


def test_tree_batch_graph_equals_sequential():
    g, T, gm, om, om_nodes = setup(40, 8)
    jobs, outs = [], []
    for i, side in enumerate((64, 96, 40)):
        _, y = synth.denoise_problem(30 + i, side, 20 / 255)
        yd = dev(y)
        jobs.append((yd, torch.empty_like(yd), None, ep.DENOISE, 20 / 255))
    opts = ep.Options(select=ep.SELECT_TREE, subset=ep.SUBSET_FRACTION, subset_param=1 / 3, seed=1)
    ep.restore_batch(gm, jobs, options=opts, mode=ep.BATCH_GRAPH, lanes=2)
    torch.cuda.synchronize()
    a = [j[1].cpu().numpy().copy() for j in jobs]
    ep.restore_batch(gm, jobs, options=opts, mode=ep.BATCH_SEQUENTIAL)
    torch.cuda.synchronize()
    for u, j in zip(a, jobs):
        np.testing.assert_array_equal(u, j[1].cpu().numpy())


def test_invalid_trees_are_rejected():
    g = synth.synthetic_gmm(20)
    T = ptree.build_tree(g.w, g.U, g.S)
    gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_FIXED, 8)
    with pytest.raises(ep.EpllError):
        ep.patch_step(gm, dev(synth.image(0, 16)), 100.0, ep.Options(select=ep.SELECT_TREE))
    bad = ptree.Tree(T.weights, T.eigvecs, T.eigvals, T.child_begin.copy(), T.leaf_component.copy(), T.levels)
    bad.leaf_component[-1] = bad.leaf_component[-2]  # a component twice
    with pytest.raises(ep.EpllError):
        ep.attach_tree(gm, bad)
    bad2 = ptree.Tree(T.weights, T.eigvecs, T.eigvals, T.child_begin.copy(), T.leaf_component.copy(), T.levels)
    bad2.child_begin[0] = 2  # root's first child not node 1
    with pytest.raises(ep.EpllError):
        ep.attach_tree(gm, bad2)
    ep.attach_tree(gm, T)
    ep.attach_tree(gm, None)
    with pytest.raises(ep.EpllError):
        ep.patch_step(gm, dev(synth.image(0, 16)), 100.0, ep.Options(select=ep.SELECT_TREE))


@pytest.mark.parametrize("K", [5, 7])
def test_small_trees_and_ragged_ranks(K):
    """Small models (two levels, clusters of 2-3) with rho-mode ragged ranks
    (children with different column counts) on a jittered subset."""
    g = synth.tiny_gmm(K, seed=50 + K)
    T = ptree.build_tree(g.w, g.U, g.S)
    gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_RHO, 0.9)
    ep.attach_tree(gm, T)
    om = oracle.Model(g.w, g.U, g.S, "rho", 0.9)
    om_nodes = oracle.Model(T.weights, T.eigvecs, T.eigvals, "rho", 0.9)
    sigma = 15 / 255
    x = (synth.image(40 + K, 33, 35) + synth.noise(40 + K, 33, 35, sigma)).astype(np.float32)
    opts = ep.Options(select=ep.SELECT_TREE, subset=ep.SUBSET_JITTER, subset_param=4, seed=9)
    check_descent(gm, om, om_nodes, T, x, 4 / sigma ** 2, opts)


def test_tree_deblur_restore_runs_and_matches_forced_oracle_step():
    """Periodic deblurring with the tree selection: the run is error-free and its
    first patch step equals the oracle's descent on the same estimate."""
    g, T, gm, om, om_nodes = setup(40, 8)
    sigma = 2 / 255
    x, k, y = synth.deblur_problem(24, 64, sigma)
    xg = ep.restore(gm, dev(y), sigma, kind=ep.CONV_PERIODIC, kernel=k,
                    options=ep.Options(select=ep.SELECT_TREE)).cpu().numpy()
    ep.last_counters(gm)
    assert np.all(np.isfinite(xg))
    check_descent(gm, om, om_nodes, T, xg, 16 * oracle.lam(oracle.CONV, 64, 64, sigma, kernel=k) / sigma ** 2,
                  ep.Options(select=ep.SELECT_TREE))
