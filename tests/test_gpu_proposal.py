"""The learned top-m proposal through the C ABI: training gradients and
inference against the FP64 network oracle, the exactness of the proposal
selection against the FP64 selection oracle, and what a trained network gains.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import mlp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1710_08124_gb300 as ep  # noqa: E402
from paper_1710_08124_gb300 import proposal as pr  # noqa: E402

TIE = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    ep.build()


def dev(a, dtype=np.float32):
    return torch.as_tensor(np.ascontiguousarray(a, dtype), device="cuda")


def random_params(K, seed, scale=0.1):
    rng = np.random.default_rng(seed)
    th = rng.standard_normal(mlp.n_params(K)) * scale
    p = mlp.unpack(th, K)
    p["W1"] *= 4.0  # patches are small numbers: give the first layer some gain
    return mlp.pack(p, K).astype(np.float32)


@pytest.mark.parametrize("K,B", [(20, 257), (200, 1000)])
def test_gradient_matches_oracle(K, B):
    """Forward + backward of the mean cross-entropy against the FP64 oracle
    evaluated at the same (BF16-rounded) weights; with and without a sample
    index list."""
    rng = np.random.default_rng(K)
    H, W = 40, 48
    ims = np.stack([synth.image(i, H, W) + synth.noise(i, H, W, 0.05) for i in range(3)]).astype(np.float32)
    n_all = B + 37
    img_idx = rng.integers(0, 3, n_all).astype(np.int32)
    anchors = rng.integers(0, H * W, n_all).astype(np.int32)
    log_ib = rng.uniform(math.log(1e-5), math.log(1e-1), n_all).astype(np.float32)
    labels = rng.integers(0, K, n_all).astype(np.int32)
    theta = random_params(K, 100 + K)
    p = ep.Proposal(K, seed=1)
    p.set(theta)
    np.testing.assert_array_equal(p.get(), theta)
    q = mlp.round_weights(mlp.unpack(theta.astype(np.float64), K))
    sel = rng.permutation(n_all)[:B].astype(np.int32)
    for use_sel in (False, True):
        s = sel if use_sel else np.arange(B, dtype=np.int32)
        X = mlp.inputs(ims.astype(np.float64), H, W, img_idx[s], anchors[s], log_ib[s].astype(np.float64))
        L, g = mlp.loss_and_grad(q, X, log_ib[s].astype(np.float64), labels[s])
        if use_sel:
            gg, loss = p.grad(dev(ims), dev(img_idx, np.int32), dev(anchors, np.int32), dev(log_ib),
                              dev(labels, np.int32), sel=dev(sel, np.int32))
        else:
            gg, loss = p.grad(dev(ims), dev(img_idx[:B], np.int32), dev(anchors[:B], np.int32), dev(log_ib[:B]),
                              dev(labels[:B], np.int32))
        assert abs(loss - L) <= 1e-5 * abs(L)
        gv = mlp.unpack(gg.cpu().numpy().astype(np.float64), K)
        for name in g:
            err = np.abs(gv[name] - g[name]).max()
            assert err <= 1e-4 * np.abs(g[name]).max() + 1e-9, (name, err, np.abs(g[name]).max())


def test_adamw_steps_match_oracle():
    """Three AdamW steps through epll_proposal_train against the oracle's
    AdamW (decoupled decay on W1, W2, W3, bias-corrected moments), each step
    on the oracle's own gradient at its own BF16-rounded weights.  Where a
    parameter's gradient is not tiny (|g| >= 1e-2 of its block's largest, so
    that the normalised step does not amplify the gradient's FP32 rounding),
    the moved parameters agree within 2 % of one step length plus FP32
    rounding; a missing bias correction or a decay folded into the gradient
    moves them by more than 10 % of a step length (pinned on the CPU)."""
    K, B, H, W = 20, 256, 40, 48
    rng = np.random.default_rng(77)
    ims = np.stack([synth.image(i, H, W) + synth.noise(i, H, W, 0.05) for i in range(2)]).astype(np.float32)
    img_idx = rng.integers(0, 2, B).astype(np.int32)
    anchors = rng.integers(0, H * W, B).astype(np.int32)
    log_ib = rng.uniform(math.log(1e-4), math.log(1e-2), B).astype(np.float32)
    labels = rng.integers(0, K, B).astype(np.int32)
    theta = random_params(K, 5)
    lr, wd = 1e-3, 2.0
    net = ep.Proposal(K, seed=1)
    net.set(theta)
    X = mlp.inputs(ims.astype(np.float64), H, W, img_idx, anchors, log_ib.astype(np.float64))
    cond = log_ib.astype(np.float64)
    q = mlp.unpack(theta.astype(np.float64), K)
    m = {k: np.zeros_like(v) for k, v in q.items()}
    v = {k: np.zeros_like(x) for k, x in q.items()}
    args = (dev(ims), dev(img_idx, np.int32), dev(anchors, np.int32), dev(log_ib), dev(labels, np.int32))
    big = None
    for t in (1, 2, 3):
        _, g = mlp.loss_and_grad(mlp.round_weights(q), X, cond, labels)
        if big is None:
            big = {k: np.abs(g[k]) >= 1e-2 * np.abs(g[k]).max() for k in g}
        q, m, v = mlp.adamw_step(q, g, m, v, t, lr, wd)
        net.train_step(*args, lr=lr, weight_decay=wd, want_loss=False)
        got = mlp.unpack(net.get().astype(np.float64), K)
        for k in q:
            d = np.abs(got[k] - q[k])[big[k]]
            tol = 0.02 * lr * t + 4 * 2.0 ** -24 * t * np.abs(q[k]).max()
            assert d.max() <= tol, (k, t, d.max(), tol)
    assert np.mean(np.concatenate([b.ravel() for b in big.values()])) > 0.2


def test_invalid_samples_are_reported():
    K, H, W = 20, 16, 16
    p = ep.Proposal(K, seed=2)
    ims = dev(np.zeros((1, H, W)))
    ok = dict(img_idx=dev([0, 0], np.int32), anchors=dev([0, 5], np.int32), log_ib=dev([0.0, 0.0]),
              labels=dev([1, 2], np.int32))
    for key, badv in (("img_idx", [0, 1]), ("anchors", [0, H * W]), ("labels", [K, 0]), ("labels", [-1, 0])):
        args = dict(ok)
        args[key] = dev(badv, np.int32)
        with pytest.raises(ep.EpllError):
            p.grad(ims, args["img_idx"], args["anchors"], args["log_ib"], args["labels"])
    p.grad(ims, **ok)  # the flag does not stick


def test_topm_matches_oracle_inference_form():
    """cand / pmass of the tensor-core inference kernels against the FP64
    inference form (BF16 patch and activations): every proposal is a top-m
    logit up to the rounding tolerance, and the mass matches."""
    K, m = 200, 8
    g = synth.synthetic_gmm(K)
    gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_FIXED, 8)
    theta = random_params(K, 7)
    p = ep.Proposal(K, seed=3)
    p.set(theta)
    ep.attach_proposal(gm, p, topm=m)
    sigma = 25 / 255
    H, W = 72, 40  # 2880 patches: 22 full tiles and a ragged one
    x = (synth.image(5, H, W) + synth.noise(5, H, W, sigma)).astype(np.float32)
    beta = 4 / sigma ** 2
    cand, pmass = ep.proposal_topm(gm, dev(x), beta)
    ep.last_counters(gm)
    cand, pmass = cand.cpu().numpy(), pmass.cpu().numpy()
    Z = mlp.patches([x.astype(np.float64)], H, W, np.zeros(H * W, int), np.arange(H * W))
    logits = mlp.forward_infer(mlp.unpack(theta.astype(np.float64), K), Z, 1 / beta)
    oi, om_ = mlp.topm(logits, m)
    tol = 1e-3 * np.abs(logits).max() + 1e-3
    srt = -np.sort(-logits, axis=1)
    lg = np.take_along_axis(logits, cand, axis=1)
    assert np.all(lg >= srt[:, m - 1:m] - tol)
    assert np.all(np.diff(lg, axis=1) <= tol)  # decreasing order
    assert np.all(np.sort(cand, axis=1)[:, 1:] != np.sort(cand, axis=1)[:, :-1])  # distinct
    assert np.mean(np.all(cand == oi, axis=1)) >= 0.95
    mx = logits.max(axis=1, keepdims=True)
    e = np.exp(logits - mx)
    mass_of_cand = np.take_along_axis(e, cand, axis=1).sum(axis=1) / e.sum(axis=1)
    assert np.abs(pmass - mass_of_cand).max() <= 2e-3
    # anchors subset, n not a multiple of the tile
    an = np.arange(0, H * W, 7).astype(np.int32)
    c2, p2 = ep.proposal_topm(gm, dev(x), beta, anchors=dev(an, np.int32))
    np.testing.assert_array_equal(c2.cpu().numpy(), cand[an])
    np.testing.assert_array_equal(p2.cpu().numpy(), pmass[an])


def exact_argmins(om, beta, x, anchors, cand):
    sc = oracle.scores(om, beta, x.astype(np.float64), anchors)
    srt = np.sort(sc, axis=1)
    kall = np.argmin(sc, axis=1)
    cs = np.take_along_axis(sc, cand, axis=1)
    kc = cand[np.arange(len(cand)), np.argmin(cs, axis=1)]
    csrt = np.sort(cs, axis=1)
    gap_all = srt[:, 1] - srt[:, 0]
    gap_c = csrt[:, 1] - csrt[:, 0] if cand.shape[1] > 1 else np.full(len(cand), np.inf)
    return kall, gap_all, kc, gap_c


@pytest.mark.parametrize("r", [64, 8])
def test_proposal_selection_is_exact_on_its_candidates(r):
    """With an untrained network (poor proposals) and pmin = 0: every patch
    gets the exact argmin over its proposals, or -- when it was sent to the
    exhaustive pass -- the exact argmin over all components; where the exact
    argmin is proposed it is selected.  The patch estimates equal those of the
    exhaustive path forced to the same selection."""
    K, m = 200, 4
    g = synth.synthetic_gmm(K)
    gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_FIXED, r)
    om = oracle.Model(g.w, g.U, g.S, "fixed", r)
    p = ep.Proposal(K, seed=4)
    ep.attach_proposal(gm, p, topm=m, pmin=0.0)
    sigma = 25 / 255
    H, W = 48, 56
    x = (synth.image(6, H, W) + synth.noise(6, H, W, sigma)).astype(np.float32)
    beta = 8 / sigma ** 2
    o = ep.Options(select=ep.SELECT_PROPOSAL)
    xt, an, ks, gp = ep.patch_step(gm, dev(x), beta, o)
    cand, _ = ep.proposal_topm(gm, dev(x), beta)
    xt, an, ks, cand = xt.cpu().numpy(), an.cpu().numpy(), ks.cpu().numpy(), cand.cpu().numpy()
    kall, gap_all, kc, gap_c = exact_argmins(om, beta, x, an, cand)
    inc = (cand == kall[:, None]).any(axis=1)
    ok = (ks == kall) | (gap_all < TIE) | ((ks == kc) & ~inc) | ((gap_c < TIE) & np.isin(ks, cand))
    assert ok.all(), np.nonzero(~ok)[0][:10]
    assert np.all((ks == kall) | ~inc | (gap_all < TIE))
    # estimation and reprojection are those of the forced selection
    xt2, _, _, _ = ep.patch_step(gm, dev(x), beta, ep.Options(precision=ep.BF16X3), forced_k=dev(ks, np.int32))
    np.testing.assert_array_equal(xt, xt2.cpu().numpy())


def test_pmin_one_falls_back_to_exhaustive():
    """pmin = 1: every patch takes the exhaustive split-BF16 pass, so the
    selection and the gaps are those of the BF16X3 path bit for bit."""
    K = 200
    g = synth.synthetic_gmm(K)
    gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_FIXED, 64)
    p = ep.Proposal(K, seed=5)
    ep.attach_proposal(gm, p, topm=8, pmin=1.0)
    sigma = 25 / 255
    x = dev(synth.image(7, 64) + synth.noise(7, 64, 64, sigma))
    beta = 1 / sigma ** 2
    o = ep.Options(select=ep.SELECT_PROPOSAL, subset=ep.SUBSET_FRACTION, subset_param=1 / 3, seed=3)
    a = ep.patch_step(gm, x, beta, o)
    b = ep.patch_step(gm, x, beta, ep.Options(precision=ep.BF16X3, subset=ep.SUBSET_FRACTION, subset_param=1 / 3,
                                               seed=3))
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u.cpu().numpy(), v.cpu().numpy())


def test_select_proposal_without_network_is_rejected():
    g = synth.synthetic_gmm(20)
    gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_FIXED, 8)
    with pytest.raises(ep.EpllError):
        ep.patch_step(gm, dev(synth.image(0, 16)), 100.0, ep.Options(select=ep.SELECT_PROPOSAL))
    p = ep.Proposal(21, seed=0)
    with pytest.raises(ep.EpllError):
        ep.attach_proposal(gm, p, topm=4)  # K mismatch
    p2 = ep.Proposal(20, seed=0)
    with pytest.raises(ep.EpllError):
        ep.attach_proposal(gm, p2, topm=9)


def test_trained_network_gains():
    """Trained on pairs the method generates (denoising trajectories, K = 200,
    sigma in [5, 50]/255), the network's top-m proposals hold the exact
    selection far more often than the untrained network's, so far fewer
    patches fall back to the exhaustive pass, and the restoration keeps the
    exhaustive path's PSNR."""
    K, r, m = 200, 8, 8
    g = synth.synthetic_gmm(K)
    gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_FIXED, r)
    rng = np.random.default_rng(9)
    n_tr = 12
    sig = rng.uniform(5, 50, n_tr) / 255
    obs = [dev(synth.image(100 + i, 64) + synth.noise(100 + i, 64, 64, s)) for i, s in enumerate(sig)]
    data = pr.make_pairs(gm, obs, sig)
    assert len(data) == n_tr * 5 * 64 * 64
    p = ep.Proposal(K, seed=6)
    p0 = ep.Proposal(K, seed=6)
    losses = pr.train(p, data, steps=400, batch=2048, lr=2e-3, seed=1, log_every=100)
    assert losses[-1][1] < 0.6 * losses[0][1]
    # held-out trajectory at sigma = 25/255
    sigma = 25 / 255
    test = pr.make_pairs(gm, [dev(synth.image(300, 96) + synth.noise(300, 96, 96, sigma))], [sigma])
    hits = {}
    for name, net in (("trained", p), ("untrained", p0)):
        ep.attach_proposal(gm, net, topm=m)
        hr = []
        for t in range(5):
            sel = test.img_idx == t
            beta = float(np.exp(-test.log_ib[sel][0].item()))
            cand, _ = ep.proposal_topm(gm, test.images[t].contiguous(), beta)
            hr.append(pr.hit_rate(cand, test.labels[sel]))
        hits[name] = float(np.mean(hr))
    assert hits["trained"] >= hits["untrained"] + 0.3, hits
    # restoration with the trained proposal stays within 0.05 dB of exhaustive
    ep.attach_proposal(gm, p, topm=m, pmin=0.5)
    x, y = synth.denoise_problem(301, 96, sigma)
    opt = dict(subset=ep.SUBSET_FRACTION, subset_param=1 / 3, seed=2)
    xe = ep.restore(gm, dev(y), sigma, options=ep.Options(precision=ep.BF16X3, **opt)).cpu().numpy()
    xp = ep.restore(gm, dev(y), sigma, options=ep.Options(select=ep.SELECT_PROPOSAL, **opt)).cpu().numpy()
    ep.last_counters(gm)
    ps = lambda a: -10 * math.log10(np.mean((a - x) ** 2))
    assert abs(ps(xp) - ps(xe)) <= 0.05, (ps(xp), ps(xe))


def test_proposal_small_k_edge_cases():
    """K = 2 with one and two proposals, an 8x8 image (one patch row), and
    topm larger than K rejected."""
    g = synth.tiny_gmm(2, seed=3)
    gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_FIXED, 64)
    om = oracle.Model(g.w, g.U, g.S, "fixed", 64)
    p = ep.Proposal(2, seed=2)
    with pytest.raises(ep.EpllError):
        ep.attach_proposal(gm, p, topm=3)
    x = (synth.image(60, 8) + synth.noise(60, 8, 8, 0.05)).astype(np.float32)
    beta = 1 / 0.05 ** 2
    for m in (1, 2):
        ep.attach_proposal(gm, p, topm=m, pmin=0.0)
        _, an, ks, _ = ep.patch_step(gm, dev(x), beta, ep.Options(select=ep.SELECT_PROPOSAL))
        cand, pm = ep.proposal_topm(gm, dev(x), beta)
        ks, cand, an = ks.cpu().numpy(), cand.cpu().numpy(), an.cpu().numpy()
        assert np.all(np.isin(ks, [0, 1])) and cand.shape == (64, m)
        if m == 2:
            # both components proposed: the selection is the exhaustive one
            _, oks, ogap, _ = oracle.patch_step(om, beta, x.astype(np.float64), an)
            assert np.all((ks == oks) | (ogap < TIE))
            np.testing.assert_allclose(pm.cpu().numpy(), 1.0, atol=1e-6)


def test_proposal_batch_graph_equals_sequential():
    K = 200
    g = synth.synthetic_gmm(K)
    gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_FIXED, 8)
    p = ep.Proposal(K, seed=8)
    ep.attach_proposal(gm, p, topm=4, pmin=0.3)
    jobs = []
    for i, side in enumerate((64, 48, 96)):
        _, y = synth.denoise_problem(70 + i, side, 25 / 255)
        yd = dev(y)
        jobs.append((yd, torch.empty_like(yd), None, ep.DENOISE, 25 / 255))
    opts = ep.Options(select=ep.SELECT_PROPOSAL, subset=ep.SUBSET_FRACTION, subset_param=1 / 3, seed=4)
    ep.restore_batch(gm, jobs, options=opts, mode=ep.BATCH_GRAPH, lanes=2)
    torch.cuda.synchronize()
    a = [j[1].cpu().numpy().copy() for j in jobs]
    ep.restore_batch(gm, jobs, options=opts, mode=ep.BATCH_SEQUENTIAL)
    torch.cuda.synchronize()
    for u, j in zip(a, jobs):
        np.testing.assert_array_equal(u, j[1].cpu().numpy())
