"""Batched restoration of uneven images (epll_restore_batch): sequential and
CUDA-graph modes give exactly the per-image results, on repeated calls
(graph replay) and with the autotuned lane count; one image against the
FP64 oracle."""
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


@pytest.fixture(scope="module", autouse=True)
def _built():
    ep.build()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")


def make_jobs():
    rng = np.random.default_rng(5)
    jobs, refs = [], []
    for i, (H, W) in enumerate([(40, 64), (16, 16), (64, 24), (33, 47), (24, 24), (56, 40)]):
        sigma = float(rng.uniform(5, 50) / 255)
        if i % 2:
            x, a, y = synth.inpaint_problem(20 + i, H, sigma, 0.7, W=W)
            jobs.append((dev(y), torch.empty((H, W), device="cuda"), dev(a), ep.PIXELWISE, sigma))
        else:
            x, y = synth.denoise_problem(20 + i, H, sigma, W=W)
            jobs.append((dev(y), torch.empty((H, W), device="cuda"), None, ep.DENOISE, sigma))
        refs.append(x)
    return jobs, refs


@pytest.mark.parametrize("prec,r", [(ep.BF16X3, 8), (ep.FP32, 8), (ep.AUTO, 64)])
def test_batch_modes_match_per_image(prec, r):
    """AUTO at rank 64 runs the FP16 pass with its candidate step in every lane."""
    g = synth.synthetic_gmm(37)
    gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_FIXED, r)
    o = ep.Options(precision=prec, subset=ep.SUBSET_FRACTION, subset_param=1 / 3, seed=4, cg_iters=50)
    jobs, _ = make_jobs()
    singles = [ep.restore(gm, y, s, kind=k, a=a, options=o).cpu().numpy() for y, _, a, k, s in jobs]
    ep.restore_batch(gm, jobs, options=o, mode=ep.BATCH_SEQUENTIAL)
    for j, ref in zip(jobs, singles):
        assert np.array_equal(j[1].cpu().numpy(), ref)
    for lanes in (2, 0):
        for rep in range(2):  # second call replays the captured graph
            for j in jobs:
                j[1].fill_(float("nan"))
            ep.restore_batch(gm, jobs, options=o, mode=ep.BATCH_GRAPH, lanes=lanes)
            torch.cuda.synchronize()
            refs = singles
            if lanes == 0:
                # the autotuned tiles: per-image restorations with the same tiles
                _, bn, agg = ep.batch_config(gm)
                assert bn in (128, 256) and agg in (1, 2)
                refs = singles_with_tiles(gm, jobs, o, bn, agg)
            for j, ref in zip(jobs, refs):
                assert np.array_equal(j[1].cpu().numpy(), ref), (lanes, rep)
    ep.last_counters(gm)


def singles_with_tiles(gm, jobs, o, bn, agg):
    ep.set_tiles(gm, bn, agg)
    try:
        return [ep.restore(gm, *job_args(j)[0], **job_args(j)[1], options=o).cpu().numpy() for j in jobs]
    finally:
        ep.set_tiles(gm, 256, 1)


def job_args(j):
    y, _, a, k, s = j[:5]
    kern = j[5] if len(j) > 5 else None
    return (y, s), dict(kind=k, a=a, kernel=kern)


def test_tile_shapes_give_the_same_restoration():
    """Selection with 128-column basis stages and reprojection with two image
    rows per warp: the same selections, the same restoration up to the order
    of the FP32 sums of the reprojection."""
    g = synth.synthetic_gmm(40)
    sigma = 25 / 255
    x, y = synth.denoise_problem(31, 96, sigma, W=80)
    for prec, r in ((ep.AUTO, 64), (ep.BF16X3, 8), (ep.BF16, 16)):
        gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_FIXED, r)
        o = ep.Options(precision=prec, subset=ep.SUBSET_FRACTION, subset_param=1 / 3, seed=2)
        _, _, k0, _ = ep.patch_step(gm, dev(y), 4 / sigma ** 2, o)
        x0 = ep.restore(gm, dev(y), sigma, options=o).cpu().numpy()
        for bn, agg in ((128, 1), (256, 2), (128, 2)):
            ep.set_tiles(gm, bn, agg)
            _, _, k1, _ = ep.patch_step(gm, dev(y), 4 / sigma ** 2, o)
            assert torch.equal(k0, k1), (prec, r, bn, agg)
            x1 = ep.restore(gm, dev(y), sigma, options=o).cpu().numpy()
            assert np.abs(x1 - x0).max() <= 1e-5, (prec, r, bn, agg)
        ep.set_tiles(gm, 256, 1)
    with pytest.raises(ep.EpllError):
        ep.set_tiles(gm, 64, 2)


def test_batch_with_blur_jobs():
    """Periodic-deblurring jobs in a batch (device copies of their kernels,
    one FFT plan per size in each lane): graph replays equal per-image
    restorations bit for bit, and the first job equals the oracle's."""
    g = synth.synthetic_gmm(24)
    gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_FIXED, 8)
    om = oracle.Model(g.w, g.U, g.S, "fixed", 8)
    o = ep.Options(precision=ep.BF16X3, subset=ep.SUBSET_FRACTION, subset_param=1 / 3, seed=6)
    jobs = []
    rng = np.random.default_rng(9)
    for i, (H, W) in enumerate([(48, 40), (32, 32), (40, 56), (32, 32), (24, 40)]):
        sigma = float(rng.uniform(2, 10) / 255)
        if i == 3:
            x, y = synth.denoise_problem(60 + i, H, sigma, W=W)
            jobs.append((dev(y), torch.empty((H, W), device="cuda"), None, ep.DENOISE, sigma))
        else:
            x, k, y = synth.deblur_problem(60 + i, H, sigma, W=W, size=9 if (i % 2 or H < 25) else 25, sigma_b=1.2 + 0.2 * i)
            jobs.append((dev(y), torch.empty((H, W), device="cuda"), None, ep.CONV_PERIODIC, sigma,
                         k.astype(np.float32)))
    singles = [ep.restore(gm, *job_args(j)[0], **job_args(j)[1], options=o).cpu().numpy() for j in jobs]
    ep.restore_batch(gm, jobs, options=o, mode=ep.BATCH_SEQUENTIAL)
    for j, ref in zip(jobs, singles):
        assert np.array_equal(j[1].cpu().numpy(), ref)
    for lanes in (2, 3):
        for rep in range(2):
            for j in jobs:
                j[1].fill_(float("nan"))
            ep.restore_batch(gm, jobs, options=o, mode=ep.BATCH_GRAPH, lanes=lanes)
            torch.cuda.synchronize()
            for j, ref in zip(jobs, singles):
                assert np.array_equal(j[1].cpu().numpy(), ref), (lanes, rep)
    y, _, _, _, sigma, k = jobs[0]
    xo = oracle.restore(om, y.cpu().numpy().astype(np.float64), sigma, deg=oracle.CONV,
                        kernel=k.astype(np.float64), subset=oracle.FRACTION, subset_param=1 / 3, seed=6)
    assert np.abs(singles[0] - xo).max() <= 1e-4


def test_batch_image_matches_oracle():
    g = synth.synthetic_gmm(37)
    gm = ep.gmm_load(g.w, g.U, g.S, ep.RANK_FIXED, 8)
    om = oracle.Model(g.w, g.U, g.S, "fixed", 8)
    o = ep.Options(precision=ep.BF16X3, subset=ep.SUBSET_FRACTION, subset_param=1 / 3, seed=4)
    jobs, refs = make_jobs()
    ep.restore_batch(gm, jobs, options=o, mode=ep.BATCH_GRAPH, lanes=3)
    y, xo, _, _, sigma = jobs[0]
    xr = oracle.restore(om, y.cpu().numpy().astype(np.float64), sigma, subset=oracle.FRACTION,
                        subset_param=1 / 3, seed=4)
    ps = lambda a: -10 * math.log10(np.mean((a - refs[0]) ** 2))
    assert abs(ps(xo.cpu().numpy()) - ps(xr)) <= 0.05
