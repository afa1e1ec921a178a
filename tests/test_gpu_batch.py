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
            for j, ref in zip(jobs, singles):
                assert np.array_equal(j[1].cpu().numpy(), ref), (lanes, rep)
    ep.last_counters(gm)


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
