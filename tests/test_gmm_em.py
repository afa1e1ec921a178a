"""The offline EM fit of the GMM prior (Eq. 2, fitted by EM in Sec. 2),
pinned on the host: the K = 1 closed form (the sample covariance), the EM
property that the likelihood never decreases, recovery of a known mixture from
its samples, the eigen form handed to the library, and the point of fitting
a prior at all: restoring with it (FP64 oracle) beats the noisy input, which
the random synthetic prior does not."""
import math

import numpy as np
import pytest

import oracle
import synth
from paper_1710_08124_gb300 import gmm_em


def test_k1_is_the_sample_covariance():
    rng = np.random.default_rng(0)
    Z = rng.standard_normal((500, 5)) @ rng.standard_normal((5, 5))
    w, U, S, ll = gmm_em.fit(Z, 1, iters=3, eps_rel=1e-3)
    eps = 1e-3 * np.mean(Z * Z)
    C = Z.T @ Z / 500 + eps * np.eye(5)
    assert np.allclose(w, [1.0])
    assert np.allclose(U[0] @ np.diag(S[0]) @ U[0].T, C, rtol=1e-10, atol=1e-12)
    # the likelihood of the closed form: -1/2 (log|C| + tr(C^-1 Zt Z / N) + D log 2 pi)
    expect = -0.5 * (np.linalg.slogdet(C)[1] + np.trace(np.linalg.solve(C, Z.T @ Z / 500))
                     + 5 * math.log(2 * math.pi))
    assert abs(ll[-1] - expect) < 1e-10 * abs(expect)


def test_likelihood_never_decreases():
    Z = synth.clean_patches(3000, seed=1, side=64)
    _, _, _, ll = gmm_em.fit(Z, 6, iters=12, seed=2, min_weight=0.0)
    assert np.all(np.diff(ll) >= -1e-9 * np.abs(ll[1:]))
    assert ll[-1] > ll[0]


def test_recovers_a_known_mixture():
    rng = np.random.default_rng(3)
    D, K, N = 6, 3, 30000
    w0 = np.array([0.5, 0.3, 0.2])
    covs = []
    for k in range(K):
        Q, _ = np.linalg.qr(rng.standard_normal((D, D)))
        covs.append(Q @ np.diag(np.geomspace(4.0, 0.01, D) * (k + 1)) @ Q.T)
    lab = rng.choice(K, N, p=w0)
    Z = np.stack([rng.multivariate_normal(np.zeros(D), covs[k]) for k in lab])
    w, U, S, _ = gmm_em.fit(Z, K, iters=60, seed=4, eps_rel=1e-6, min_weight=0.0)
    fitted = [U[k] @ np.diag(S[k]) @ U[k].T for k in range(K)]
    for k in range(K):
        # the fitted component closest to the true one
        err = [np.linalg.norm(f - covs[k]) / np.linalg.norm(covs[k]) for f in fitted]
        j = int(np.argmin(err))
        assert err[j] < 0.1, (k, err)
        assert abs(w[j] - w0[k]) < 0.03, (k, w[j])


def test_eigen_form():
    Z = synth.clean_patches(2000, seed=5, side=64)
    w, U, S, _ = gmm_em.fit(Z, 4, iters=5, seed=6)
    assert U.shape == (4, 64, 64) and S.shape == (4, 64)
    assert abs(w.sum() - 1.0) < 1e-12 and np.all(w > 0)
    assert np.all(S > 0) and np.all(np.diff(S, axis=1) <= 0)
    for k in range(4):
        assert np.allclose(U[k].T @ U[k], np.eye(64), atol=1e-10)


def test_fitted_prior_denoises():
    """EM on 20,000 dead-leaves patches (K = 8): the FP64 oracle's restoration of
    a noisy 40x40 dead-leaves image gains PSNR over the noisy input, while the
    random synthetic prior of the same size loses it."""
    Z = synth.clean_patches(20000, seed=7, side=128)
    w, U, S, _ = gmm_em.fit(Z, 8, iters=15, seed=8)
    sigma = 25 / 255
    x, y = synth.denoise_problem(9, 40, sigma)
    ps = lambda a: -10 * math.log10(np.mean((a - x) ** 2))
    em = oracle.restore(oracle.Model(w, U, S, "fixed", 64), y.astype(np.float64), sigma)
    g = synth.synthetic_gmm(8)
    rnd = oracle.restore(oracle.Model(g.w, g.U, g.S, "fixed", 64), y.astype(np.float64), sigma)
    assert ps(em) > ps(y) + 3.0, (ps(em), ps(y))
    assert ps(rnd) < ps(y)
