"""Offline fit of the zero-mean GMM patch prior of Eq. 2 by
Expectation-Maximization (Dempster, Laird & Rubin, 1977), as in Sec. 2 where
the weights and covariances are estimated by EM on clean patches.  The
paper's training set (2 million BSDS patches) is not available here; DC-free
8x8 patches of synthetic dead-leaves images stand in for it
(`synth.clean_patches`).  The result is returned in the eigen form `gmm_load`
takes.

Host numpy, run once per prior; nothing here is on the restoration path.

E step (log domain, per component k with Sigma_k = L_k L_k^T):
    log p_ik = log w_k - (1/2) (log|Sigma_k| + |L_k^-1 z_i|^2 + P log 2 pi)
    gamma_ik = p_ik / sum_l p_il
M step:
    N_k = sum_i gamma_ik,  w_k = N_k / N,
    Sigma_k = sum_i gamma_ik z_i z_i^T / N_k + eps I
eps (a small multiple of the data's mean variance) keeps every covariance
positive definite: DC-free patches leave the constant direction empty, and a
component may hold few patches.  A component whose weight falls below
min_weight is re-seeded with the covariance of a share of the patches the
model explains worst (a heuristic step outside EM; min_weight = 0 turns it
off).
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular


def _log_resp(Z, w, covs):
    """(log p_ik [N, K], per-sample log-likelihood [N])."""
    N, D = Z.shape
    K = w.shape[0]
    lp = np.empty((N, K))
    for k in range(K):
        L = np.linalg.cholesky(covs[k])
        y = solve_triangular(L, Z.T, lower=True)         # L^-1 z_i as columns
        maha = np.einsum("ij,ij->j", y, y)
        logdet = 2.0 * np.log(np.diag(L)).sum()
        lp[:, k] = np.log(max(w[k], 1e-300)) - 0.5 * (logdet + maha + D * np.log(2.0 * np.pi))
    mx = lp.max(axis=1, keepdims=True)
    ll = mx[:, 0] + np.log(np.exp(lp - mx).sum(axis=1))
    return lp, ll


def _init(Z, K, rng):
    """Hard initial assignment: K seeds chosen k-means++-style on the patch
    directions (|cos| similarity, so a seed and its negative are alike), each
    patch to its most similar seed."""
    norm = np.linalg.norm(Z, axis=1)
    Y = Z[norm > 0] / norm[norm > 0, None]
    seeds = [Y[rng.integers(0, Y.shape[0])]]
    best = np.abs(Y @ seeds[0])
    for _ in range(1, K):
        d = np.maximum(1.0 - best ** 2, 0.0)
        tot = d.sum()
        j = rng.integers(0, Y.shape[0]) if tot <= 0 else rng.choice(Y.shape[0], p=d / tot)
        seeds.append(Y[j])
        best = np.maximum(best, np.abs(Y @ Y[j]))
    S = np.stack(seeds)
    lab = np.argmax(np.abs((Z / np.maximum(norm, 1e-300)[:, None]) @ S.T), axis=1)
    R = np.zeros((Z.shape[0], K))
    R[np.arange(Z.shape[0]), lab] = 1.0
    return R


def _mstep(Z, R, eps):
    N, D = Z.shape
    Nk = R.sum(axis=0)
    w = Nk / N
    covs = np.empty((R.shape[1], D, D))
    for k in range(R.shape[1]):
        covs[k] = (Z.T * R[:, k]) @ Z / max(Nk[k], 1e-300) + eps * np.eye(D)
    return w, covs


def fit(Z: np.ndarray, K: int, iters: int = 30, seed: int = 0, eps_rel: float = 1e-3,
        min_weight: float = 1e-4):
    """EM fit of a K-component zero-mean GMM to the rows of Z.

    Returns (w [K], U [K][D][D] with eigenvectors as columns, S [K][D]
    non-increasing, loglik [iters + 1]: mean log-likelihood after the initial
    M step and after every iteration).  min_weight = 0 disables the
    re-seeding, leaving plain EM (whose log-likelihood never decreases)."""
    Z = np.asarray(Z, np.float64)
    N, D = Z.shape
    rng = np.random.default_rng(seed)
    eps = eps_rel * float(np.mean(Z * Z))
    w, covs = _mstep(Z, _init(Z, K, rng), eps)
    hist = []
    for it in range(iters + 1):
        lp, ll = _log_resp(Z, w, covs)
        hist.append(float(ll.mean()))
        if it == iters:
            break
        R = np.exp(lp - ll[:, None])
        w, covs = _mstep(Z, R, eps)
        dead = np.nonzero(w < min_weight)[0] if min_weight > 0 else np.zeros(0, int)
        if dead.size:
            # re-seed collapsed components on the worst-explained patches
            worst = np.argsort(ll)[: dead.size * max(D, 8)]
            for j, k in enumerate(dead):
                zs = Z[worst[j::dead.size]]
                covs[k] = zs.T @ zs / zs.shape[0] + eps * np.eye(D)
                w[k] = min_weight
            w /= w.sum()
    S, U = np.linalg.eigh(covs)
    S, U = S[:, ::-1], U[:, :, ::-1]
    return w, np.ascontiguousarray(U), np.ascontiguousarray(S), np.array(hist)
