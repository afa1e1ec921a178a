"""Seeded synthetic inputs for the EPLL / FEPLL restoration workloads.

This module is shared by the CUDA path's tests and benchmark and by the CPU
oracle's tests. It holds no arithmetic of the restoration method itself: it
only draws images, noise, masks, blur kernels and a Gaussian mixture patch
prior in the eigen-decomposed form the library consumes.

The paper evaluates on BSDS and six standard images with the 200-component
GMM of Zoran & Weiss; none of these are available, so seeded stand-ins with
the same shapes are used:

* images: a dead-leaves model (occluding discs, power-law radii r^-3 on
  [2, 20] px, grey levels U[0, 1]) -- a standard synthetic model of natural
  image statistics with sharp edges and flat regions;
* prior: K zero-mean Gaussians in 64-D (8x8 patches), each with a Haar-random
  orthonormal eigenbasis U_k and the shared power-law spectrum
  lambda_j = 0.05 j^-2, and Dirichlet(1) weights;
* degradations: additive white Gaussian noise, Bernoulli pixel masks, and a
  normalised 25x25 Gaussian blur kernel applied with periodic boundaries.

Seeds: image i uses 1000+i, its noise 2000+i, its mask 3000+i, the prior 7,
the uneven batch 4000.
"""
from __future__ import annotations

import functools
from dataclasses import dataclass

import numpy as np

PATCH = 8
P = PATCH * PATCH

# ----------------------------------------------------------------------------
# dead leaves
# ----------------------------------------------------------------------------
R_MIN, R_MAX = 2.0, 20.0
MARGIN = 20


def _radius_from_uniform(u: np.ndarray) -> np.ndarray:
    """Inverse CDF of the density proportional to r^-3 on [R_MIN, R_MAX]."""
    a, b = R_MIN ** -2, R_MAX ** -2
    return (a - u * (a - b)) ** -0.5


@functools.lru_cache(maxsize=64)
def _dead_leaves_cached(H: int, W: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    img = np.full((H, W), np.nan)
    uncovered = H * W
    n_drawn = 0
    chunk = 2048
    cap = 1_000_000
    while uncovered > 0 and n_drawn < cap:
        m = min(chunk, cap - n_drawn)
        r = _radius_from_uniform(rng.random(m))
        cy = rng.uniform(-MARGIN, H + MARGIN, m)
        cx = rng.uniform(-MARGIN, W + MARGIN, m)
        val = rng.random(m)
        n_drawn += m
        # Front-to-back painting: discs are drawn in order; a pixel (integer
        # centre) keeps the grey level of the first disc that covers it.
        for d in range(m):
            i0 = max(int(np.ceil(cy[d] - r[d])), 0)
            i1 = min(int(np.floor(cy[d] + r[d])), H - 1)
            j0 = max(int(np.ceil(cx[d] - r[d])), 0)
            j1 = min(int(np.floor(cx[d] + r[d])), W - 1)
            if i0 > i1 or j0 > j1:
                continue
            ii = np.arange(i0, i1 + 1)[:, None]
            jj = np.arange(j0, j1 + 1)[None, :]
            inside = (ii - cy[d]) ** 2 + (jj - cx[d]) ** 2 <= r[d] ** 2
            sub = img[i0:i1 + 1, j0:j1 + 1]
            fill = inside & np.isnan(sub)
            k = int(fill.sum())
            if k:
                sub[fill] = val[d]
                uncovered -= k
    if uncovered > 0:
        left = np.isnan(img)
        img[left] = rng.random(int(left.sum()))
    img.setflags(write=False)
    return img


def dead_leaves(H: int, W: int, seed: int) -> np.ndarray:
    """H x W float64 dead-leaves image in [0, 1] (a fresh writable copy)."""
    return _dead_leaves_cached(int(H), int(W), int(seed)).copy()


def image(i: int, H: int, W: int | None = None) -> np.ndarray:
    """Clean image number i of a workload (seed 1000+i)."""
    return dead_leaves(H, H if W is None else W, 1000 + i)


def noise(i: int, H: int, W: int, sigma: float) -> np.ndarray:
    """White Gaussian noise of standard deviation sigma (seed 2000+i)."""
    return sigma * np.random.default_rng(2000 + i).standard_normal((H, W))


def observed_mask(i: int, H: int, W: int, p_observed: float) -> np.ndarray:
    """0/1 float64 mask, each pixel observed with probability p_observed (seed 3000+i)."""
    return (np.random.default_rng(3000 + i).random((H, W)) < p_observed).astype(np.float64)


def gaussian_kernel(size: int = 25, sigma_b: float = 1.6) -> np.ndarray:
    """size x size Gaussian blur kernel, sum 1, centre at (size//2, size//2)."""
    c = size // 2
    u = np.arange(size) - c
    g = np.exp(-(u[:, None] ** 2 + u[None, :] ** 2) / (2.0 * sigma_b ** 2))
    return g / g.sum()


def blur_periodic(x: np.ndarray, kernel: np.ndarray) -> np.ndarray:
    """Circular convolution y[p] = sum_q kernel[q] x[p - (q - centre)] (input generation only)."""
    H, W = x.shape
    kh, kw = kernel.shape
    acc = np.zeros_like(x, dtype=np.float64)
    for u in range(kh):
        for v in range(kw):
            acc += kernel[u, v] * np.roll(x, (u - kh // 2, v - kw // 2), axis=(0, 1))
    return acc


# ----------------------------------------------------------------------------
# synthetic GMM patch prior
# ----------------------------------------------------------------------------
@dataclass(frozen=True)
class GMM:
    """Zero-mean GMM in eigen form: weights w[K], eigvecs U[K,P,P] (column j of
    U[k] is eigenvector j), eigvals S[K,P] in decreasing order."""
    w: np.ndarray
    U: np.ndarray
    S: np.ndarray

    @property
    def K(self) -> int:
        return int(self.w.shape[0])


def spectrum(P_: int = P) -> np.ndarray:
    j = np.arange(1, P_ + 1, dtype=np.float64)
    return 0.05 * j ** -2.0


@functools.lru_cache(maxsize=8)
def _gmm_cached(K: int, seed: int) -> GMM:
    rng = np.random.default_rng(seed)
    U = np.empty((K, P, P))
    for k in range(K):
        G = rng.standard_normal((P, P))
        Q, R = np.linalg.qr(G)
        Q = Q * np.sign(np.diag(R))[None, :]  # Haar measure: diag(R) > 0
        U[k] = Q
    w = rng.exponential(1.0, K)  # Dirichlet(1) = normalised Exp(1)
    w = w / w.sum()
    S = np.tile(spectrum(), (K, 1))
    for a in (w, U, S):
        a.setflags(write=False)
    return GMM(w=w, U=U, S=S)


def synthetic_gmm(K: int, seed: int = 7) -> GMM:
    return _gmm_cached(int(K), int(seed))


def tiny_gmm(K: int, seed: int, P_: int = P) -> GMM:
    """A small GMM with distinct random spectra per component (for pins that
    need components to differ in their log-determinants too)."""
    rng = np.random.default_rng(seed)
    U = np.empty((K, P_, P_))
    S = np.empty((K, P_))
    for k in range(K):
        Q, R = np.linalg.qr(rng.standard_normal((P_, P_)))
        U[k] = Q * np.sign(np.diag(R))[None, :]
        S[k] = np.sort(rng.uniform(0.0005, 0.05, P_) * rng.uniform(0.2, 1.0)
                       * np.arange(1, P_ + 1) ** -1.0)[::-1]
    w = rng.exponential(1.0, K)
    return GMM(w=w / w.sum(), U=U, S=S)


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------
@dataclass(frozen=True)
class Job:
    """One restoration problem of the uneven batch: side, sigma, task."""
    side: int
    sigma: float
    inpaint: bool


def uneven_batch(n: int = 64, seed: int = 4000) -> list[Job]:
    rng = np.random.default_rng(seed)
    sides = rng.choice([128, 256, 384, 512, 768, 1024], size=n)
    sig = rng.uniform(5.0, 50.0, size=n) / 255.0
    task = rng.random(n) < 0.5
    return [Job(int(s), float(g), bool(t)) for s, g, t in zip(sides, sig, task)]


def denoise_problem(i: int, H: int, sigma: float, W: int | None = None):
    """(clean x, observation y = x + w) for image i."""
    W = H if W is None else W
    x = image(i, H, W)
    return x, x + noise(i, H, W, sigma)


def inpaint_problem(i: int, H: int, sigma: float, p_observed: float = 0.7, W: int | None = None):
    """(clean x, mask a, observation y = a*x + w)."""
    W = H if W is None else W
    x = image(i, H, W)
    a = observed_mask(i, H, W, p_observed)
    return x, a, a * x + noise(i, H, W, sigma)


def deblur_problem(i: int, H: int, sigma: float, W: int | None = None,
                   size: int = 25, sigma_b: float = 1.6):
    """(clean x, kernel, observation y = kernel (*) x + w), periodic blur."""
    W = H if W is None else W
    x = image(i, H, W)
    k = gaussian_kernel(size, sigma_b)
    return x, k, blur_periodic(x, k) + noise(i, H, W, sigma)


def clean_patches(n: int, seed: int = 0, side: int = 256) -> np.ndarray:
    """n DC-free 8x8 patches (rows of 64) at random positions (periodic wrap)
    of dead-leaves images side x side, the i-th image drawn with seed
    5000 + 1000 seed + i; training data for an EM-fitted prior."""
    rng = np.random.default_rng(seed)
    per_image = side * side // 4
    out = np.empty((n, P))
    got, i = 0, 0
    while got < n:
        img = dead_leaves(side, side, 5000 + seed * 1000 + i)
        m = min(per_image, n - got)
        a = rng.integers(0, side * side, m)
        r, c = np.divmod(a, side)
        rows = (r[:, None] + np.arange(8)[None, :]) % side
        cols = (c[:, None] + np.arange(8)[None, :]) % side
        p = img[rows[:, :, None], cols[:, None, :]].reshape(m, P)
        out[got:got + m] = p - p.mean(axis=1, keepdims=True)
        got += m
        i += 1
    return out
