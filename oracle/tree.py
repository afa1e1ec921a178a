"""ORACLE -- test infrastructure only.

FP64 reference of the balanced search tree of the Gaussian selection
(Sec. "Speed-up via a balanced search tree"): the symmetric KL divergence
between zero-mean Gaussians (Eq. 17), a partition of a level's components
into clusters of about equal size that lowers the clustering cost of Eq. 18,
the collapse of each cluster into one Gaussian by moment matching (Eq. 19),
and the descent that follows the cheapest child from the root to a leaf.

The paper solves Eq. 18 with a third-party genetic algorithm; the partition
here is a deterministic stand-in (farthest-point seeds, size-capped greedy
assignment, pairwise swaps that lower Eq. 18), which the library's builder
implements separately.  Level sizes: the smallest power of two not below
K / 4, then halving down to one (200 -> 64, 32, 16, 8, 4, 2, 1), so that the
last clusters hold at most four leaves and the others two.

Readings: Eq. 18 sums KL(Sigma_k1, Sigma_k2) over the pairs of a cluster (the
printed KL(Sigma_k1, Sigma_k1) is read as this); the descent starts with the
root's children (the "two first nodes"); ties go to the lowest child index.
"""
from __future__ import annotations

import numpy as np


def sym_kl(S1, S2):
    """Eq. 17: 1/2 Tr(S2^-1 S1 + S1^-1 S2 - 2 I), written with explicit inverses."""
    P = S1.shape[0]
    return 0.5 * (np.trace(np.linalg.solve(S2, S1)) + np.trace(np.linalg.solve(S1, S2)) - 2 * P)


def kl_matrix(covs):
    K = len(covs)
    D = np.zeros((K, K))
    for a in range(K):
        for b in range(a + 1, K):
            D[a, b] = D[b, a] = sym_kl(covs[a], covs[b])
    return D


def cost(D, parts):
    """Eq. 18 over ordered pairs of every cluster."""
    return float(sum(D[np.ix_(p, p)].sum() for p in parts))


def level_sizes(K: int):
    if K <= 4:
        return [1]
    L = 1
    while 4 * L < K:
        L *= 2
    out = []
    while True:
        out.append(L)
        if L == 1:
            return out
        L //= 2


def partition(D, w, L: int):
    """Clusters of sizes floor(n/L) or ceil(n/L) (the larger ones for the
    earliest seeds), each a sorted list of indices, in seed order."""
    n = D.shape[0]
    if L == 1:
        return [list(range(n))]
    # farthest-point seeds, the heaviest component first (lowest index on ties)
    seeds = [int(np.argmax(w))]
    mind = D[seeds[0]].copy()
    while len(seeds) < L:
        mind[seeds] = -1.0
        s = int(np.argmax(mind))
        seeds.append(s)
        mind = np.minimum(mind, D[s])
    cap = [n // L + (1 if i < n % L else 0) for i in range(L)]
    label = -np.ones(n, int)
    for i, s in enumerate(seeds):
        label[s] = i
        cap[i] -= 1
    # greedy: (distance, node, seed rank) ascending
    pairs = sorted((D[x, s], x, i) for x in range(n) for i, s in enumerate(seeds) if label[x] < 0)
    for d, x, i in pairs:
        if label[x] < 0 and cap[i] > 0:
            label[x] = i
            cap[i] -= 1
    # pairwise swaps: for each node in turn, the swap that lowers Eq. 18 most
    for _ in range(100):
        improved = False
        for a in range(n):
            best, bb = -1e-12, -1
            for b in range(n):
                if label[b] == label[a]:
                    continue
                A = [x for x in range(n) if label[x] == label[a]]
                B = [x for x in range(n) if label[x] == label[b]]
                delta = 2 * (sum(D[a, x] for x in B if x != b) + sum(D[b, x] for x in A if x != a)
                             - sum(D[a, x] for x in A if x != a) - sum(D[b, x] for x in B if x != b))
                if delta < best:
                    best, bb = delta, b
            if bb >= 0:
                label[a], label[bb] = label[bb], label[a]
                improved = True
        if not improved:
            break
    return [sorted(np.nonzero(label == i)[0].tolist()) for i in range(L)]


def collapse(w, covs, parts):
    """Eq. 19: summed weights and weight-averaged covariances."""
    wl = np.array([sum(w[k] for k in p) for p in parts])
    cl = [sum(w[k] * covs[k] for k in p) / wl[i] for i, p in enumerate(parts)]
    return wl, cl


def build(w, U, S):
    """Returns the levels from the leaves up: a list of (weights, covariances,
    parts), parts[l] = the indices (in the level below) collapsed into node l."""
    covs = [U[k] @ np.diag(S[k]) @ U[k].T for k in range(len(w))]
    cur_w, cur_c = np.asarray(w, float), covs
    levels = []
    for L in level_sizes(len(w)):
        D = kl_matrix(cur_c)
        parts = partition(D, cur_w, L)
        cur_w, cur_c = collapse(cur_w, cur_c, parts)
        levels.append((cur_w, cur_c, parts))
    return levels


def descend(scores, child_begin, root: int = 0):
    """Leaf reached by every patch and the smallest top-2 gap among the
    siblings compared on its way.  scores: [n][nodes] (lower is better);
    node v's children are child_begin[v] .. child_begin[v+1]-1."""
    n = scores.shape[0]
    leaf = np.zeros(n, int)
    gap = np.full(n, np.inf)
    for i in range(n):
        v = root
        while child_begin[v + 1] > child_begin[v]:
            ch = range(child_begin[v], child_begin[v + 1])
            best = min(ch, key=lambda c: (scores[i, c], c))
            others = [scores[i, c] for c in ch if c != best]
            if others:
                gap[i] = min(gap[i], min(others) - scores[i, best])
            v = best
        leaf[i] = v
    return leaf, gap
