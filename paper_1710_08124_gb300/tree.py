"""Offline construction of the balanced search tree of the Gaussian selection
(Sec. "Speed-up via a balanced search tree").

The GMM is collapsed level by level: a level's components are partitioned
into clusters of about equal size that keep similar components together
(symmetric KL divergence, Eq. 17; clustering cost, Eq. 18) and every cluster
is replaced by one Gaussian with the summed weight and the weight-averaged
covariance (Eq. 19), until one component remains.  The paper solves Eq. 18
with a genetic algorithm for the multiple travelling salesmen problem; this
builder is deterministic: farthest-point seeds (the heaviest component
first), a size-capped greedy assignment by increasing divergence, then
pairwise swaps between clusters while one lowers Eq. 18.  Level sizes are
the smallest power of two not below K / 4, then halving down to one
(K = 200: 64, 32, 16, 8, 4, 2, 1), so no node has more than four children.

The result is handed to the library (``attach_tree``) as arrays over the
nodes in breadth-first order, the root first and the children of every node
consecutive, leaves mapped back to the model's components.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Tree:
    weights: np.ndarray        # [n_nodes]
    eigvecs: np.ndarray        # [n_nodes][64][64], column j = j-th eigenvector
    eigvals: np.ndarray        # [n_nodes][64], non-increasing
    child_begin: np.ndarray    # [n_nodes + 1] int32: children of v are child_begin[v] .. child_begin[v+1]-1
    leaf_component: np.ndarray  # [n_nodes] int32: the model component of a leaf, -1 for internal nodes
    levels: list               # from the leaves up: (parts) per collapse

    @property
    def n_nodes(self) -> int:
        return int(self.weights.shape[0])

    @property
    def depth(self) -> int:
        return len(self.levels)


def level_sizes(K: int):
    if K <= 4:
        return [1]
    L = 1
    while 4 * L < K:
        L *= 2
    sizes = []
    while True:
        sizes.append(L)
        if L == 1:
            return sizes
        L //= 2


def kl_divergences(covs: np.ndarray) -> np.ndarray:
    """Symmetric KL (Eq. 17) between all pairs of zero-mean Gaussians."""
    K, P, _ = covs.shape
    inv = np.linalg.inv(covs)
    # A[a, b] = Tr(Sigma_a^-1 Sigma_b)
    A = inv.reshape(K, P * P) @ covs.transpose(0, 2, 1).reshape(K, P * P).T
    D = 0.5 * (A + A.T) - P
    np.fill_diagonal(D, 0.0)
    return D


def balanced_partition(D: np.ndarray, w: np.ndarray, L: int, max_passes: int = 100):
    n = D.shape[0]
    if L == 1:
        return [list(range(n))]
    seeds = [int(np.argmax(w))]
    mind = D[seeds[0]].copy()
    while len(seeds) < L:
        mind[seeds] = -1.0
        s = int(np.argmax(mind))
        seeds.append(s)
        mind = np.minimum(mind, D[s])
    cap = np.array([n // L + (1 if i < n % L else 0) for i in range(L)])
    label = np.full(n, -1)
    label[seeds] = np.arange(L)
    cap -= 1
    free = np.nonzero(label < 0)[0]
    d = D[np.ix_(free, seeds)]                       # [free][L]
    xs = np.repeat(free, L)
    ss = np.tile(np.arange(L), free.size)
    order = np.lexsort((ss, xs, d.ravel()))          # distance, then node, then seed rank
    for x, i in zip(xs[order], ss[order]):
        if label[x] < 0 and cap[i] > 0:
            label[x] = i
            cap[i] -= 1
    onehot = np.zeros((n, L))
    onehot[np.arange(n), label] = 1.0
    S = D @ onehot                                   # S[x, l] = sum of D[x, c] over cluster l
    for _ in range(max_passes):
        improved = False
        for a in range(n):
            la = label[a]
            lb = label
            delta = 2.0 * (S[a, lb] - D[a] + S[:, la] - D[:, a] - S[a, la] - S[np.arange(n), lb])
            delta[lb == la] = np.inf
            b = int(np.argmin(delta))
            if delta[b] < -1e-12:
                lbb = label[b]
                S[:, la] += D[:, b] - D[:, a]
                S[:, lbb] += D[:, a] - D[:, b]
                label[a], label[b] = lbb, la
                improved = True
        if not improved:
            break
    return [sorted(np.nonzero(label == i)[0].tolist()) for i in range(L)]


def build_tree(w, U, S) -> Tree:
    """Balanced search tree of the GMM (weights w [K], eigenvectors U [K][64][64],
    eigenvalues S [K][64], non-increasing)."""
    w = np.asarray(w, np.float64)
    U = np.asarray(U, np.float64)
    S = np.asarray(S, np.float64)
    K = w.shape[0]
    covs = np.einsum("kij,kj,klj->kil", U, S, U)
    cur_w, cur_c = w, covs
    levels, node_w, node_c = [], [w], [covs]
    for L in level_sizes(K):
        parts = balanced_partition(kl_divergences(cur_c), cur_w, L)
        nw = np.array([cur_w[p].sum() for p in parts])
        nc = np.stack([np.einsum("k,kij->ij", cur_w[p], cur_c[p]) / nw[i] for i, p in enumerate(parts)])
        levels.append(parts)
        cur_w, cur_c = nw, nc
        node_w.append(nw)
        node_c.append(nc)
    # breadth-first order from the root: every node's children consecutive
    depth = len(levels)
    order = [[0]]                                    # indices within each level, top (root) first
    for lev in range(depth - 1, -1, -1):
        parts = levels[lev]
        order.append([c for v in order[-1] for c in parts[v]])
    n_nodes = sum(len(o) for o in order)
    weights = np.zeros(n_nodes)
    eigvecs = np.zeros((n_nodes, 64, 64))
    eigvals = np.zeros((n_nodes, 64))
    child_begin = np.zeros(n_nodes + 1, np.int32)
    leaf = np.full(n_nodes, -1, np.int32)
    base = np.cumsum([0] + [len(o) for o in order])
    for t, idx in enumerate(order):                  # t = 0 root ... depth = leaves
        lev = depth - t                              # index into node_w (0 = leaves)
        for pos, v in enumerate(idx):
            g = base[t] + pos
            weights[g] = node_w[lev][v]
            if lev == 0:
                eigvecs[g], eigvals[g] = U[v], S[v]
                leaf[g] = v
            else:
                lam, vec = np.linalg.eigh(node_c[lev][v])
                eigvals[g] = np.maximum(lam[::-1], 1e-300)
                eigvecs[g] = vec[:, ::-1]
        if t < depth:
            parts = levels[depth - 1 - t]
            nxt = 0
            for pos, v in enumerate(idx):
                child_begin[base[t] + pos] = base[t + 1] + nxt
                nxt += len(parts[v])
    child_begin[base[depth]:] = n_nodes
    return Tree(weights, eigvecs, eigvals, child_begin, leaf, levels)
