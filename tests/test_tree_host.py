"""The library's tree builder (host, offline model preparation) against the
FP64 tree oracle: same partitions on small models, valid breadth-first node
arrays, node covariances equal to the oracle's collapse (Eq. 19), and the
paper's level structure at K = 200."""
import numpy as np

import synth
from oracle import tree as ot
from paper_1710_08124_gb300 import tree as pt


def test_builder_matches_oracle_partitions():
    for K in (5, 20, 40):
        g = synth.synthetic_gmm(K)
        lv = ot.build(g.w, g.U, g.S)
        T = pt.build_tree(g.w, g.U, g.S)
        assert [p for _, _, p in lv] == T.levels


def test_node_arrays_are_a_valid_tree():
    K = 40
    g = synth.synthetic_gmm(K)
    T = pt.build_tree(g.w, g.U, g.S)
    cb = T.child_begin
    n = T.n_nodes
    assert cb[0] == 1 and cb[-1] == n and np.all(np.diff(cb) >= 0)
    parent = -np.ones(n, int)
    for v in range(n):
        for c in range(cb[v], cb[v + 1]):
            assert parent[c] < 0 and c > v
            parent[c] = v
    assert parent[0] == -1 and np.all(parent[1:] >= 0)
    leaves = np.nonzero(cb[:-1] == cb[1:])[0]
    assert sorted(T.leaf_component[leaves].tolist()) == list(range(K))
    assert np.all(T.leaf_component[cb[:-1] != cb[1:]] == -1)
    # every leaf at the same depth
    depth = np.zeros(n, int)
    for v in range(1, n):
        depth[v] = depth[parent[v]] + 1
    assert len(set(depth[leaves].tolist())) == 1 and depth[leaves][0] == T.depth
    # node covariances: the oracle's collapse of the oracle's levels
    lv = ot.build(g.w, g.U, g.S)
    covs = {}
    # map builder nodes back to (level, index) through the leaves' ancestry
    for v in leaves:
        k = T.leaf_component[v]
        u, lev_idx = v, k
        for L, (w_l, c_l, parts) in enumerate(lv):
            u = parent[u]
            lev_idx = next(i for i, p in enumerate(parts) if lev_idx in p)
            covs[u] = (c_l[lev_idx], w_l[lev_idx])
    for u, (c, wl) in covs.items():
        rec = T.eigvecs[u] @ np.diag(T.eigvals[u]) @ T.eigvecs[u].T
        assert np.abs(rec - c).max() <= 1e-10 * np.abs(c).max()
        assert abs(T.weights[u] - wl) <= 1e-12
        assert np.all(np.diff(T.eigvals[u]) <= 0)


def test_paper_level_structure_at_k200():
    g = synth.synthetic_gmm(200)
    T = pt.build_tree(g.w, g.U, g.S)
    assert T.n_nodes == 327 and T.depth == 7
    sizes = [sorted({len(c) for c in p}) for p in T.levels]
    assert sizes[0] in ([3, 4], [3], [4]) and all(s == [2] for s in sizes[1:])
