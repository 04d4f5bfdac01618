"""Seed-selection workload variants (the paper's seed-selection study):
BFS levels against scipy's BFS, and the structural property each strategy
is defined by.  Input generation only; no Steiner arithmetic."""
import numpy as np
import pytest

import paper_2205_14503_gb300.workloads as wl

scipy_csgraph = pytest.importorskip("scipy.sparse.csgraph")
scipy_sparse = pytest.importorskip("scipy.sparse")


def _scipy_levels(g, root):
    a = scipy_sparse.csr_matrix((np.ones(g.n_arcs), g.col, g.row_ptr.astype(np.int64)),
                                shape=(g.n, g.n))
    d = scipy_csgraph.shortest_path(a, unweighted=True, indices=[root])[0]
    return np.where(np.isinf(d), -1, d).astype(np.int64)


def test_bfs_levels_match_scipy():
    g = wl.rmat(12, 8, wmax=50, seed=71)
    for root in (0, 17, int(wl.largest_cc(g)[5])):
        np.testing.assert_array_equal(wl.bfs_levels(g, root), _scipy_levels(g, root))


def test_bfs_level_seeds_follow_level_sizes():
    g = wl.grid(40, 30, 100, seed=72)
    pool = np.arange(g.n, dtype=np.int32)
    k = 120
    s = wl.seeds_bfs_level(g, pool, k, 9)
    assert s.size == k and np.unique(s).size == k and np.isin(s, pool).all()
    root = int(wl.sample_distinct(pool, 1, 9)[0])
    lvl = wl.bfs_levels(g, root)
    levels, counts = np.unique(lvl[pool], return_counts=True)
    got = np.array([(lvl[s] == L).sum() for L in levels])
    quota = counts * k / counts.sum()
    assert (np.abs(got - quota) < 1.0).all()          # floor or ceil of each quota
    np.testing.assert_array_equal(s, wl.seeds_bfs_level(g, pool, k, 9))   # seeded


def test_k_bfs_choices_follow_the_level_sums():
    """Each k-BFS source is the pool vertex with the largest (eccentric) or
    smallest (proximate) sum of BFS levels from the sources before it
    (ties: smallest id); proximate seeds form a tight cluster."""
    g = wl.grid(50, 50, 100, seed=73)
    pool = np.arange(g.n, dtype=np.int32)
    k = 9
    for far in (True, False):
        s = (wl.seeds_eccentric if far else wl.seeds_proximate)(g, pool, k, 4)
        assert s.size == k and np.unique(s).size == k and np.isin(s, pool).all()
        acc = np.zeros(g.n, dtype=np.int64)
        for i in range(1, k):
            acc += wl.bfs_levels(g, int(s[i - 1]))
            score = acc.astype(np.float64)
            score[s[:i]] = -np.inf if far else np.inf
            best = np.argmax(score) if far else np.argmin(score)
            assert s[i] == best, (far, i)
        if not far:
            assert max(int(wl.bfs_levels(g, int(a))[s].max()) for a in s) <= 4
    # the second eccentric source is the vertex farthest from the first
    e = wl.seeds_eccentric(g, pool, 2, 4)
    lvl0 = wl.bfs_levels(g, int(e[0]))
    assert lvl0[e[1]] == lvl0.max()


def test_k_bfs_on_a_path():
    g = wl.from_edges(6, [0, 1, 2, 3, 4], [1, 2, 3, 4, 5], [1, 1, 1, 1, 1])
    pool = np.arange(6, dtype=np.int32)
    first = int(wl.sample_distinct(pool, 1, 5)[0])
    far = wl.seeds_eccentric(g, pool, 3, 5)
    near = wl.seeds_proximate(g, pool, 3, 5)
    assert far[0] == near[0] == first
    ends = {0, 5}
    assert set(far[1:].tolist()) <= ends | {first}
    assert np.ptp(near) == 2                          # three consecutive vertices
