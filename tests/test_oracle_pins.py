"""Pins for the CPU oracle: each test checks it against something other than
itself — hand-worked examples, per-seed Dijkstra from scipy, Mehlhorn's
theorem, the textbook MST (scipy) for S = V, closed forms on paths and
trees, Dreyfus-Wagner optima on tiny graphs, and structural invariants.
"""
import itertools
import json
import os

import numpy as np
import pytest
import scipy.sparse.csgraph as csg

import oracle
import paper_2205_14503_gb300.workloads as wl
from tests import graphs as G

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
INF = 0xFFFFFFFF

# The oracle library under test.  None = the committed oracle; the mutation
# tests swap in copies with planted mistakes and expect these pins to fail.
LIB = None


def _steiner(g, seeds, **kw):
    return oracle.steiner(g, seeds, lib=LIB, **kw)


def _voronoi(g, seeds):
    return oracle.voronoi(g, seeds, lib=LIB)


def _seed_dists(g, seeds):
    """d_G(s, v) for every seed s (rows in ascending seed order)."""
    ss = np.sort(np.asarray(seeds))
    return ss, csg.dijkstra(G.to_scipy(g), directed=True, indices=ss)


def _arc_id(g, u, v):
    lo, hi = int(g.row_ptr[u]), int(g.row_ptr[u + 1])
    idx = lo + int(np.searchsorted(g.col[lo:hi], v))
    assert idx < hi and g.col[idx] == v
    return idx


def _cases():
    yield "rmat9", wl.rmat(9, 8, wmax=100, seed=11), 12
    yield "rmat9_unit", wl.rmat(9, 8, wmax=1, seed=12), 9
    yield "rmat10_w3", wl.rmat(10, 4, wmax=3, seed=13), 30
    yield "grid", wl.grid(23, 17, 1000, seed=14), 7
    yield "grid_unit", wl.grid(16, 16, 1, seed=15), 5
    yield "connected", G.random_connected(300, 200, 1, 50, 16), 20
    yield "complete", G.complete(25, 1, 10, 17), 6
    yield "disconnected", G.random_graph(400, 300, 1, 20, 18), 25
    yield "star", G.star(50, 1, 5, 19), 10
    yield "path", G.path(60, 1, 9, 20), 4


CASES = list(_cases())


# ---------------------------------------------------------------------------
# hand-worked examples
# ---------------------------------------------------------------------------

def _worked_examples():
    """The hand-worked fixtures (each carries its derivation); the other
    JSON files in golden/ are oracle-written digests of the full-size
    workloads, checked by the GPU tests."""
    out = []
    for f in sorted(os.listdir(GOLDEN)):
        if f.endswith(".json"):
            with open(os.path.join(GOLDEN, f)) as fh:
                if "derivation" in json.load(fh):
                    out.append(f)
    return out


WORKED = _worked_examples()


@pytest.mark.parametrize("fname", WORKED)
def test_golden_worked_example(fname):
    ex = json.load(open(os.path.join(GOLDEN, fname)))
    e = np.array(ex["edges"])
    g = wl.from_edges(ex["n"], e[:, 0], e[:, 1], e[:, 2])
    r = _steiner(g, ex["seeds"], want_labels=True, want_pairs=True)
    assert r.status == oracle.OK
    assert r.cell.tolist() == ex["cell"]
    assert r.dist.tolist() == ex["dist"]
    assert r.pred.tolist() == ex["pred"]
    want_pairs = []
    for ra, rb, b, arc in ex["pairs"]:
        u, v = (int(x) for x in arc.split("->"))
        want_pairs.append([ra, rb, b, _arc_id(g, u, v)])
    assert r.pairs.tolist() == want_pairs
    assert int(r.mst[:, 2].sum()) == ex["mst_weight"]
    assert r.edges.tolist() == ex["tree"]
    assert r.total == ex["total"]


# ---------------------------------------------------------------------------
# Step 1: Voronoi cells against per-seed Dijkstra (scipy)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,g,k", CASES, ids=[c[0] for c in CASES])
def test_voronoi_equals_min_over_seed_dijkstra(name, g, k):
    seeds = G.seeds_from(np.arange(g.n), k, 100 + k)
    ss, D = _seed_dists(g, seeds)
    v = _voronoi(g, seeds)
    assert v.status == oracle.OK
    dmin = D.min(axis=0)
    reached = np.isfinite(dmin)
    # argmin returns the first minimum: the smallest seed id among ties
    want_cell = np.where(reached, ss[np.argmin(D, axis=0)], -1)
    want_dist = np.where(reached, dmin, INF).astype(np.uint64)
    assert np.array_equal(v.dist.astype(np.uint64), want_dist)
    assert np.array_equal(v.cell, want_cell)


@pytest.mark.parametrize("name,g,k", CASES, ids=[c[0] for c in CASES])
def test_pred_chains_are_shortest_paths_to_own_seed(name, g, k):
    seeds = G.seeds_from(np.arange(g.n), k, 200 + k)
    v = _voronoi(g, seeds)
    ss, D = _seed_dists(g, seeds)
    seed_set = set(int(s) for s in seeds)
    for x in range(g.n):
        if v.cell[x] < 0:
            assert v.pred[x] == -1
            continue
        if x in seed_set:
            assert v.pred[x] == x
            continue
        # walk to the seed, summing edge weights: must equal d_G(cell, x)
        y, total, hops = x, 0, 0
        while y not in seed_set:
            p = int(v.pred[y])
            assert v.cell[p] == v.cell[x]
            total += int(g.w[_arc_id(g, y, p)])
            y, hops = p, hops + 1
            assert hops <= g.n
        assert y == v.cell[x]
        assert total == D[np.searchsorted(ss, v.cell[x]), x]
        # tie rule: no smaller-id neighbour is tight inside the cell
        lo, hi = int(g.row_ptr[x]), int(g.row_ptr[x + 1])
        for e in range(lo, hi):
            u = int(g.col[e])
            if u >= v.pred[x]:
                break
            assert not (v.cell[u] == v.cell[x] and int(v.dist[u]) + int(g.w[e]) == int(v.dist[x]))


# ---------------------------------------------------------------------------
# Step 2 + 3: distance graph and MST (Mehlhorn's theorem)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,g,k", CASES, ids=[c[0] for c in CASES])
def test_mehlhorn_mst_weight_equals_kmb_mst_weight(name, g, k):
    """Every MST of G'_1 is an MST of G_1 (Section 'Preliminaries'): the
    oracle's MST weight equals scipy's MST of the complete seed distance
    graph G_1 built from per-seed Dijkstra.  Per connected component of
    seeds when the input is disconnected (spanning forests)."""
    seeds = G.seeds_from(np.arange(g.n), k, 300 + k)
    r = _steiner(g, seeds, want_pairs=True)
    assert r.status in (oracle.OK, oracle.EDISCONNECTED)
    ss, D = _seed_dists(g, seeds)
    G1 = D[:, ss]
    G1 = np.where(np.isfinite(G1), G1, 0.0)
    kmb = csg.minimum_spanning_tree(G1).sum()
    assert int(r.mst[:, 2].sum()) == int(kmb)
    # d'_1 >= d_G on every pair, and equality on MST pairs is not required
    for ra, rb, b, arc in r.pairs.tolist():
        assert b >= G1[ra, rb]
    # a pair is present exactly when some edge joins the two cells
    eu, ev, _ = G.undirected_edges(g)
    rank = {int(s): i for i, s in enumerate(ss)}
    cu, cv = r.cell[eu], r.cell[ev]
    want = set()
    for a, b in zip(cu.tolist(), cv.tolist()):
        if a >= 0 and b >= 0 and a != b:
            want.add((min(rank[a], rank[b]), max(rank[a], rank[b])))
    assert set((int(a), int(b)) for a, b in r.pairs[:, :2].tolist()) == want


def test_bridge_minimum_by_enumeration():
    """Brute force over all cross edges of d1(s,u)+d(u,v)+d1(v,t), with the
    (b, arc) tie rule, on unit weights where ties abound."""
    g = wl.grid(12, 9, 1, seed=3)
    seeds = G.seeds_from(np.arange(g.n), 6, 9)
    r = _steiner(g, seeds, want_pairs=True)
    ss = np.sort(seeds)
    rank = {int(s): i for i, s in enumerate(ss)}
    best = {}
    for u in range(g.n):
        for e in range(int(g.row_ptr[u]), int(g.row_ptr[u + 1])):
            v = int(g.col[e])
            a, b = rank[int(r.cell[u])], rank[int(r.cell[v])]
            if a < b:
                key = (int(r.dist[u]) + int(g.w[e]) + int(r.dist[v]), e)
                best[(a, b)] = min(best.get((a, b), key), key)
    got = {(int(a), int(b)): (int(c), int(d)) for a, b, c, d in r.pairs.tolist()}
    assert got == best


def test_two_seed_distance_graph_edge_is_shortest_path():
    g = G.random_connected(200, 400, 1, 30, 4)
    for trial in range(5):
        s = G.seeds_from(np.arange(g.n), 2, trial)
        r = _steiner(g, s, want_pairs=True)
        d = csg.dijkstra(G.to_scipy(g), indices=int(s[0]))[int(s[1])]
        assert r.pairs.shape[0] == 1 and int(r.pairs[0, 2]) == int(d)


# ---------------------------------------------------------------------------
# end-to-end closed forms and bounds
# ---------------------------------------------------------------------------

def _check_tree(g, seeds, r, connected=True):
    edges = r.edges.astype(np.int64)
    assert np.all(edges[:, 0] < edges[:, 1])
    keys = edges[:, 0] * g.n + edges[:, 1]
    assert np.all(np.diff(keys) > 0), "edges sorted ascending and unique"
    for u, v, w in edges.tolist():
        assert int(g.w[_arc_id(g, u, v)]) == w
    assert int(edges[:, 2].sum()) == r.total
    verts = set(edges[:, :2].ravel().tolist()) | set(int(s) for s in seeds)
    # acyclic + connectivity via union-find
    parent = {x: x for x in verts}

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x
    for u, v, _ in edges.tolist():
        a, b = find(u), find(v)
        assert a != b, "cycle"
        parent[a] = b
    roots = {find(x) for x in verts}
    if connected:
        assert len(roots) == 1
        assert len(edges) == len(verts) - 1
    deg = {}
    for u, v, _ in edges.tolist():
        deg[u] = deg.get(u, 0) + 1
        deg[v] = deg.get(v, 0) + 1
    seed_set = set(int(s) for s in seeds)
    for x, d in deg.items():
        if d == 1:
            assert x in seed_set, "every leaf is a seed"


@pytest.mark.parametrize("name,g,k", CASES, ids=[c[0] for c in CASES])
def test_tree_invariants_and_kmb_bound(name, g, k):
    seeds = G.seeds_from(np.arange(g.n), k, 400 + k)
    r = _steiner(g, seeds)
    ss, D = _seed_dists(g, seeds)
    if r.status == oracle.EDISCONNECTED:
        _check_tree(g, seeds, r, connected=False)
        return
    assert r.status == oracle.OK
    _check_tree(g, seeds, r)
    kmb = csg.minimum_spanning_tree(D[:, ss]).sum()
    assert r.total <= kmb


def test_two_seeds_give_a_shortest_path():
    """With |S| = 2 the tree is a shortest s-t path (Section 'Introduction')."""
    for seed in range(6):
        g = G.random_connected(150, 300, 1, 40, seed)
        s = G.seeds_from(np.arange(g.n), 2, 50 + seed)
        r = _steiner(g, s)
        d = csg.dijkstra(G.to_scipy(g), indices=int(s[0]))[int(s[1])]
        assert r.total == int(d)
        deg = np.bincount(r.edges[:, :2].ravel().astype(np.int64), minlength=g.n)
        assert set(np.flatnonzero(deg == 1).tolist()) == set(int(x) for x in s)
        assert deg.max() <= 2


def test_seed_set_equal_to_vertex_set_gives_textbook_mst():
    """S = V: every cell is a single vertex, G'_1 = G, so the tree is the MST
    of G.  Distinct weights make the MST unique: the edge set must equal
    scipy's."""
    for seed in range(4):
        n = 120
        r_ = np.random.default_rng(seed)
        iu, iv = np.triu_indices(n, 1)
        pick = r_.random(iu.size) < 0.08
        iu, iv = iu[pick], iv[pick]
        w = r_.permutation(iu.size) + 1        # distinct weights
        g = wl.from_edges(n, iu, iv, w)
        comp, rep, size = wl.components(g)
        if size != n:
            continue
        r = _steiner(g, np.arange(n))
        assert r.status == oracle.OK
        mst = csg.minimum_spanning_tree(G.to_scipy(g)).tocoo()
        want = sorted((min(a, b), max(a, b)) for a, b in zip(mst.row.tolist(), mst.col.tolist()))
        assert r.edges[:, :2].tolist() == [list(x) for x in want]
        assert r.total == int(mst.sum())


def test_seed_set_equal_to_vertex_set_with_ties():
    """S = V with unit and {1,2} weights: total equals the MST weight."""
    for wmax in (1, 2):
        g = wl.grid(11, 7, wmax, seed=wmax)
        r = _steiner(g, np.arange(g.n))
        assert r.status == oracle.OK
        assert r.total == int(csg.minimum_spanning_tree(G.to_scipy(g)).sum())
        assert r.edges.shape[0] == g.n - 1


def _prune_to_steiner_subtree(g, seeds):
    """Minimal subtree of a tree graph spanning the seeds (leaf pruning)."""
    eu, ev, ew = G.undirected_edges(g)
    adj = {x: {} for x in range(g.n)}
    for a, b, c in zip(eu.tolist(), ev.tolist(), ew.tolist()):
        adj[a][b] = c
        adj[b][a] = c
    seed_set = set(int(s) for s in seeds)
    stack = [x for x in adj if len(adj[x]) == 1 and x not in seed_set]
    while stack:
        x = stack.pop()
        if x in seed_set or len(adj[x]) != 1:
            continue
        (y, _), = adj[x].items()
        del adj[y][x]
        del adj[x]
        if len(adj[y]) == 1 and y not in seed_set:
            stack.append(y)
    return sum(c for a in adj for b, c in adj[a].items() if a < b)


def test_tree_shaped_graph_gives_the_exact_steiner_tree():
    for seed in range(8):
        g = G.random_tree(200, 1, 100, seed)
        s = G.seeds_from(np.arange(g.n), 3 + seed, seed)
        r = _steiner(g, s)
        assert r.status == oracle.OK
        assert r.total == _prune_to_steiner_subtree(g, s)


def dreyfus_wagner(g, terminals):
    """Exact Steiner minimal tree weight (Dreyfus-Wagner dynamic programme)."""
    D = csg.floyd_warshall(G.to_scipy(g), directed=False)
    t = list(terminals)
    k = len(t)
    full = (1 << k) - 1
    dp = np.full((1 << k, g.n), np.inf)
    for i in range(k):
        dp[1 << i] = D[t[i]]
    for mask in range(1, full + 1):
        if mask & (mask - 1) == 0:
            continue
        best = np.full(g.n, np.inf)
        sub = (mask - 1) & mask
        while sub:
            if sub < (mask ^ sub):
                best = np.minimum(best, dp[sub] + dp[mask ^ sub])
            sub = (sub - 1) & mask
        dp[mask] = (best[:, None] + D).min(axis=0)
    return dp[full].min()


def test_dreyfus_wagner_two_approximation_bound():
    """OPT <= D <= 2 (1 - 1/|S|) OPT (Takahashi/KMB bound) on tiny graphs."""
    checked = 0
    for seed in range(40):
        n = 12 + seed % 8
        g = G.random_connected(n, n, 1, 12, seed)
        k = 3 + seed % 4
        s = G.seeds_from(np.arange(n), k, seed)
        r = _steiner(g, s)
        assert r.status == oracle.OK
        opt = dreyfus_wagner(g, s.tolist())
        assert opt - 1e-9 <= r.total <= 2 * (1 - 1 / k) * opt + 1e-9
        checked += 1
    assert checked == 40


def test_result_does_not_depend_on_seed_order():
    g = wl.rmat(10, 8, wmax=20, seed=21)
    s = wl.sample_distinct(wl.largest_cc(g), 15, 5)
    base = _steiner(g, s)
    for p in itertools.islice(itertools.permutations(range(15)), 0, 40, 13):
        r = _steiner(g, s[list(p)])
        assert r.total == base.total and np.array_equal(r.edges, base.edges)
        assert np.array_equal(r.cell, base.cell) and np.array_equal(r.pred, base.pred)


# ---------------------------------------------------------------------------
# degenerate cases and errors
# ---------------------------------------------------------------------------

def test_single_seed_gives_empty_tree():
    g = wl.grid(5, 5, 9, seed=1)
    r = _steiner(g, [12])
    assert r.status == oracle.OK and r.edges.shape[0] == 0 and r.total == 0
    assert r.dist[12] == 0 and np.all(r.cell == 12)


def test_invalid_seed_lists():
    g = wl.grid(5, 5, 9, seed=1)
    assert _steiner(g, []).status == oracle.EINVAL
    assert _steiner(g, [3, 3]).status == oracle.EINVAL
    assert _steiner(g, [25]).status == oracle.EINVAL
    assert _steiner(g, [-1, 2]).status == oracle.EINVAL


def test_disconnected_seeds_give_a_spanning_forest():
    e = np.array([[0, 1, 3], [1, 2, 4], [3, 4, 5], [4, 5, 1]])
    g = wl.from_edges(7, e[:, 0], e[:, 1], e[:, 2])
    r = _steiner(g, [0, 2, 3, 5])
    assert r.status == oracle.EDISCONNECTED
    assert r.edges.tolist() == [[0, 1, 3], [1, 2, 4], [3, 4, 5], [4, 5, 1]]
    assert r.total == 13
    assert r.cell[6] == -1 and r.dist[6] == INF and r.pred[6] == -1


def test_distance_overflow_is_reported():
    big = 0xFFFFFFFF // 2 + 1
    g = wl.from_edges(4, [0, 1, 2], [1, 2, 3], [big, big, 5])
    assert _steiner(g, [0, 3]).status == oracle.EOVERFLOW
    # bridge sum overflow with in-range distances
    g = wl.from_edges(2, [0], [1], [0xFFFFFFFF - 1])
    assert _steiner(g, [0, 1]).status == oracle.OK
    g = wl.from_edges(3, [0, 1], [1, 2], [0xFFFFFFFE, 1])
    assert _steiner(g, [0, 2]).status == oracle.EOVERFLOW


def test_check_graph_rejects_malformed_csr():
    g = wl.grid(4, 4, 9, seed=1)
    assert oracle.check_graph(g, lib=LIB) == oracle.OK
    bad = wl.Graph(g.n, g.row_ptr.copy(), g.col.copy(), g.w.copy())
    bad.w[3] = 0
    assert oracle.check_graph(bad, lib=LIB) == oracle.EINVAL
    bad = wl.Graph(g.n, g.row_ptr.copy(), g.col.copy(), g.w.copy())
    bad.w[3] += 1                        # asymmetric weight
    assert oracle.check_graph(bad, lib=LIB) == oracle.EINVAL
    bad = wl.Graph(g.n, g.row_ptr.copy(), g.col.copy(), g.w.copy())
    bad.col[0], bad.col[1] = bad.col[1], bad.col[0]   # unsorted row
    assert oracle.check_graph(bad, lib=LIB) == oracle.EINVAL
    bad = wl.Graph(g.n, g.row_ptr.copy(), g.col.copy(), g.w.copy())
    bad.col[0] = 0                       # self-loop on vertex 0
    assert oracle.check_graph(bad, lib=LIB) == oracle.EINVAL
