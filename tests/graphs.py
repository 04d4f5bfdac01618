"""Small seeded test graphs (inputs only; no Steiner arithmetic here)."""
import numpy as np

import paper_2205_14503_gb300.workloads as wl


def rng(seed):
    return np.random.default_rng(seed)


def random_graph(n, m, wlo, whi, seed, name="random"):
    r = rng(seed)
    u = r.integers(0, n, m)
    v = r.integers(0, n, m)
    w = r.integers(wlo, whi + 1, m)
    return wl.from_edges(n, u, v, w, name)


def random_connected(n, extra, wlo, whi, seed):
    """Random spanning tree plus ``extra`` random edges."""
    r = rng(seed)
    perm = r.permutation(n)
    parents = [perm[r.integers(0, i)] for i in range(1, n)]
    u = list(perm[1:]) + list(r.integers(0, n, extra))
    v = parents + list(r.integers(0, n, extra))
    w = r.integers(wlo, whi + 1, len(u))
    return wl.from_edges(n, np.array(u), np.array(v), w, "connected")


def random_tree(n, wlo, whi, seed):
    r = rng(seed)
    perm = r.permutation(n)
    u = perm[1:]
    v = np.array([perm[r.integers(0, i)] for i in range(1, n)])
    w = r.integers(wlo, whi + 1, n - 1)
    return wl.from_edges(n, u, v, w, "tree")


def path(n, wlo, whi, seed):
    r = rng(seed)
    u = np.arange(n - 1)
    return wl.from_edges(n, u, u + 1, r.integers(wlo, whi + 1, n - 1), "path")


def star(n, wlo, whi, seed):
    r = rng(seed)
    v = np.arange(1, n)
    return wl.from_edges(n, np.zeros(n - 1, np.int64), v, r.integers(wlo, whi + 1, n - 1), "star")


def complete(n, wlo, whi, seed):
    r = rng(seed)
    iu, iv = np.triu_indices(n, 1)
    return wl.from_edges(n, iu, iv, r.integers(wlo, whi + 1, iu.size), "complete")


def seeds_from(pool, k, seed):
    r = rng(seed)
    return r.choice(np.asarray(pool), size=k, replace=False).astype(np.int32)


def to_scipy(g):
    import scipy.sparse as sp
    return sp.csr_matrix((g.w.astype(np.float64), g.col.astype(np.int64),
                          g.row_ptr.astype(np.int64)), shape=(g.n, g.n))


def undirected_edges(g):
    """(u, v, w) arrays with u < v, one row per undirected edge."""
    rp = g.row_ptr.astype(np.int64)
    src = np.repeat(np.arange(g.n), np.diff(rp))
    keep = src < g.col
    return src[keep], g.col[keep].astype(np.int64), g.w[keep].astype(np.int64)
