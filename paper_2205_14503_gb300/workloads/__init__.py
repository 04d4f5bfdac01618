"""Seeded synthetic workloads: graphs, seed sets and query streams.

The paper evaluates on real graphs (Table "evaluation_datasets": web, social,
citation and co-author graphs with symmetric arcs and positive integer
weights in ranges such as [1, 5K] ... [1, 500K]).  Those datasets are not
available here, so seeded synthetic graphs of the same structure stand in:
R-MAT graphs for the scale-free web/social graphs and 2-D grids for the
high-diameter case.  Seeds are drawn uniformly from the largest connected
component, the uniform-random strategy of the paper's seed-selection study.

This module holds input generation only and none of the Steiner-tree
arithmetic; the CPU oracle's tests and the CUDA path's tests both take their
inputs from here.  The heavy lifting is in ``gen.c`` (compiled with gcc into
``_libworkloads.so`` by :func:`build`), driven by a counter-based splitmix64
generator so that every graph is identical on any host and thread count.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "_libworkloads.so")
_lib = None

GOLDEN = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1


def build(force: bool = False) -> str:
    """Compile gen.c into a shared library next to this file."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-pthread", "-std=c11",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    u32, u64, i32, vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
    lib.wl_splitmix64.restype = u64
    lib.wl_splitmix64.argtypes = [u64, u64]
    lib.wl_rmat_begin.restype = vp
    lib.wl_rmat_begin.argtypes = [i32, u64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  u32, u64, i32, i32, ctypes.POINTER(u64)]
    lib.wl_grid_begin.restype = vp
    lib.wl_grid_begin.argtypes = [u32, u32, u32, u64, i32, ctypes.POINTER(u64)]
    lib.wl_edges_begin.restype = vp
    lib.wl_edges_begin.argtypes = [u32, u64, vp, vp, vp, i32, ctypes.POINTER(u64)]
    lib.wl_finish.restype = i32
    lib.wl_finish.argtypes = [vp, vp, vp, vp]
    lib.wl_abort.restype = None
    lib.wl_abort.argtypes = [vp]
    lib.wl_components.restype = ctypes.c_int64
    lib.wl_components.argtypes = [u32, vp, vp, vp, i32, ctypes.POINTER(u64)]
    lib.wl_bfs_levels.restype = ctypes.c_int64
    lib.wl_bfs_levels.argtypes = [u32, vp, vp, u32, vp]
    _lib = lib
    return lib


def _threads(nthreads: int | None) -> int:
    if nthreads:
        return int(nthreads)
    return max(1, min(64, os.cpu_count() or 1))


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


@dataclass
class Graph:
    """Symmetric weighted CSR graph (adjacency rows sorted by neighbour id)."""

    n: int
    row_ptr: np.ndarray      # uint32[n + 1]
    col: np.ndarray          # int32[n_arcs]
    w: np.ndarray            # uint32[n_arcs]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_arcs(self) -> int:
        return int(self.col.shape[0])

    @property
    def n_edges(self) -> int:
        return self.n_arcs // 2


def _finish(handle, n: int, n_arcs: int, name: str, meta: dict) -> Graph:
    lib = _load()
    row_ptr = np.empty(n + 1, dtype=np.uint32)
    col = np.empty(max(n_arcs, 1), dtype=np.int32)
    w = np.empty(max(n_arcs, 1), dtype=np.uint32)
    rc = lib.wl_finish(handle, _ptr(row_ptr), _ptr(col), _ptr(w))
    if rc != 0:
        raise ValueError(f"CSR build failed ({rc}): arc count {n_arcs} does not fit uint32 offsets")
    return Graph(n, row_ptr, col[:n_arcs], w[:n_arcs], name, meta)


def rmat(scale: int, edge_factor: int = 16, abc=(0.57, 0.19, 0.19), wmax: int = 100,
         seed: int = 0x5EED, permute: bool = True, nthreads: int | None = None) -> Graph:
    """R-MAT graph with 2**scale vertices and edge_factor * 2**scale edge draws.

    Quadrant probabilities (a, b, c, 1-a-b-c); no noise.  A seeded bijective
    relabelling scatters the hubs over the id range (Graph500 practice).
    Weight of each drawn edge is uniform in [1, wmax].
    """
    lib = _load()
    arcs = ctypes.c_uint64(0)
    a, b, c = abc
    h = lib.wl_rmat_begin(scale, edge_factor, a, b, c, wmax, seed & MASK64, int(permute),
                          _threads(nthreads), ctypes.byref(arcs))
    if not h:
        raise MemoryError("R-MAT generation failed")
    meta = dict(kind="rmat", scale=scale, edge_factor=edge_factor, abc=tuple(abc), wmax=wmax,
                seed=seed, permute=permute)
    return _finish(h, 1 << scale, arcs.value, f"rmat{scale}", meta)


def grid(width: int, height: int, wmax: int = 1000, seed: int = 0x5EED,
         nthreads: int | None = None) -> Graph:
    """4-connected width x height grid; vertex id = row * width + col."""
    lib = _load()
    arcs = ctypes.c_uint64(0)
    h = lib.wl_grid_begin(width, height, wmax, seed & MASK64, _threads(nthreads), ctypes.byref(arcs))
    if not h:
        raise MemoryError("grid generation failed")
    meta = dict(kind="grid", width=width, height=height, wmax=wmax, seed=seed)
    return _finish(h, width * height, arcs.value, f"grid{width}x{height}", meta)


def from_edges(n: int, u, v, w, name: str = "edges") -> Graph:
    """Symmetric CSR from an undirected edge list (self-loops dropped,
    parallel edges merged to the minimum weight)."""
    lib = _load()
    u = np.ascontiguousarray(u, dtype=np.uint32)
    v = np.ascontiguousarray(v, dtype=np.uint32)
    w = np.ascontiguousarray(w, dtype=np.uint32)
    if not (u.shape == v.shape == w.shape):
        raise ValueError("edge arrays differ in length")
    arcs = ctypes.c_uint64(0)
    h = lib.wl_edges_begin(n, u.shape[0], _ptr(u), _ptr(v), _ptr(w), 1, ctypes.byref(arcs))
    if not h:
        raise ValueError("edge endpoint out of range")
    return _finish(h, n, arcs.value, name, dict(kind="edges"))


def components(g: Graph, nthreads: int | None = None):
    """(comp, representative of the largest component, its size).

    comp[v] is the smallest vertex id in v's connected component.
    """
    lib = _load()
    comp = np.empty(max(g.n, 1), dtype=np.uint32)
    size = ctypes.c_uint64(0)
    rep = lib.wl_components(g.n, _ptr(g.row_ptr), _ptr(g.col), _ptr(comp), _threads(nthreads),
                            ctypes.byref(size))
    if rep < 0 and g.n > 0:
        raise MemoryError("component labelling failed")
    return comp[: g.n], int(rep), int(size.value)


def largest_cc(g: Graph) -> np.ndarray:
    """Ascending vertex ids of the largest connected component."""
    comp, rep, _ = components(g)
    return np.flatnonzero(comp == rep).astype(np.int32)


# ---------------------------------------------------------------------------
# counter-based draws for seeds and query streams (same splitmix64 as gen.c)
# ---------------------------------------------------------------------------

def splitmix64(seed: int, ctr) -> np.ndarray:
    """Vectorised splitmix64 output for counters ``ctr`` (uint64 wraparound)."""
    ctr = np.asarray(ctr, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + (ctr + np.uint64(1)) * np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, ctr) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits."""
    return (splitmix64(seed, ctr) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def sample_distinct(pool: np.ndarray, k: int, seed: int) -> np.ndarray:
    """k distinct elements drawn uniformly from ``pool`` (in draw order)."""
    pool = np.asarray(pool)
    if k > pool.shape[0]:
        raise ValueError(f"cannot draw {k} distinct from {pool.shape[0]}")
    out, seen, ctr = [], set(), 0
    while len(out) < k:
        batch = max(64, 2 * (k - len(out)))
        x = splitmix64(seed, np.arange(ctr, ctr + batch, dtype=np.uint64))
        ctr += batch
        idx = ((x >> np.uint64(32)) * np.uint64(pool.shape[0])) >> np.uint64(32)
        for i in idx.tolist():
            if i not in seen:
                seen.add(i)
                out.append(i)
                if len(out) == k:
                    break
    return pool[np.asarray(out, dtype=np.int64)].astype(np.int32)


def log_uniform_sizes(q: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """q sizes floor(exp(U(ln lo, ln(hi + 1)))) clipped to [lo, hi]."""
    u = uniform01(seed, np.arange(q, dtype=np.uint64))
    k = np.floor(np.exp(math.log(lo) + u * (math.log(hi + 1) - math.log(lo))))
    return np.clip(k, lo, hi).astype(np.int64)


def poisson_arrivals(q: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process of the given rate."""
    u = uniform01(seed, np.arange(q, dtype=np.uint64))
    gaps = -np.log1p(-u) / rate
    return np.cumsum(gaps)


# ---------------------------------------------------------------------------
# seed-selection variants (the paper's seed-selection study): uniform random
# is sample_distinct over the largest component; the others are below
# ---------------------------------------------------------------------------

def bfs_levels(g: Graph, root: int) -> np.ndarray:
    """Hop counts from ``root`` (int64; -1 where unreachable)."""
    lvl = np.empty(g.n, dtype=np.uint32)
    rc = _load().wl_bfs_levels(g.n, _ptr(g.row_ptr), _ptr(g.col), int(root), _ptr(lvl))
    if rc < 0:
        raise ValueError("bad BFS root")
    out = lvl.astype(np.int64)
    out[lvl == np.uint32(0xFFFFFFFF)] = -1
    return out


def seeds_bfs_level(g: Graph, pool: np.ndarray, k: int, seed: int) -> np.ndarray:
    """k seeds spread over the BFS levels of a random root of ``pool`` (one
    component): each level contributes in proportion to its size (largest
    remainders), drawn uniformly within the level."""
    pool = np.asarray(pool)
    root = int(sample_distinct(pool, 1, seed)[0])
    lvl = bfs_levels(g, root)[pool]
    levels, counts = np.unique(lvl, return_counts=True)
    quota = counts * k / counts.sum()
    take = np.floor(quota).astype(np.int64)
    rest = k - int(take.sum())
    order = np.lexsort((levels, -(quota - take)))       # largest remainders, then lower level
    take[order[:rest]] += 1
    out = []
    for i, (L, t) in enumerate(zip(levels.tolist(), take.tolist())):
        if t:
            out.append(sample_distinct(pool[lvl == L], t, seed + 1 + i))
    return np.concatenate(out).astype(np.int32)


def _k_bfs(g: Graph, pool: np.ndarray, k: int, seed: int, far: bool) -> np.ndarray:
    pool = np.asarray(pool)
    first = int(sample_distinct(pool, 1, seed)[0])
    inside = np.zeros(g.n, dtype=bool)
    inside[pool] = True
    acc = np.zeros(g.n, dtype=np.int64)
    chosen = [first]
    taken = np.zeros(g.n, dtype=bool)
    taken[first] = True
    for _ in range(k - 1):
        acc += bfs_levels(g, chosen[-1])
        score = acc.astype(np.float64)
        score[~inside | taken] = -np.inf if far else np.inf
        nxt = int(np.argmax(score) if far else np.argmin(score))   # ties: smallest id
        chosen.append(nxt)
        taken[nxt] = True
    return np.asarray(chosen, dtype=np.int32)


def seeds_eccentric(g: Graph, pool: np.ndarray, k: int, seed: int) -> np.ndarray:
    """k-BFS sources far apart: from a random first source, each next one is
    the vertex of ``pool`` (one component) with the largest sum of BFS levels
    from the sources chosen so far."""
    return _k_bfs(g, pool, k, seed, far=True)


def seeds_proximate(g: Graph, pool: np.ndarray, k: int, seed: int) -> np.ndarray:
    """As seeds_eccentric with the smallest sum: seeds close together."""
    return _k_bfs(g, pool, k, seed, far=False)


# ---------------------------------------------------------------------------
# the five evaluation workloads
# ---------------------------------------------------------------------------

CONFIG_SEED = 0x5EED

CONFIGS = {
    1: dict(name="rmat16_k16", kind="rmat", scale=16, wmax=100, k=16),
    2: dict(name="grid4096_k256", kind="grid", side=4096, wmax=1000, k=256),
    3: dict(name="rmat26_k10000", kind="rmat", scale=26, wmax=1000, k=10000),
    4: dict(name="rmat22_batch64", kind="rmat", scale=22, wmax=1000, queries=64, klo=3, khi=1000),
    5: dict(name="rmat24_serve2000", kind="rmat", scale=24, wmax=1000, queries=2000, klo=3, khi=10000),
}


def config_graph(idx: int, nthreads: int | None = None) -> Graph:
    c = CONFIGS[idx]
    seed = CONFIG_SEED + idx
    if c["kind"] == "grid":
        g = grid(c["side"], c["side"], c["wmax"], seed, nthreads)
    else:
        g = rmat(c["scale"], 16, (0.57, 0.19, 0.19), c["wmax"], seed, True, nthreads)
    g.name = c["name"]
    return g


def config_seed_sets(idx: int, g: Graph) -> list[np.ndarray]:
    """Seed sets of workload ``idx`` (one set for single-query workloads)."""
    c = CONFIGS[idx]
    seed = CONFIG_SEED + idx
    if c["kind"] == "grid":
        pool = np.arange(g.n, dtype=np.int32)
    else:
        pool = largest_cc(g)
    if "queries" not in c:
        return [sample_distinct(pool, c["k"], seed ^ 0x51ED)]
    ks = log_uniform_sizes(c["queries"], c["klo"], c["khi"], seed ^ 0x517E)
    return [sample_distinct(pool, int(k), (seed ^ 0xC0FFEE) + 7919 * i) for i, k in enumerate(ks)]
