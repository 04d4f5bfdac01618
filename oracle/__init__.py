"""CPU oracle for the Voronoi-cell 2-approximation Steiner tree.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the benchmark's CPU-baseline leg, never by the library's product path.  It
shares no code with the CUDA path; the arithmetic lives in
``steiner_oracle.c`` (plain C, compiled with gcc by :func:`build`), which
follows the paper's Algorithm 2 step by step:

* Step 1 (Voronoi cells, Algorithm 4): multi-source Dijkstra with labels
  (distance, seed rank); pred(v) is the smallest-id neighbour on a tight
  edge inside v's cell.
* Step 2 (distance graph G'_1, Algorithm 5): per adjacent cell pair the
  minimum (d1(s,u) + d(u,v) + d1(v,t), arc id).
* Step 3 (MST of G'_1): Kruskal under the order (weight, rank a, rank b).
* Steps 4-7 (Algorithm 6): bridge edges of the MST pairs plus predecessor
  paths to the seeds; D = sum of the tree's edge weights.

Parity status: every function here is pinned by tests in
``tests/test_oracle_pins.py`` against quantities fixed by the mathematics
(per-seed Dijkstra from scipy, Mehlhorn's MST-weight theorem, textbook MST
for S = V, Dreyfus-Wagner optima, closed forms on trees and paths).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "steiner_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lib = None

OK = 0
EINVAL = -1
ENOMEM = -2
EOVERFLOW = -3
EDISCONNECTED = -4

DIST_INF = 0xFFFFFFFF


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-std=c11", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _bind(lib):
    vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
    lib.oracle_check_graph.restype = ctypes.c_int
    lib.oracle_check_graph.argtypes = [u32, vp, vp, vp]
    lib.oracle_voronoi.restype = ctypes.c_int
    lib.oracle_voronoi.argtypes = [u32, vp, vp, vp, u32, vp, vp, vp, vp]
    lib.oracle_steiner.restype = ctypes.c_int
    lib.oracle_steiner.argtypes = ([u32, vp, vp, vp, u32, vp, vp, vp, vp]
                                   + [vp] * 4 + [u64, vp] + [vp] * 4 + [vp]
                                   + [vp] * 3 + [vp, vp])
    return lib


def compile_variant(source_text: str, path: str):
    """Compile a modified copy of the oracle source (used by the tests that
    plant mistakes in the oracle to show the pins catch them)."""
    cpath = path + ".c"
    with open(cpath, "w") as f:
        f.write(source_text)
    subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-std=c11", "-o", path, cpath])
    return _bind(ctypes.CDLL(path))


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _load(lib=None):
    global _lib
    if lib is not None:
        return lib
    if _lib is None:
        build()
        _lib = _bind(ctypes.CDLL(_LIB))
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _graph_args(g):
    row_ptr = np.ascontiguousarray(g.row_ptr, dtype=np.uint32)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    w = np.ascontiguousarray(g.w, dtype=np.uint32)
    if col.size == 0:   # keep valid pointers for empty graphs
        col = np.zeros(1, dtype=np.int32)
        w = np.zeros(1, dtype=np.uint32)
    return row_ptr, col, w


def check_graph(g, lib=None) -> int:
    row_ptr, col, w = _graph_args(g)
    return _load(lib).oracle_check_graph(g.n, _p(row_ptr), _p(col), _p(w))


@dataclass
class Voronoi:
    status: int
    cell: np.ndarray    # int32[n]: seed vertex id, -1 unreached
    dist: np.ndarray    # uint32[n]: 0xFFFFFFFF unreached
    pred: np.ndarray    # int32[n]: -1 unreached, self for seeds


def voronoi(g, seeds, lib=None) -> Voronoi:
    """Algorithm 2 Step 1 for seed list ``seeds`` (any order)."""
    row_ptr, col, w = _graph_args(g)
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    n = g.n
    cell = np.empty(max(n, 1), np.int32)
    dist = np.empty(max(n, 1), np.uint32)
    pred = np.empty(max(n, 1), np.int32)
    rc = _load(lib).oracle_voronoi(n, _p(row_ptr), _p(col), _p(w), seeds.size,
                                _p(seeds) if seeds.size else None, _p(cell), _p(dist), _p(pred))
    return Voronoi(rc, cell[:n], dist[:n], pred[:n])


@dataclass
class Steiner:
    status: int
    edges: np.ndarray          # uint32[n_edges, 3]: (u, v, w), u < v, ascending
    total: int
    cell: np.ndarray | None = None
    dist: np.ndarray | None = None
    pred: np.ndarray | None = None
    pairs: np.ndarray | None = None   # uint64[n_pairs, 4]: (ra, rb, b, arc), ascending (ra, rb)
    mst: np.ndarray | None = None     # uint64[n_mst, 4]: Kruskal order


def steiner(g, seeds, want_labels: bool = True, want_pairs: bool = False, lib=None) -> Steiner:
    """Algorithm 2 end to end; returns tree edges, total distance and,
    optionally, the per-vertex labels and the distance graph G'_1."""
    row_ptr, col, w = _graph_args(g)
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    n, k = g.n, seeds.size
    cell = np.empty(max(n, 1), np.int32) if want_labels else None
    dist = np.empty(max(n, 1), np.uint32) if want_labels else None
    pred = np.empty(max(n, 1), np.int32) if want_labels else None
    cap = 0
    pra = prb = pb = parc = None
    if want_pairs:
        cap = min(k * (k - 1) // 2, g.n_arcs // 2 + 1)
        pra = np.empty(max(cap, 1), np.uint32)
        prb = np.empty(max(cap, 1), np.uint32)
        pb = np.empty(max(cap, 1), np.uint64)
        parc = np.empty(max(cap, 1), np.uint32)
    mra = np.empty(max(k, 1), np.uint32)
    mrb = np.empty(max(k, 1), np.uint32)
    mb = np.empty(max(k, 1), np.uint64)
    marc = np.empty(max(k, 1), np.uint32)
    eu = np.empty(max(n, 1), np.uint32)
    ev = np.empty(max(n, 1), np.uint32)
    ew = np.empty(max(n, 1), np.uint32)
    n_pairs = ctypes.c_uint64(0)
    n_mst = ctypes.c_uint64(0)
    n_edges = ctypes.c_uint64(0)
    total = ctypes.c_uint64(0)
    rc = _load(lib).oracle_steiner(
        n, _p(row_ptr), _p(col), _p(w), k, _p(seeds) if k else None,
        _p(cell), _p(dist), _p(pred),
        _p(pra), _p(prb), _p(pb), _p(parc), cap, ctypes.byref(n_pairs),
        _p(mra), _p(mrb), _p(mb), _p(marc), ctypes.byref(n_mst),
        _p(eu), _p(ev), _p(ew), ctypes.byref(n_edges), ctypes.byref(total))
    ne = n_edges.value
    edges = np.stack([eu[:ne], ev[:ne], ew[:ne]], axis=1) if rc in (OK, EDISCONNECTED) \
        else np.zeros((0, 3), np.uint32)
    out = Steiner(rc, edges, int(total.value) if rc in (OK, EDISCONNECTED) else 0)
    if want_labels:
        out.cell, out.dist, out.pred = cell[:n], dist[:n], pred[:n]
    if want_pairs and rc in (OK, EDISCONNECTED):
        npairs = min(n_pairs.value, cap)
        out.pairs = np.stack([pra[:npairs].astype(np.uint64), prb[:npairs].astype(np.uint64),
                              pb[:npairs], parc[:npairs].astype(np.uint64)], axis=1)
    if rc in (OK, EDISCONNECTED):
        nm = n_mst.value
        out.mst = np.stack([mra[:nm].astype(np.uint64), mrb[:nm].astype(np.uint64), mb[:nm],
                            marc[:nm].astype(np.uint64)], axis=1)
    return out
