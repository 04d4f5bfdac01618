"""Thin Python binding of the C ABI in ``include/steiner.h``.

Argument marshalling only: every step of the method runs in the CUDA
library ``libsteiner.so`` (built in-tree by :mod:`paper_2205_14503_gb300.build`).
There is no CPU fallback — if the library is missing or no GPU is present
the calls raise.  Functions keep the C names (``steiner_load_graph``,
``steiner_query``, ...); :class:`SteinerGraph` wraps a handle for
convenience.  PyTorch is used only for device buffers and streams (the
``steiner_voronoi`` outputs may be CUDA tensors).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsteiner.so")

STEINER_OK = 0
STEINER_PENDING = 1
STEINER_EINVAL = -1
STEINER_ENOMEM = -2
STEINER_EOVERFLOW = -3
STEINER_EDISCONNECTED = -4
STEINER_ETIMEOUT = -5
STEINER_EBUSY = -6
STEINER_ECUDA = -7

STATUS_NAMES = {0: "OK", 1: "PENDING", -1: "EINVAL", -2: "ENOMEM", -3: "EOVERFLOW",
                -4: "EDISCONNECTED", -5: "ETIMEOUT", -6: "EBUSY", -7: "ECUDA"}


class SteinerError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class steiner_edge_t(ctypes.Structure):
    _fields_ = [("u", ctypes.c_uint32), ("v", ctypes.c_uint32), ("w", ctypes.c_uint32)]


class steiner_result_t(ctypes.Structure):
    _fields_ = [("edges", ctypes.POINTER(steiner_edge_t)), ("n_edges", ctypes.c_uint32),
                ("total", ctypes.c_uint64), ("status", ctypes.c_int32)]


class steiner_pair_t(ctypes.Structure):
    _fields_ = [("ra", ctypes.c_uint32), ("rb", ctypes.c_uint32), ("b", ctypes.c_uint64),
                ("arc", ctypes.c_uint32), ("in_mst", ctypes.c_uint32)]


class steiner_stats_t(ctypes.Structure):
    _fields_ = [("relax_attempts", ctypes.c_uint64), ("relax_improved", ctypes.c_uint64),
                ("iterations", ctypes.c_uint32), ("phases", ctypes.c_uint32),
                ("n_pairs", ctypes.c_uint64), ("n_tree_edges", ctypes.c_uint32),
                ("gpu_launches", ctypes.c_uint32), ("ms_init", ctypes.c_float),
                ("ms_voronoi", ctypes.c_float), ("ms_bridges", ctypes.c_float),
                ("ms_mst", ctypes.c_float), ("ms_tree", ctypes.c_float)]


# name -> (restype, argtypes); every symbol declared in include/steiner.h
_vp, _u32, _u64, _i32, _i64 = (ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int,
                               ctypes.c_int64)
SIGNATURES = {
    "steiner_load_graph": (_i32, [_vp, _vp, _vp, _u32, _u64, _i32, ctypes.POINTER(_vp)]),
    "steiner_free_graph": (None, [_vp]),
    "steiner_query": (_i32, [_vp, _vp, _u32, ctypes.POINTER(steiner_result_t)]),
    "steiner_query_detail": (_i32, [_vp, _vp, _u32, ctypes.POINTER(steiner_result_t),
                                    ctypes.POINTER(ctypes.POINTER(steiner_pair_t)),
                                    ctypes.POINTER(_u64), ctypes.POINTER(steiner_stats_t)]),
    "steiner_voronoi": (_i32, [_vp, _vp, _u32, _vp, _vp, _vp]),
    "steiner_query_batch": (_i32, [_vp, ctypes.POINTER(_vp), _vp, _u32,
                                   ctypes.POINTER(steiner_result_t)]),
    "steiner_serve_start": (_i32, [_vp, _u32, _u64]),
    "steiner_submit": (_i32, [_vp, _vp, _u32, ctypes.POINTER(_u64)]),
    "steiner_poll": (_i32, [_vp, _u64, ctypes.POINTER(steiner_result_t)]),
    "steiner_serve_stop": (_i32, [_vp]),
    "steiner_voronoi_noalloc": (_i32, [_vp, _vp, _vp, _u32, _u64, _vp, _u32, _vp, _vp, _vp,
                                       _vp]),
    "steiner_set_param": (_i32, [_vp, ctypes.c_char_p, _i64]),
    "steiner_get_param": (_i64, [_vp, ctypes.c_char_p]),
    "steiner_result_free": (None, [ctypes.POINTER(steiner_result_t)]),
    "steiner_pairs_free": (None, [ctypes.POINTER(steiner_pair_t)]),
    "steiner_last_error": (ctypes.c_char_p, []),
    "steiner_version": (ctypes.c_char_p, []),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libsteiner.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing "
                           "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def last_error() -> str:
    return load_library().steiner_last_error().decode()


def _check(code: int, allowed=(STEINER_OK,)) -> int:
    if code not in allowed:
        raise SteinerError(code, last_error())
    return code


def _i32array(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.int64).astype(np.int32))


@dataclass
class Result:
    status: int
    edges: np.ndarray       # uint32[n_edges, 3]: (u, v, w), u < v, ascending
    total: int
    pairs: np.ndarray | None = None   # uint64[n_pairs, 5]: (ra, rb, b, arc, in_mst)
    stats: dict = field(default_factory=dict)


def _take_result(r: steiner_result_t) -> Result:
    n = int(r.n_edges)
    if n and r.edges:
        buf = np.ctypeslib.as_array(ctypes.cast(r.edges, ctypes.POINTER(ctypes.c_uint32)),
                                    shape=(n * 3,))
        edges = buf.reshape(n, 3).copy()
    else:
        edges = np.zeros((0, 3), np.uint32)
    out = Result(int(r.status), edges, int(r.total))
    load_library().steiner_result_free(ctypes.byref(r))
    return out


# ---------------------------------------------------------------------------
# C-named functions
# ---------------------------------------------------------------------------

def steiner_load_graph(row_ptr, col, w, device: int = 0) -> int:
    """Upload a CSR graph; returns the opaque handle (int)."""
    lib = load_library()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.uint32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.uint32)
    n = row_ptr.shape[0] - 1
    h = ctypes.c_void_p()
    _check(lib.steiner_load_graph(row_ptr.ctypes.data, col.ctypes.data if col.size else None,
                                  w.ctypes.data if w.size else None, n, col.shape[0], device,
                                  ctypes.byref(h)))
    return h.value


def steiner_free_graph(h: int) -> None:
    load_library().steiner_free_graph(h)


def steiner_query(h: int, seeds) -> Result:
    s = _i32array(seeds)
    r = steiner_result_t()
    load_library().steiner_query(h, s.ctypes.data if s.size else None, s.size, ctypes.byref(r))
    return _take_result(r)


def steiner_query_detail(h: int, seeds, pairs: bool = True) -> Result:
    """steiner_query plus the distance graph G'_1 (``pairs``) and counters."""
    lib = load_library()
    s = _i32array(seeds)
    r = steiner_result_t()
    pp = ctypes.POINTER(steiner_pair_t)()
    npairs = ctypes.c_uint64(0)
    st = steiner_stats_t()
    lib.steiner_query_detail(h, s.ctypes.data if s.size else None, s.size, ctypes.byref(r),
                             ctypes.byref(pp) if pairs else None, ctypes.byref(npairs),
                             ctypes.byref(st))
    out = _take_result(r)
    n = int(npairs.value)
    if pp:
        arr = np.zeros((n, 5), np.uint64)
        if n:
            rec = np.ctypeslib.as_array(pp, shape=(n,))
            for i, f in enumerate(("ra", "rb", "b", "arc", "in_mst")):
                arr[:, i] = rec[f]
        lib.steiner_pairs_free(pp)
        out.pairs = arr
    out.stats = {f: getattr(st, f) for f, _ in steiner_stats_t._fields_}
    return out


def steiner_voronoi(h: int, seeds, cell=None, dist=None, pred=None, n: int | None = None):
    """Voronoi cells.  Outputs may be numpy arrays (host) or CUDA tensors
    (device, written in place); missing outputs are allocated on the host."""
    lib = load_library()
    s = _i32array(seeds)
    if n is None:
        sizes = [len(x) for x in (cell, dist, pred) if x is not None]
        if not sizes:
            raise ValueError("pass n or at least one output buffer")
        n = sizes[0]
    if cell is None:
        cell = np.empty(n, np.int32)
    if dist is None:
        dist = np.empty(n, np.uint32)
    if pred is None:
        pred = np.empty(n, np.int32)

    def ptr(x):
        if isinstance(x, np.ndarray):
            assert x.flags.c_contiguous and x.itemsize == 4 and x.size >= n
            return x.ctypes.data
        assert x.is_contiguous() and x.element_size() == 4 and x.numel() >= n
        return x.data_ptr()
    rc = lib.steiner_voronoi(h, s.ctypes.data if s.size else None, s.size, ptr(cell), ptr(dist),
                             ptr(pred))
    return rc, cell, dist, pred


def steiner_voronoi_noalloc(row_ptr, col, w, seeds, cell, dist, pred, stream=None) -> int:
    """Voronoi cells without any device allocation.  Every argument is a
    CUDA tensor the caller allocated (4-byte elements; seeds sorted
    ascending); ``stream`` is a torch stream (default: the current one)."""
    import torch
    lib = load_library()
    n = row_ptr.numel() - 1
    st = (stream or torch.cuda.current_stream()).cuda_stream

    def p(t):
        return None if t is None else t.data_ptr()
    return int(lib.steiner_voronoi_noalloc(p(row_ptr), p(col), p(w), n, col.numel(), p(seeds),
                                           seeds.numel(), p(cell), p(dist), p(pred), st))


def steiner_query_batch(h: int, seed_sets) -> tuple[int, list[Result]]:
    lib = load_library()
    arrs = [_i32array(s) for s in seed_sets]
    q = len(arrs)
    ptrs = (ctypes.c_void_p * max(q, 1))(*[a.ctypes.data if a.size else None for a in arrs])
    ks = np.array([a.size for a in arrs] or [0], dtype=np.uint32)
    outs = (steiner_result_t * max(q, 1))()
    rc = lib.steiner_query_batch(h, ptrs, ks.ctypes.data, q, outs)
    return rc, [_take_result(outs[i]) for i in range(q)]


def steiner_serve_start(h: int, slots: int = 64, budget_bytes: int = 40 << 30) -> None:
    _check(load_library().steiner_serve_start(h, slots, budget_bytes))


def steiner_submit(h: int, seeds) -> tuple[int, int]:
    s = _i32array(seeds)
    t = ctypes.c_uint64(0)
    rc = load_library().steiner_submit(h, s.ctypes.data if s.size else None, s.size,
                                       ctypes.byref(t))
    return rc, int(t.value)


def steiner_poll(h: int, ticket: int):
    r = steiner_result_t()
    # steiner_poll writes *out only when it returns a result; the sentinel
    # tells a pending or unknown ticket (no result: None) from a query that
    # finished with an error status
    r.status = STEINER_PENDING
    rc = load_library().steiner_poll(h, ticket, ctypes.byref(r))
    if rc == STEINER_PENDING or r.status == STEINER_PENDING:
        return rc, None
    return rc, _take_result(r)


def steiner_serve_stop(h: int) -> None:
    load_library().steiner_serve_stop(h)


def steiner_set_param(h: int, key: str, value: int) -> None:
    _check(load_library().steiner_set_param(h, key.encode(), int(value)))


def steiner_get_param(h: int, key: str) -> int:
    return int(load_library().steiner_get_param(h, key.encode()))


def steiner_version() -> str:
    return load_library().steiner_version().decode()


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------

class SteinerGraph:
    """A graph resident on one GPU."""

    def __init__(self, graph, device: int = 0):
        self.n = int(graph.n)
        self.handle = steiner_load_graph(graph.row_ptr, graph.col, graph.w, device)

    def close(self):
        if self.handle:
            steiner_free_graph(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def query(self, seeds) -> Result:
        return steiner_query(self.handle, seeds)

    def query_detail(self, seeds, pairs: bool = True) -> Result:
        return steiner_query_detail(self.handle, seeds, pairs)

    def voronoi(self, seeds, cell=None, dist=None, pred=None):
        return steiner_voronoi(self.handle, seeds, cell, dist, pred, n=self.n)

    def query_batch(self, seed_sets):
        return steiner_query_batch(self.handle, seed_sets)

    def set_param(self, key, value):
        steiner_set_param(self.handle, key, value)

    def get_param(self, key):
        return steiner_get_param(self.handle, key)
