"""Canonical digests of query outputs, for golden files too large to store.

Both the scripts that write golden files (from the oracle only) and the GPU
tests that check against them build the same canonical arrays and hash them
here, so a stored digest and a recomputed one agree exactly when the
underlying arrays do.  Every array is hashed as little-endian bytes of a
fixed dtype; a per-chunk digest list lets a mismatch name the index range
where the two sides part.  No Steiner arithmetic lives here.
"""
from __future__ import annotations

import hashlib

import numpy as np

N_CHUNKS = 64


def canon(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a).astype(np.dtype(dtype).newbyteorder("<"),
                                                      copy=False))


def sha(a, dtype) -> str:
    return hashlib.sha256(canon(a, dtype).tobytes()).hexdigest()


def chunk_shas(a, dtype, n_chunks: int = N_CHUNKS) -> list[str]:
    """Short digests of n_chunks contiguous pieces along axis 0."""
    c = canon(a, dtype)
    return [hashlib.sha256(p.tobytes()).hexdigest()[:16] for p in np.array_split(c, n_chunks)]


def graph_fingerprint(g) -> dict:
    """Cheap fingerprint of a CSR graph: its sizes, the full row offsets and
    a strided sample of neighbours and weights."""
    return {"n": int(g.n), "arcs": int(g.n_arcs),
            "row_ptr": sha(g.row_ptr, np.uint32),
            "col_stride_4099": sha(g.col[::4099], np.int32),
            "w_stride_4099": sha(g.w[::4099], np.uint32)}


def pairs_array(ra, rb, b, arc) -> np.ndarray:
    """(n, 4) int64 rows (rank a, rank b, bridge distance, arc), ascending (ra, rb)."""
    P = np.stack([np.asarray(x, dtype=np.int64) for x in (ra, rb, b, arc)], axis=1) \
        if len(ra) else np.zeros((0, 4), np.int64)
    order = np.lexsort((P[:, 1], P[:, 0]))
    return P[order]


def tree_digest(status: int, edges, total: int) -> dict:
    E = np.asarray(edges, dtype=np.int64).reshape(-1, 3)
    return {"status": int(status), "total": int(total), "n_edges": int(E.shape[0]),
            "edges": sha(E, np.int64)}
