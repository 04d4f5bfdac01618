"""Writes tests/golden/rmat26_k10000.json from the CPU oracle alone.

Workload: R-MAT scale 26 (2^26 vertices, 2^30 edge draws, (a,b,c) =
(.57,.19,.19), weights uniform in [1, 1000]) with 10,000 seeds drawn
uniformly from its largest component, exactly as the workload generators
define it.  The oracle runs Algorithm 2 end to end (Steps 1-7) on it; the
file keeps digests of every output (cell, dist, pred per vertex; the
distance graph G'_1 as (rank a, rank b, bridge distance, arc); the MST pair
set; the tree edges), the total D, the counts, and a strided sample of tree
edges, so that a GPU test can compare the CUDA path with the oracle bit for
bit without running the oracle (about 20 GB of host memory and minutes).

Run:  python tests/golden/make_rmat26.py   (needs ~35 GB of host RAM)
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)

import oracle  # noqa: E402
import paper_2205_14503_gb300.workloads as wl  # noqa: E402
from digests import (chunk_shas, graph_fingerprint, pairs_array, sha,  # noqa: E402
                     tree_digest)

CFG = 3
OUT = os.path.join(HERE, "rmat26_k10000.json")
EDGE_SAMPLE_STRIDE = 97


def main():
    t0 = time.time()
    g = wl.config_graph(CFG)
    (seeds,) = wl.config_seed_sets(CFG, g)
    t_gen = time.time() - t0
    t1 = time.time()
    r = oracle.steiner(g, seeds, want_labels=True, want_pairs=True)
    t_orc = time.time() - t1
    if r.status != oracle.OK:
        raise SystemExit(f"oracle status {r.status}")
    P = pairs_array(r.pairs[:, 0], r.pairs[:, 1], r.pairs[:, 2], r.pairs[:, 3])
    M = pairs_array(r.mst[:, 0], r.mst[:, 1], r.mst[:, 2], r.mst[:, 3])
    E = r.edges.astype(np.int64)
    out = {
        "title": "Oracle outputs for R-MAT scale 26 with 10,000 seeds (workload rmat26_k10000)",
        "cites": ["Algorithm 2 Steps 1-7 (Voronoi cells, distance graph G'_1, MST, expansion)",
                  "Section 'Evaluation': seed sets of up to 10K vertices on billion-edge graphs"],
        "written_by": "tests/golden/make_rmat26.py (calls oracle/ and the seeded generators only)",
        "graph": graph_fingerprint(g),
        "seeds": {"k": int(seeds.size), "sha": sha(seeds, np.int32)},
        "status": int(r.status),
        "total": int(r.total),
        "n_pairs": int(P.shape[0]),
        "n_mst": int(M.shape[0]),
        "cell": {"sha": sha(r.cell, np.int32), "chunks": chunk_shas(r.cell, np.int32)},
        "dist": {"sha": sha(r.dist, np.uint32), "chunks": chunk_shas(r.dist, np.uint32)},
        "pred": {"sha": sha(r.pred, np.int32), "chunks": chunk_shas(r.pred, np.int32)},
        "pairs": {"sha": sha(P, np.int64), "chunks": chunk_shas(P, np.int64)},
        "mst": {"sha": sha(M, np.int64), "chunks": chunk_shas(M, np.int64)},
        "tree": dict(tree_digest(r.status, E, r.total), chunks=chunk_shas(E, np.int64)),
        "edge_sample_stride": EDGE_SAMPLE_STRIDE,
        "edge_sample": E[::EDGE_SAMPLE_STRIDE].tolist(),
        "oracle_seconds": round(t_orc, 1),
        "generate_seconds": round(t_gen, 1),
    }
    with open(OUT + ".tmp", "w") as f:
        json.dump(out, f, indent=0)
        f.write("\n")
    os.replace(OUT + ".tmp", OUT)
    print(f"wrote {OUT}: n_pairs {P.shape[0]}, tree edges {E.shape[0]}, total {r.total}, "
          f"oracle {t_orc:.1f} s, generation {t_gen:.1f} s")


if __name__ == "__main__":
    main()
