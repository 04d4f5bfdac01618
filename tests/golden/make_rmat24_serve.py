"""Writes tests/golden/rmat24_serve2000_sample.json from the CPU oracle alone.

Workload: R-MAT scale 24 (2^24 vertices, 2^28 edge draws, weights uniform
in [1, 1000]) and its stream of 2,000 seed sets of log-uniform size in
[3, 10000], exactly as the workload generators define them.  The oracle
runs Algorithm 2 end to end on every SAMPLE_STRIDE-th query of the stream
(125 queries); the file keeps, per sampled query, its status, total D,
tree-edge count and the digest of its tree edges, so the served stream on
the GPU can be checked against the oracle without running it.

Run:  python tests/golden/make_rmat24_serve.py [workers]
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)

CFG = 5
SAMPLE_STRIDE = 16
OUT = os.path.join(HERE, "rmat24_serve2000_sample.json")

_G = {}


def _job(i):
    import oracle
    import paper_2205_14503_gb300.workloads as wl
    from digests import tree_digest
    if "g" not in _G:
        _G["g"] = wl.config_graph(CFG, nthreads=2)
        _G["qs"] = wl.config_seed_sets(CFG, _G["g"])
    q = _G["qs"][i]
    r = oracle.steiner(_G["g"], q, want_labels=False)
    return i, int(q.size), tree_digest(r.status, r.edges, r.total)


def main():
    workers = int(sys.argv[1]) if len(sys.argv) > 1 else max(1, (os.cpu_count() or 2) - 1)
    import paper_2205_14503_gb300.workloads as wl
    from digests import graph_fingerprint, sha
    t0 = time.time()
    g = wl.config_graph(CFG)
    qs = wl.config_seed_sets(CFG, g)
    fp = graph_fingerprint(g)
    idx = list(range(0, len(qs), SAMPLE_STRIDE))
    seeds_sha = {str(i): sha(qs[i], "int32") for i in idx}
    del g
    with mp.get_context("spawn").Pool(workers) as pool:
        rows = sorted(pool.map(_job, idx, chunksize=1))
    out = {
        "title": "Oracle trees for a sample of the R-MAT 24 served stream (workload rmat24_serve2000)",
        "cites": ["Algorithm 2 Steps 1-7", "Section 'Evaluation': seed sets of 3 to 10K vertices"],
        "written_by": "tests/golden/make_rmat24_serve.py (calls oracle/ and the seeded generators only)",
        "graph": fp,
        "n_queries": len(qs),
        "sample_stride": SAMPLE_STRIDE,
        "queries": [{"index": i, "k": k, "seeds_sha": seeds_sha[str(i)], **d}
                    for i, k, d in rows],
        "seconds": round(time.time() - t0, 1),
    }
    with open(OUT + ".tmp", "w") as f:
        json.dump(out, f, indent=0)
        f.write("\n")
    os.replace(OUT + ".tmp", OUT)
    print(f"wrote {OUT}: {len(rows)} queries in {out['seconds']} s")


if __name__ == "__main__":
    main()
