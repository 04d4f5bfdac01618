"""Parity at the full workload sizes.

* grid 4096^2 / 256 seeds: the CPU oracle runs whole; every output compared.
* R-MAT 22 / 64 batched queries: the oracle for every query (process pool,
  spawned before any GPU work), bit-exact.
* R-MAT 24 served stream: all 2,000 served results equal the single-query
  path, and 125 sampled queries equal the oracle (stored digests).
* R-MAT 26 / 10,000 seeds: the oracle takes minutes and ~20 GB of host
  memory, so its outputs were computed once by tests/golden/make_rmat26.py
  (oracle and seeded generators only) and stored as digests; every output
  of the CUDA path is compared with them bit for bit.
"""
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np
import pytest

import oracle
import paper_2205_14503_gb300.workloads as wl

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

st = pytest.importorskip("paper_2205_14503_gb300.steiner")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, GOLDEN)
import digests  # noqa: E402


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


_GRAPHS = {}


def _oracle_job(args):
    """Oracle on workload `cfg` (the worker rebuilds the seeded graph once)."""
    import oracle as orc
    import paper_2205_14503_gb300.workloads as wlw
    cfg, seeds = args
    if cfg not in _GRAPHS:
        _GRAPHS.clear()
        _GRAPHS[cfg] = wlw.config_graph(cfg, nthreads=2)
    r = orc.steiner(_GRAPHS[cfg], seeds, want_labels=False)
    return r.status, r.edges, r.total


@pytest.fixture(scope="module")
def pool():
    # spawned before any GPU work in this process
    ctx = mp.get_context("spawn")
    p = ctx.Pool(max(1, min(12, (os.cpu_count() or 2) - 2)))
    yield p
    p.close()
    p.join()


@pytest.fixture(scope="module", autouse=True)
def _cuda(pool):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_14503_gb300 import build
    build.build()
    st.load_library()


def test_grid4096_k256_full_oracle():
    g = wl.config_graph(2)
    (seeds,) = wl.config_seed_sets(2, g)
    ref = oracle.steiner(g, seeds, want_labels=True, want_pairs=True)
    with st.SteinerGraph(g) as G:
        rc, cell, dist, pred = G.voronoi(seeds)
        res = G.query_detail(seeds)
    assert res.status == ref.status == oracle.OK
    np.testing.assert_array_equal(cell, ref.cell)
    np.testing.assert_array_equal(dist, ref.dist)
    np.testing.assert_array_equal(pred, ref.pred)
    np.testing.assert_array_equal(res.pairs[:, :4], ref.pairs)
    np.testing.assert_array_equal(res.edges, ref.edges)
    assert res.total == ref.total


def test_rmat22_batch64_full_oracle(pool):
    g = wl.config_graph(4)
    qs = wl.config_seed_sets(4, g)
    refs = pool.map(_oracle_job, [(4, q) for q in qs], chunksize=1)
    with st.SteinerGraph(g) as G:
        rc, res = G.query_batch(qs)
    for i, (r, (status, edges, total)) in enumerate(zip(res, refs)):
        assert r.status == status, i
        np.testing.assert_array_equal(r.edges, edges, err_msg=f"query {i}")
        assert r.total == total


def test_rmat24_served_stream():
    """The whole 2,000-query stream is served (continuous batching); every
    served tree equals the same query run alone through the single-query
    path, and the sampled queries equal the oracle's trees (digests written
    by tests/golden/make_rmat24_serve.py from the oracle alone)."""
    gold = _golden("rmat24_serve2000_sample.json")
    g = wl.config_graph(5)
    qs = wl.config_seed_sets(5, g)
    assert digests.graph_fingerprint(g) == gold["graph"]
    assert len(qs) == gold["n_queries"]
    with st.SteinerGraph(g) as G:
        h = G.handle
        st.steiner_serve_start(h, 64, 40 << 30)
        tickets = [st.steiner_submit(h, q)[1] for q in qs]
        got, deadline = {}, time.time() + 900
        while len(got) < len(tickets) and time.time() < deadline:
            for t in tickets:
                if t not in got:
                    rc, r = st.steiner_poll(h, t)
                    if rc != st.STEINER_PENDING:
                        got[t] = r
            time.sleep(0.002)
        admitted_busy = st.steiner_get_param(h, "batch_admitted_busy")
        launches = st.steiner_get_param(h, "batch_launches")
        st.steiner_serve_stop(h)
        assert len(got) == len(tickets)
        served = [got[t] for t in tickets]
        for i, q in enumerate(qs):
            alone = G.query(q)
            assert served[i].status == alone.status, i
            assert served[i].total == alone.total, i
            assert np.array_equal(served[i].edges, alone.edges), i
    assert admitted_busy > 0 and launches < len(qs)
    for row in gold["queries"]:
        i = row["index"]
        assert digests.sha(qs[i], np.int32) == row["seeds_sha"], i
        r = served[i]
        assert digests.tree_digest(r.status, r.edges, r.total) == \
            {k: row[k] for k in ("status", "total", "n_edges", "edges")}, i


def _same_digest(name, arr, dtype, gold):
    """Digest of arr equals the golden one; on a mismatch, name the first
    chunk (of digests.N_CHUNKS contiguous pieces) where they part."""
    if digests.sha(arr, dtype) == gold["sha"]:
        return
    got = digests.chunk_shas(arr, dtype)
    bad = [i for i, (x, y) in enumerate(zip(got, gold["chunks"])) if x != y]
    raise AssertionError(f"{name}: differs from the oracle in chunks {bad[:8]} of {len(got)}")


@pytest.mark.parametrize("label_bits,far_scan", [(32, 1), (64, 0)])
def test_rmat26_k10000_matches_oracle(label_bits, far_scan):
    """R-MAT 26 with 10,000 seeds, bit for bit against the oracle's outputs
    (digests written by tests/golden/make_rmat26.py from the oracle alone):
    cell, dist and pred of all 67M vertices; the whole distance graph G'_1
    (every adjacent cell pair with its minimum bridge distance and arc, so
    the pair set is complete as well as minimal); the MST pair set; the
    tree edges and the total; under both label widths and both ways of
    splitting bands."""
    gold = _golden("rmat26_k10000.json")
    g = wl.config_graph(3)
    (seeds,) = wl.config_seed_sets(3, g)
    assert digests.graph_fingerprint(g) == gold["graph"]
    assert digests.sha(seeds, np.int32) == gold["seeds"]["sha"]
    with st.SteinerGraph(g) as G:
        G.set_param("label_bits", label_bits)
        G.set_param("far_scan", far_scan)
        rc, cell, dist, pred = G.voronoi(seeds)
        res = G.query_detail(seeds)
        assert G.get_param("label_bits_last") == label_bits
    assert rc == st.STEINER_OK and res.status == gold["status"] == st.STEINER_OK
    _same_digest("cell", cell, np.int32, gold["cell"])
    _same_digest("dist", dist, np.uint32, gold["dist"])
    _same_digest("pred", pred, np.int32, gold["pred"])
    P = res.pairs.astype(np.int64)
    assert P.shape[0] == gold["n_pairs"]
    _same_digest("pairs", digests.pairs_array(P[:, 0], P[:, 1], P[:, 2], P[:, 3]), np.int64,
                 gold["pairs"])
    M = P[P[:, 4] == 1]
    assert M.shape[0] == gold["n_mst"]
    _same_digest("mst", digests.pairs_array(M[:, 0], M[:, 1], M[:, 2], M[:, 3]), np.int64,
                 gold["mst"])
    E = res.edges.astype(np.int64)
    np.testing.assert_array_equal(E[::gold["edge_sample_stride"]], np.array(gold["edge_sample"]))
    assert res.total == gold["total"]
    _same_digest("tree", E, np.int64, {"sha": gold["tree"]["edges"],
                                        "chunks": gold["tree"]["chunks"]})
