"""GPU parity: the CUDA path through the C ABI against the CPU oracle,
element by element and bit-exact (all results are integers): per-vertex
cell / distance / predecessor, the distance graph G'_1 (pairs, bridge
distance, arc), the MST pairs, the tree edge list and its total distance,
and the status codes of the degenerate cases."""
import numpy as np
import pytest

import oracle
import paper_2205_14503_gb300.workloads as wl
from tests import graphs as G

pytestmark = pytest.mark.gpu

st = pytest.importorskip("paper_2205_14503_gb300.steiner")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_14503_gb300 import build
    build.build()
    st.load_library()


def _compare(g, seeds, detail=True):
    """Run both sides; assert bit-exact agreement; return the oracle result."""
    ref = oracle.steiner(g, seeds, want_labels=True, want_pairs=detail)
    with st.SteinerGraph(g) as Gd:
        rc, cell, dist, pred = Gd.voronoi(seeds)
        res = Gd.query_detail(seeds) if detail else Gd.query(seeds)
    assert res.status == ref.status, (res.status, ref.status, st.last_error())
    if ref.status in (oracle.OK, oracle.EDISCONNECTED):
        assert rc == st.STEINER_OK
        np.testing.assert_array_equal(cell, ref.cell)
        np.testing.assert_array_equal(dist, ref.dist)
        np.testing.assert_array_equal(pred, ref.pred)
        np.testing.assert_array_equal(res.edges, ref.edges)
        assert res.total == ref.total
        if detail:
            np.testing.assert_array_equal(res.pairs[:, :4], ref.pairs)
            mst_gpu = {(int(a), int(b)) for a, b, _, _, m in res.pairs.tolist() if m}
            mst_ref = {(int(a), int(b)) for a, b, _, _ in ref.mst.tolist()}
            assert mst_gpu == mst_ref
    return ref


def _cases():
    yield "rmat9", wl.rmat(9, 8, wmax=100, seed=11), [1, 2, 12, 60]
    yield "rmat10_unit", wl.rmat(10, 8, wmax=1, seed=12), [3, 9, 100]
    yield "rmat11_w3", wl.rmat(11, 16, wmax=3, seed=13), [5, 30, 400]
    yield "grid23x17", wl.grid(23, 17, 1000, seed=14), [2, 7, 40]
    yield "grid_unit", wl.grid(40, 31, 1, seed=15), [2, 5, 64]
    yield "connected", G.random_connected(3000, 2000, 1, 50, 16), [20, 200]
    yield "complete", G.complete(60, 1, 10, 17), [6, 60]
    yield "disconnected", G.random_graph(4000, 3000, 1, 20, 18), [25, 300]
    yield "star", G.star(3000, 1, 5, 19), [10, 500]
    yield "path", G.path(2000, 1, 9, 20), [2, 4, 33]
    yield "tree", G.random_tree(5000, 1, 100, 21), [3, 50]


CASES = list(_cases())


@pytest.mark.parametrize("name,g,ks", CASES, ids=[c[0] for c in CASES])
def test_parity_small_graphs(name, g, ks):
    for i, k in enumerate(ks):
        seeds = G.seeds_from(np.arange(g.n), k, 1000 + 17 * i + k)
        _compare(g, seeds)


def test_parity_rmat_scale16_k16():
    """R-MAT scale 16, edge factor 16, weights [1,100], 16 seeds from the
    largest component (the plain single-query workload)."""
    g = wl.config_graph(1)
    (seeds,) = wl.config_seed_sets(1, g)
    ref = _compare(g, seeds)
    assert ref.status == oracle.OK


def test_parity_hubs_and_many_seeds():
    """Heavy rows (degree >= 256, chunked), a multi-block MST (k > 362) and
    a large pair table."""
    g = wl.rmat(16, 16, wmax=1000, seed=99)
    seeds = wl.sample_distinct(wl.largest_cc(g), 2000, 3)
    _compare(g, seeds)


def test_parity_unit_weights_maximal_ties():
    g = wl.rmat(15, 16, wmax=1, seed=5)
    seeds = wl.sample_distinct(wl.largest_cc(g), 300, 4)
    _compare(g, seeds)


def test_single_seed_and_all_vertices_seeded():
    g = wl.grid(30, 20, 50, seed=3)
    ref = _compare(g, [123])
    assert ref.edges.shape[0] == 0 and ref.total == 0
    _compare(g, np.arange(g.n))


def test_seed_order_does_not_matter():
    g = wl.rmat(12, 16, wmax=100, seed=8)
    seeds = wl.sample_distinct(wl.largest_cc(g), 40, 8)
    with st.SteinerGraph(g) as Gd:
        a = Gd.query(seeds)
        b = Gd.query(seeds[::-1])
        c = Gd.query(np.roll(seeds, 7))
    assert np.array_equal(a.edges, b.edges) and np.array_equal(a.edges, c.edges)
    assert a.total == b.total == c.total


def test_repeated_queries_reuse_workspace():
    """Back-to-back queries of different sizes on one handle (stamp epochs,
    pair-table regrowth) give the oracle's answer every time."""
    g = wl.rmat(13, 16, wmax=200, seed=9)
    pool = wl.largest_cc(g)
    with st.SteinerGraph(g) as Gd:
        for i, k in enumerate([5, 300, 2, 50, 300, 1, 17]):
            seeds = wl.sample_distinct(pool, k, 100 + i)
            res = Gd.query(seeds)
            ref = oracle.steiner(g, seeds, want_labels=False)
            assert res.status == ref.status
            np.testing.assert_array_equal(res.edges, ref.edges)
            assert res.total == ref.total


def test_invalid_seed_lists_are_rejected():
    g = wl.grid(8, 8, 9, seed=1)
    with st.SteinerGraph(g) as Gd:
        assert Gd.query([]).status == st.STEINER_EINVAL
        assert Gd.query([3, 3]).status == st.STEINER_EINVAL
        assert Gd.query([64]).status == st.STEINER_EINVAL
        assert Gd.query([-1, 5]).status == st.STEINER_EINVAL
        assert Gd.query([0, 63]).status == st.STEINER_OK


def test_overflow_and_disconnected_statuses():
    big = 0xFFFFFFFF // 2 + 1
    g = wl.from_edges(4, [0, 1, 2], [1, 2, 3], [big, big, 5])
    _compare(g, [0, 3], detail=False)
    g = wl.from_edges(3, [0, 1], [1, 2], [0xFFFFFFFE, 1])
    _compare(g, [0, 2], detail=False)
    g = wl.from_edges(2, [0], [1], [0xFFFFFFFE])
    _compare(g, [0, 1])
    e = np.array([[0, 1, 3], [1, 2, 4], [3, 4, 5], [4, 5, 1]])
    g = wl.from_edges(7, e[:, 0], e[:, 1], e[:, 2])
    ref = _compare(g, [0, 2, 3, 5])
    assert ref.status == oracle.EDISCONNECTED


def test_malformed_graphs_are_rejected_at_load():
    g = wl.grid(6, 5, 9, seed=2)

    def bad(mod):
        rp, col, w = g.row_ptr.copy(), g.col.copy(), g.w.copy()
        mod(rp, col, w)
        with pytest.raises(st.SteinerError) as ei:
            st.steiner_load_graph(rp, col, w)
        assert ei.value.code == st.STEINER_EINVAL

    bad(lambda rp, col, w: w.__setitem__(3, 0))
    bad(lambda rp, col, w: w.__setitem__(3, w[3] + 1))
    bad(lambda rp, col, w: col.__setitem__(0, 0))
    bad(lambda rp, col, w: (col.__setitem__(0, col[1]), col.__setitem__(1, col[0])))
    bad(lambda rp, col, w: col.__setitem__(2, 10 ** 6))
    h = st.steiner_load_graph(g.row_ptr, g.col, g.w)
    st.steiner_free_graph(h)


def test_voronoi_into_device_tensors():
    import torch
    g = wl.rmat(12, 16, wmax=50, seed=4)
    seeds = wl.sample_distinct(wl.largest_cc(g), 9, 4)
    ref = oracle.voronoi(g, seeds)
    cell = torch.empty(g.n, dtype=torch.int32, device="cuda")
    dist = torch.empty(g.n, dtype=torch.int32, device="cuda")
    pred = torch.empty(g.n, dtype=torch.int32, device="cuda")
    with st.SteinerGraph(g) as Gd:
        rc, _, _, _ = Gd.voronoi(seeds, cell, dist, pred)
    assert rc == st.STEINER_OK
    np.testing.assert_array_equal(cell.cpu().numpy(), ref.cell)
    np.testing.assert_array_equal(dist.cpu().numpy().view(np.uint32), ref.dist)
    np.testing.assert_array_equal(pred.cpu().numpy(), ref.pred)


@pytest.mark.parametrize("delta,local", [(1, 0), (7, 0), (100, 0), (5000, 0), (10 ** 8, 0),
                                         (7, 4), (100, 32), (5000, 2)])
def test_result_is_independent_of_delta(delta, local):
    """The near/far band width and the block-local rounds change the
    schedule, never the fixed point."""
    g = wl.rmat(13, 16, wmax=1000, seed=6)
    seeds = wl.sample_distinct(wl.largest_cc(g), 64, 6)
    ref = oracle.steiner(g, seeds)
    with st.SteinerGraph(g) as Gd:
        Gd.set_param("delta", delta)
        Gd.set_param("local_rounds", local)
        rc, cell, dist, pred = Gd.voronoi(seeds)
        res = Gd.query(seeds)
    np.testing.assert_array_equal(cell, ref.cell)
    np.testing.assert_array_equal(pred, ref.pred)
    np.testing.assert_array_equal(res.edges, ref.edges)


@pytest.mark.parametrize("delta,local", [(50, 0), (300, 8), (999, 0), (1000, 32)])
def test_light_heavy_arc_split_on_grid_and_hubs(delta, local):
    """With delta at or below the largest weight the bands relax light arcs
    only and close with a heavy-arc pass; labels, preds and trees are
    unchanged (a high-diameter grid, and an R-MAT graph whose hubs span
    several heavy-row chunks)."""
    for g, k in ((wl.grid(180, 140, 1000, seed=8), 40), (wl.rmat(12, 48, wmax=1000, seed=9), 25)):
        pool = np.arange(g.n, dtype=np.int32) if g.n == 180 * 140 else wl.largest_cc(g)
        seeds = wl.sample_distinct(pool, k, 8)
        ref = oracle.steiner(g, seeds)
        with st.SteinerGraph(g) as Gd:
            Gd.set_param("delta", delta)
            Gd.set_param("local_rounds", local)
            rc, cell, dist, pred = Gd.voronoi(seeds)
            res = Gd.query(seeds)
        assert rc == st.STEINER_OK
        np.testing.assert_array_equal(cell, ref.cell)
        np.testing.assert_array_equal(dist, ref.dist)
        np.testing.assert_array_equal(pred, ref.pred)
        np.testing.assert_array_equal(res.edges, ref.edges)
        assert res.total == ref.total


@pytest.mark.parametrize("relabel", ["0", "1"])
def test_internal_vertex_order_is_invisible(relabel, monkeypatch):
    """The library may renumber vertices internally (by descending degree);
    forced off and on, every output stays in the caller's ids and arc
    indices and equals the oracle: cells, distances, preds, the distance
    graph with its tie-broken bridge arcs (small weights: many equal
    bridges), the tree, and the batched path's trees."""
    monkeypatch.setenv("STEINER_RELABEL", relabel)
    cases = [(wl.rmat(12, 16, wmax=5, seed=31), 40), (wl.grid(120, 90, 1000, seed=32), 30),
             (wl.rmat(12, 48, wmax=1000, seed=33), 25)]
    for g, k in cases:
        is_grid = g.n == 120 * 90
        pool = np.arange(g.n, dtype=np.int32) if is_grid else wl.largest_cc(g)
        seeds = wl.sample_distinct(pool, k, 34)
        seeds2 = wl.sample_distinct(pool, k // 2 + 2, 35)
        ref = oracle.steiner(g, seeds, want_labels=True, want_pairs=True)
        ref2 = oracle.steiner(g, seeds2)
        with st.SteinerGraph(g) as Gd:
            rc, cell, dist, pred = Gd.voronoi(seeds)
            res = Gd.query_detail(seeds)
            rcb, batch = Gd.query_batch([seeds, seeds2])
        assert rc == st.STEINER_OK and res.status == st.STEINER_OK and rcb == st.STEINER_OK
        np.testing.assert_array_equal(cell, ref.cell)
        np.testing.assert_array_equal(dist, ref.dist)
        np.testing.assert_array_equal(pred, ref.pred)
        np.testing.assert_array_equal(res.pairs[:, :4], ref.pairs)
        np.testing.assert_array_equal(res.edges, ref.edges)
        assert res.total == ref.total
        for r, rf in zip(batch, (ref, ref2)):
            np.testing.assert_array_equal(r.edges, rf.edges)
            assert r.total == rf.total


def test_iteration_cap_reports_timeout():
    """A loop cap that cannot be met returns STEINER_ETIMEOUT (bounded
    device loops; no hang) and the handle stays usable."""
    g = G.path(5000, 1, 9, 3)
    with st.SteinerGraph(g) as Gd:
        Gd.set_param("max_iters", 10)
        assert Gd.query([0, 4999]).status == st.STEINER_ETIMEOUT
        Gd.set_param("max_iters", 1 << 22)
        res = Gd.query([0, 4999])
    ref = oracle.steiner(g, [0, 4999], want_labels=False)
    assert res.status == st.STEINER_OK and res.total == ref.total


def test_autotuner_changes_time_not_results(tmp_path):
    from paper_2205_14503_gb300 import autotune
    g = wl.grid(300, 300, 1000, seed=5)
    seeds = G.seeds_from(np.arange(g.n), 20, 5)
    ref = oracle.steiner(g, seeds, want_labels=False)
    cache = str(tmp_path / "tune.json")
    with st.SteinerGraph(g) as Gd:
        entry = autotune.tune(Gd, g, [seeds], delta_factors=(0.5, 2), block_fractions=(0.5, 1.0),
                              local_rounds=(0, 8), reps=1, cache_path=cache)
        assert Gd.get_param("delta") == entry["delta"]
        assert Gd.get_param("sssp_blocks") == entry["sssp_blocks"]
        res = Gd.query(seeds)
    assert np.array_equal(res.edges, ref.edges) and res.total == ref.total
    with st.SteinerGraph(g) as Gd:
        assert autotune.apply_cached(Gd, g, cache) == entry
        assert Gd.get_param("sssp_blocks") == entry["sssp_blocks"]
        res = Gd.query(seeds)
    assert np.array_equal(res.edges, ref.edges)


@pytest.mark.parametrize("local", [1, 4, 64])
def test_block_local_rounds_on_grids(local):
    """High-diameter graphs are where block-local rounds run many hops."""
    for side, k, wmax in [(200, 9, 1000), (150, 40, 1), (300, 5, 3)]:
        g = wl.grid(side, side, wmax, seed=side + local)
        seeds = G.seeds_from(np.arange(g.n), k, side)
        ref = oracle.steiner(g, seeds, want_labels=True)
        with st.SteinerGraph(g) as Gd:
            Gd.set_param("local_rounds", local)
            rc, cell, dist, pred = Gd.voronoi(seeds)
            res = Gd.query(seeds)
        np.testing.assert_array_equal(cell, ref.cell)
        np.testing.assert_array_equal(dist, ref.dist)
        np.testing.assert_array_equal(pred, ref.pred)
        np.testing.assert_array_equal(res.edges, ref.edges)


def _compare_forced(g, seeds, **params):
    """_compare with handle parameters set first; returns the handle's
    label-width counters after the two calls."""
    ref = oracle.steiner(g, seeds, want_labels=True, want_pairs=True)
    with st.SteinerGraph(g) as Gd:
        for key, value in params.items():
            Gd.set_param(key, value)
        rc, cell, dist, pred = Gd.voronoi(seeds)
        res = Gd.query_detail(seeds)
        counters = {k: Gd.get_param(k) for k in ("label_bits_last", "narrow_reruns")}
        counters["pull_passes"] = Gd.get_param("pull_passes_last")
        counters["tail_iteration"] = Gd.get_param("tail_iteration_last")
    assert rc == st.STEINER_OK and res.status == ref.status == oracle.OK, st.last_error()
    np.testing.assert_array_equal(cell, ref.cell)
    np.testing.assert_array_equal(dist, ref.dist)
    np.testing.assert_array_equal(pred, ref.pred)
    np.testing.assert_array_equal(res.pairs[:, :4], ref.pairs)
    np.testing.assert_array_equal(res.edges, ref.edges)
    assert res.total == ref.total
    return counters


@pytest.mark.parametrize("bits", [32, 64])
def test_label_width_forced(bits):
    """Both label widths reach the oracle's fixed point: a 32-bit label
    packs (distance << rank bits) | rank, a 64-bit one (distance << 32) |
    rank, both ordered by (distance, rank).  Hubs in chunked rows with many
    seeds, unit weights (maximal ties), a grid with the light/heavy split,
    and a sparse random graph."""
    cases = [(wl.rmat(14, 16, wmax=1000, seed=41), 500, True),
             (wl.rmat(12, 16, wmax=1, seed=42), 200, True),
             (wl.grid(150, 110, 1000, seed=43), 60, False),
             (G.random_connected(3000, 2000, 1, 50, 44), 30, False)]
    for g, k, lcc in cases:
        pool = wl.largest_cc(g) if lcc else np.arange(g.n, dtype=np.int32)
        seeds = wl.sample_distinct(pool, k, 40 + k)
        for delta in (None, 150):
            params = {"label_bits": bits} if delta is None else {"label_bits": bits, "delta": delta}
            c = _compare_forced(g, seeds, **params)
            assert (c["label_bits_last"], c["narrow_reruns"]) == (bits, 0)


def test_narrow_labels_fall_back_to_64_bits():
    """A query whose distances do not fit a 32-bit label is rerun with
    64-bit labels and still equals the oracle.  Here 4096 seeds sit at one
    end of a 50,000-vertex path (12 rank bits leave 20 distance bits, so
    distances up to about 10^6) and the far end lies about 2 * 10^7 away.
    The automatic choice picks 32 bits (weights below 512 leave 11 spare
    bits), falls back once, and then takes 64 bits up front for queries
    with as few distance bits."""
    n = 50_000
    rng = np.random.default_rng(7)
    g = wl.from_edges(n, np.arange(n - 1), np.arange(1, n), rng.integers(400, 512, n - 1))
    seeds = np.arange(4096, dtype=np.int32)
    c = _compare_forced(g, seeds, label_bits=32)
    assert (c["label_bits_last"], c["narrow_reruns"]) == (64, 2)
    c = _compare_forced(g, seeds)
    assert (c["label_bits_last"], c["narrow_reruns"]) == (64, 1)


@pytest.mark.parametrize("far_scan", [0, 1])
@pytest.mark.parametrize("delta,local", [(50, 0), (999, 8), (5000, 0), (5000, 16)])
def test_band_split_by_pile_or_scan(far_scan, delta, local):
    """A band split finds the vertices left for later bands either from a
    pile of far proposals or by scanning every label; both, with and without
    the light/heavy split and warp-local rounds, give the oracle's labels,
    distance graph and tree."""
    for g, k, lcc in ((wl.grid(150, 110, 1000, seed=51), 60, False),
                      (wl.rmat(12, 48, wmax=1000, seed=52), 25, True)):
        pool = wl.largest_cc(g) if lcc else np.arange(g.n, dtype=np.int32)
        seeds = wl.sample_distinct(pool, k, 50 + k)
        _compare_forced(g, seeds, far_scan=far_scan, delta=delta, local_rounds=local)


@pytest.mark.parametrize("tail", [0, 1])
@pytest.mark.parametrize("pull", [0, 1, 2])
@pytest.mark.parametrize("bits", [32, 64])
def test_heavy_pass_push_or_pull(pull, bits, tail):
    """A band's heavy-arc pass pushes the heavy arcs of the band's vertices
    (pull 0), reads them from the unsettled side (pull 2: every vertex at or
    above the threshold takes the best proposal from its settled heavy-arc
    neighbours), or picks the form that reads fewer arcs (pull 1); after a
    pull pass the rest runs as one unbounded band over whole rows (tail 1)
    or keeps its bands (tail 0).  All reach the oracle's labels, distance
    graph and tree, on skewed and flat graphs, dense and sparse frontiers,
    many bands and few."""
    cases = [(wl.rmat(14, 16, wmax=1000, seed=81), 400, True, 125),
             (wl.rmat(13, 16, wmax=1000, seed=82), 7, True, 31),
             (wl.grid(150, 110, 1000, seed=83), 60, False, 200),
             (G.random_connected(4000, 3000, 1, 300, 84), 40, False, 60)]
    for g, k, lcc, delta in cases:
        pool = wl.largest_cc(g) if lcc else np.arange(g.n, dtype=np.int32)
        seeds = wl.sample_distinct(pool, k, 80 + k)
        for dense in (0, 1):
            c = _compare_forced(g, seeds, pull=pull, delta=delta, dense=dense, far_scan=1,
                                label_bits=bits, tail=tail)
            if pull == 0:
                assert c["pull_passes"] == 0 and c["tail_iteration"] == 0
            elif pull == 2:
                assert c["pull_passes"] > 0
            if tail == 0:
                assert c["tail_iteration"] == 0
            elif pull == 2:
                # the first pull pass starts the tail, unless it converged
                assert c["pull_passes"] == 1


def test_heavy_pass_pull_chosen_on_small_world_graphs():
    """With the cost rule, the first band of an R-MAT query (most vertices
    and nearly all heavy arcs) runs its heavy-arc pass in the pull form."""
    g = wl.rmat(15, 16, wmax=1000, seed=85)
    seeds = wl.sample_distinct(wl.largest_cc(g), 30, 86)
    c = _compare_forced(g, seeds, pull=1, delta=125, far_scan=1)
    assert c["pull_passes"] == 1 and c["tail_iteration"] > 0


@pytest.mark.parametrize("wmax", [10_000, 100_000])
@pytest.mark.parametrize("mode", ["tuned", "frontier"])
def test_wide_weight_ranges(wmax, mode):
    """The weight-range study's wide ranges (weights uniform in [1, 10^4]
    and [1, 10^5] on R-MAT): cells, distances, preds, the distance graph
    and the tree equal the oracle's, at a band width scaled to the weights
    (with the light/heavy split) and as a plain frontier (one unbounded
    band)."""
    g = wl.rmat(15, 16, wmax=wmax, seed=61 + wmax % 97)
    seeds = wl.sample_distinct(wl.largest_cc(g), 48, 62)
    delta = max(1, wmax // 8) if mode == "tuned" else 0x7FFFFFFF
    _compare_forced(g, seeds, delta=delta)


@pytest.mark.parametrize("strategy", ["bfs_level", "eccentric", "proximate"])
def test_seed_selection_strategies(strategy):
    """The seed-selection study's strategies (BFS-level, eccentric and
    proximate k-BFS seeds) as inputs to the CUDA path, against the oracle
    element by element, on an R-MAT graph and a grid."""
    for g, lcc in ((wl.rmat(14, 16, wmax=1000, seed=71), True),
                   (wl.grid(96, 80, 1000, seed=72), False)):
        pool = wl.largest_cc(g) if lcc else np.arange(g.n, dtype=np.int32)
        make = {"bfs_level": wl.seeds_bfs_level, "eccentric": wl.seeds_eccentric,
                "proximate": wl.seeds_proximate}[strategy]
        seeds = make(g, pool, 40, 73)
        _compare_forced(g, seeds)


@pytest.mark.parametrize("dense", [0, 1])
@pytest.mark.parametrize("relabel", ["0", "1"])
def test_dense_frontiers(dense, relabel, monkeypatch):
    """Large frontiers and the band lists of the light/heavy split kept as
    bitmaps read in vertex order (dense) or as queues; with the internal
    degree order (hubs first, so an id tells a light vertex) and without;
    band widths below, near and above the weights.  Every output equals
    the oracle's."""
    monkeypatch.setenv("STEINER_RELABEL", relabel)
    for g, k in ((wl.rmat(14, 16, wmax=1000, seed=81), 400),
                 (wl.rmat(13, 48, wmax=100, seed=82), 60)):
        seeds = wl.sample_distinct(wl.largest_cc(g), k, 83)
        for delta in (30, 200, 5000):
            _compare_forced(g, seeds, dense=dense, far_scan=1, delta=delta, local_rounds=0)
