"""GPU parity of the multi-query modes: steiner_query_batch and the serving
calls give, for every query, exactly the tree (edges, total, status) that
the CPU oracle and the single-query path give — alone and in the mix."""
import time

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


def _queries(pool, sizes, salt):
    return [wl.sample_distinct(pool, int(k), salt * 1000 + i) for i, k in enumerate(sizes)]


def _check(g, seed_sets, results):
    for i, (seeds, r) in enumerate(zip(seed_sets, results)):
        ref = oracle.steiner(g, seeds, want_labels=False)
        assert r.status == ref.status, (i, r.status, ref.status)
        np.testing.assert_array_equal(r.edges, ref.edges, err_msg=f"query {i}")
        assert r.total == ref.total, i


@pytest.mark.parametrize("tails", [0, 1])
def test_batch_64_queries_log_uniform_sizes(tails):
    """64 queries in one batch; the tails (MST, expansion, sorted edges) of
    the queries that finish together run batched (1) or one at a time (0)."""
    g = wl.rmat(14, 16, wmax=1000, seed=41)
    pool = wl.largest_cc(g)
    sizes = wl.log_uniform_sizes(64, 3, 300, 7)
    qs = _queries(pool, sizes, 1)
    with st.SteinerGraph(g) as Gd:
        Gd.set_param("batch_tails", tails)
        rc, res = Gd.query_batch(qs)
        batches = Gd.get_param("batch_tail_batches")
    assert rc == st.STEINER_OK
    assert (batches > 0) == bool(tails)
    _check(g, qs, res)


def test_batch_more_queries_than_slots_reuses_slots():
    g = wl.rmat(13, 16, wmax=100, seed=42)
    pool = wl.largest_cc(g)
    sizes = wl.log_uniform_sizes(150, 2, 120, 8)
    qs = _queries(pool, sizes, 2)
    with st.SteinerGraph(g) as Gd:
        rc, res = Gd.query_batch(qs)
        single = [Gd.query(s) for s in qs[:20]]
    assert rc == st.STEINER_OK
    _check(g, qs, res)
    for a, b in zip(res[:20], single):     # same in the batch as alone
        assert np.array_equal(a.edges, b.edges) and a.total == b.total


@pytest.mark.parametrize("tails", [0, 1])
def test_batch_high_diameter_grid(tails):
    g = wl.grid(300, 200, 1000, seed=43)
    pool = np.arange(g.n, dtype=np.int32)
    qs = _queries(pool, [2, 5, 17, 64, 3, 200, 9, 40], 3)
    with st.SteinerGraph(g) as Gd:
        Gd.set_param("batch_tails", tails)
        rc, res = Gd.query_batch(qs)
    assert rc == st.STEINER_OK
    _check(g, qs, res)


@pytest.mark.parametrize("tails", [0, 1])
def test_batch_mixed_statuses_and_degenerate_queries(tails):
    """Disconnected seed sets (forests), a single seed, duplicates, an
    unreachable vertex and an overflowing distance in one batch."""
    big = 0xFFFFFFFF // 2 + 1
    e = np.array([[0, 1, 3], [1, 2, 4], [3, 4, 5], [4, 5, 1], [5, 6, 2], [0, 2, 9],
                  [9, 10, big], [10, 11, big]])
    g = wl.from_edges(12, e[:, 0], e[:, 1], e[:, 2])
    qs = [np.array([0, 2]), np.array([0, 5]), np.array([4]), np.array([3, 3]),
          np.array([1, 2, 3, 6]), np.array([8, 0]), np.array([2, 0, 1]), np.array([9, 11]),
          np.array([9, 10, 1, 4])]
    with st.SteinerGraph(g) as Gd:
        Gd.set_param("batch_tails", tails)
        rc, res = Gd.query_batch(qs)
        alone = [Gd.query(s) for s in qs]
    assert rc != st.STEINER_OK
    for s, r, a in zip(qs, res, alone):
        ref = oracle.steiner(g, s, want_labels=False)
        assert r.status == ref.status == a.status
        if ref.status in (oracle.OK, oracle.EDISCONNECTED):
            np.testing.assert_array_equal(r.edges, ref.edges)
            assert r.total == ref.total


@pytest.mark.parametrize("nq", [1, 5, 17, 33, 47])
def test_batch_scan_slot_layouts(nq):
    """The batched pred + bridge scan takes slot pairs per lane above 32
    slots and lane groups below; odd counts leave half pairs and idle lanes,
    and the hub rows (degree >= 256) go through the chunked, atomic path."""
    g = wl.rmat(13, 16, wmax=1000, seed=47)
    assert np.diff(g.row_ptr).max() >= 256
    pool = wl.largest_cc(g)
    qs = _queries(pool, wl.log_uniform_sizes(nq, 2, 150, 10 + nq), 5 + nq)
    with st.SteinerGraph(g) as Gd:
        rc, res = Gd.query_batch(qs)
    assert rc == st.STEINER_OK
    _check(g, qs, res)


def test_batch_unit_weights_ties():
    g = wl.rmat(12, 16, wmax=1, seed=44)
    pool = wl.largest_cc(g)
    qs = _queries(pool, wl.log_uniform_sizes(40, 2, 200, 9), 4)
    with st.SteinerGraph(g) as Gd:
        rc, res = Gd.query_batch(qs)
    assert rc == st.STEINER_OK
    _check(g, qs, res)


def test_serving_stream_matches_alone():
    """Requests submitted while others run (continuous batching) give the
    same trees as each query alone."""
    g = wl.rmat(14, 16, wmax=1000, seed=45)
    pool = wl.largest_cc(g)
    sizes = wl.log_uniform_sizes(120, 3, 500, 10)
    qs = _queries(pool, sizes, 5)
    arrivals = wl.poisson_arrivals(len(qs), 4000.0, 11)
    with st.SteinerGraph(g) as Gd:
        h = Gd.handle
        st.steiner_serve_start(h, 64, 8 << 30)
        tickets, t0 = [], time.perf_counter()
        for s, at in zip(qs, arrivals):
            while time.perf_counter() - t0 < at:
                pass
            rc, t = st.steiner_submit(h, s)
            assert rc == st.STEINER_OK
            tickets.append(t)
        results = {}
        deadline = time.time() + 120
        while len(results) < len(tickets) and time.time() < deadline:
            for t in tickets:
                if t in results:
                    continue
                rc, r = st.steiner_poll(h, t)
                if rc != st.STEINER_PENDING:
                    results[t] = r
            time.sleep(0.001)
        # a result is handed out once: the ticket is unknown afterwards
        rc_again, r_again = st.steiner_poll(h, tickets[0])
        launches = st.steiner_get_param(h, "batch_launches")
        admitted = st.steiner_get_param(h, "batch_admitted")
        admitted_busy = st.steiner_get_param(h, "batch_admitted_busy")
        st.steiner_serve_stop(h)
        alone = [Gd.query(s) for s in qs[:30]]
    assert rc_again == st.STEINER_EINVAL and r_again is None
    # continuous batching happened: queries joined while others were on the
    # device, and far fewer kernel launches ran than there were queries
    assert admitted == sum(1 for s in qs if len(s) > 1)
    assert admitted_busy > 0
    assert 0 < launches < len(qs)
    assert len(results) == len(tickets)
    res = [results[t] for t in tickets]
    _check(g, qs, res)
    for a, b in zip(res[:30], alone):
        assert np.array_equal(a.edges, b.edges) and a.total == b.total


def test_serving_budget_refusals():
    g = wl.rmat(11, 8, wmax=50, seed=46)
    pool = wl.largest_cc(g)
    with st.SteinerGraph(g) as Gd:
        h = Gd.handle
        with pytest.raises(st.SteinerError):
            st.steiner_serve_start(h, 64, 1024)             # below the per-slot label state
        fixed = g.n * 64 * 12
        st.steiner_serve_start(h, 4, fixed + 8 * 1000)       # room for pair tables of k <= ~45
        rc, t_big = st.steiner_submit(h, wl.sample_distinct(pool, 400, 1))
        rc2, t_ok = st.steiner_submit(h, wl.sample_distinct(pool, 20, 2))
        got = {}
        deadline = time.time() + 60
        while len(got) < 2 and time.time() < deadline:
            for t in (t_big, t_ok):
                if t not in got:
                    r, res = st.steiner_poll(h, t)
                    if r != st.STEINER_PENDING:
                        got[t] = (r, res)
            time.sleep(0.001)
        st.steiner_serve_stop(h)
    assert got[t_big][0] == st.STEINER_EBUSY
    assert got[t_ok][0] == st.STEINER_OK


@pytest.mark.parametrize("pull", [0, 1])
@pytest.mark.parametrize("batch_delta", [1, 100, 999])
def test_batch_light_heavy_split(batch_delta, pull):
    """Band widths at or below the largest weight switch on the per-slot
    light/heavy arc split of the batched kernel (heavy-arc passes of
    different slots interleaved with other slots' bands); a slot's first
    heavy-arc pass pushes the band's heavy arcs (pull 0) or lets every
    vertex unsettled in that slot read its own (pull 1), while other slots
    push or relax in the same iterations.  Trees equal the oracle's on a
    grid and on an R-MAT graph with hubs."""
    for g, grid in ((wl.grid(160, 120, 1000, seed=47), True), (wl.rmat(12, 48, wmax=1000, seed=48), False)):
        pool = np.arange(g.n, dtype=np.int32) if grid else wl.largest_cc(g)
        qs = _queries(pool, [2, 9, 40, 3, 120, 17, 64, 5], 6 + batch_delta)
        with st.SteinerGraph(g) as Gd:
            Gd.set_param("batch_delta", batch_delta)
            Gd.set_param("batch_pull", pull)
            rc, res = Gd.query_batch(qs)
            sweeps = Gd.get_param("batch_pull_sweeps")
        assert rc == st.STEINER_OK
        assert (sweeps > 0) == bool(pull)
        _check(g, qs, res)


def test_batched_tails_many_seeds_and_shared_vertices():
    """Tails of queries with large seed sets (pair tables of many tiles, the
    MST over thousands of pairs in one block) finishing together, on an
    R-MAT graph whose hubs lie in many queries' trees (the walkers of
    different queries cross the same vertices): batched and one-at-a-time
    tails give the oracle's trees."""
    g = wl.rmat(15, 16, wmax=100, seed=48)
    pool = wl.largest_cc(g)
    qs = _queries(pool, [2000, 3, 700, 2000, 64, 1500, 9, 2], 6)
    out = {}
    for tails in (1, 0):
        with st.SteinerGraph(g) as Gd:
            Gd.set_param("batch_tails", tails)
            rc, out[tails] = Gd.query_batch(qs)
            if tails:
                assert Gd.get_param("batch_tail_batches") > 0
        assert rc == st.STEINER_OK
    _check(g, qs, out[1])
    for a, b in zip(out[1], out[0]):
        assert np.array_equal(a.edges, b.edges) and a.total == b.total


def test_batch_labels_that_outgrow_32_bits():
    """The engine keeps 32-bit labels, (distance << b) | rank with b the bits
    of the slot's largest rank; a query whose distances do not fit (here a
    path of weight-10^6 edges with up to 1000 seeds at one end: 10 rank bits
    leave distances below about 4 * 10^6) is answered by the single-query
    path, and every tree equals the oracle's."""
    n = 4000
    rng = np.random.default_rng(9)
    g = wl.from_edges(n, np.arange(n - 1), np.arange(1, n), rng.integers(900_000, 1_000_001, n - 1))
    qs = [np.arange(1000, dtype=np.int32), np.array([0, 5, 17]), np.arange(0, 600, 2),
          np.array([10, 3990]), np.arange(200, dtype=np.int32)]
    with st.SteinerGraph(g) as Gd:
        rc, res = Gd.query_batch(qs)
        reruns = Gd.get_param("batch_narrow_reruns")
    assert rc == st.STEINER_OK
    assert reruns >= 1
    _check(g, qs, res)
