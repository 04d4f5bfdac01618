"""Host logic of the autotuner, without a GPU: a stand-in handle answers
queries with times from a fixed cost model, and the tuner must find that
model's optimum, refine the band width between its grid points, and keep
or drop the unbounded tail by its measured time."""
import types

import numpy as np

from paper_2205_14503_gb300 import autotune
from paper_2205_14503_gb300 import steiner as st


class FakeHandle:
    """set_param/get_param like a graph handle; query_detail returns a
    result whose phase times come from `cost(params)`."""

    def __init__(self, cost, delta0=1000, max_blocks=456, sm=152):
        self.p = {"delta": delta0, "sssp_max_blocks": max_blocks, "sm_count": sm,
                  "sssp_blocks": max_blocks, "local_rounds": 0, "label_bits": 0,
                  "far_scan": -1, "tail": 1}
        self.cost = cost
        self.queries = 0

    def set_param(self, key, value):
        self.p[key] = value

    def get_param(self, key):
        return self.p[key]

    def query_detail(self, seeds, pairs=False):
        self.queries += 1
        ms = self.cost(self.p)
        stats = {"ms_init": 0.0, "ms_voronoi": ms, "ms_bridges": 1.0, "ms_mst": 0.0,
                 "ms_tree": 0.0}
        return types.SimpleNamespace(status=st.STEINER_OK, stats=stats)


def _graph():
    g = types.SimpleNamespace(n=4, row_ptr=np.array([0, 1, 2, 3, 4], np.uint32),
                              col=np.array([1, 0, 3, 2], np.int32),
                              w=np.array([5, 5, 7, 7], np.uint32))
    g.n_arcs = 4
    return g


def test_refines_delta_between_grid_points_and_keeps_the_tail():
    # optimum near delta 45: between the grid points 31 (1/32) and 62 (1/16)
    def cost(p):
        return abs(np.log(p["delta"] / 45.0)) + (0.5 if p["tail"] == 0 else 0.0) + \
            (0.2 if p["local_rounds"] else 0.0) + (0.1 if p["sssp_blocks"] != 456 else 0.0)

    G = FakeHandle(cost)
    e = autotune.tune(G, _graph(), [np.array([0, 2], np.int32)], cache_path=None, reps=1)
    assert e["delta"] == 44           # 62 * 0.707, the refined point nearest 45
    assert (e["sssp_blocks"], e["local_rounds"], e["tail"]) == (456, 0, 1)
    assert G.p["delta"] == 44 and G.p["tail"] == 1


def test_drops_the_tail_when_the_bands_are_faster():
    def cost(p):
        return abs(np.log(p["delta"] / 125.0)) + (0.0 if p["tail"] == 0 else 0.3)

    G = FakeHandle(cost)
    e = autotune.tune(G, _graph(), [np.array([0, 2], np.int32)], cache_path=None, reps=1)
    assert e["delta"] == 125 and e["tail"] == 0
    assert G.p["tail"] == 0
    assert e["ms_query"] == e["ms_no_tail"]


def test_apply_cached_restores_every_choice(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "_gpu_name", lambda device: "fake")
    G = FakeHandle(lambda p: abs(np.log(p["delta"] / 250.0)))
    path = str(tmp_path / "cache.json")
    g = _graph()
    e = autotune.tune(G, g, [np.array([0, 2], np.int32)], cache_path=path, reps=1)
    H = FakeHandle(lambda p: 0.0)
    H.p["tail"] = 0
    got = autotune.apply_cached(H, g, cache_path=path)
    assert got["delta"] == e["delta"] == 250
    for key in ("delta", "sssp_blocks", "local_rounds", "label_bits", "far_scan", "tail"):
        assert H.p[key] == e[key]


class FakeBatchHandle(FakeHandle):
    """query_batch advances a fake wall clock by `bcost(params)` ms."""

    def __init__(self, bcost, clock, **kw):
        super().__init__(lambda p: 0.0, **kw)
        self.p.update({"batch_delta": 0, "batch_pull": 1})
        self.bcost = bcost
        self.clock = clock

    def query_batch(self, queries):
        self.clock[0] += self.bcost(self.p) / 1e3
        return st.STEINER_OK, []


def _fake_clock(monkeypatch):
    import time
    clock = [0.0]
    monkeypatch.setattr(time, "perf_counter", lambda: clock[0])
    return clock


def test_tune_batch_picks_width_then_push_or_pull(monkeypatch):
    clock = _fake_clock(monkeypatch)
    g = _graph()
    g.w = np.array([1000, 1000, 7, 7], np.uint32)        # w_max 1000: widths 31 .. 500

    def bcost(p):
        return abs(np.log(p["batch_delta"] / 250.0)) * 10 + (3.0 if p["batch_pull"] else 1.0)

    G = FakeBatchHandle(bcost, clock, delta0=45)
    e = autotune.tune_batch(G, g, [np.array([0, 2], np.int32)], reps=1)
    assert (e["batch_delta"], e["batch_pull"]) == (250, 0)       # push measured faster here
    assert (G.p["batch_delta"], G.p["batch_pull"]) == (250, 0)
    assert abs(e["ms_push"] - 1.0) < 1e-6

    G = FakeBatchHandle(lambda p: abs(np.log(p["batch_delta"] / 125.0)) * 10 +
                        (1.0 if p["batch_pull"] else 3.0), clock, delta0=45)
    e = autotune.tune_batch(G, g, [np.array([0, 2], np.int32)], reps=1)
    assert (e["batch_delta"], e["batch_pull"]) == (125, 1)
