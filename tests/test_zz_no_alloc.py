"""steiner_voronoi_noalloc: the allocation-free Voronoi entry point.

It serves callers that cannot call cudaMalloc (a framework that owns every
device allocation through its own pool, or code that must not grow its
device footprint), so these tests hand it only caller-allocated tensors and
compare its output, exactly, with the regular steiner_voronoi entry point on
two calls in a row (the second call must not see the first call's state).
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import paper_2205_14503_gb300.workloads as wl

pytestmark = pytest.mark.gpu

st = pytest.importorskip("paper_2205_14503_gb300.steiner")
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_14503_gb300 import build
    build.build()
    st.load_library()


def _dev(a):
    """numpy 4-byte array -> CUDA int32 tensor with the same bits."""
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32).copy()).cuda()


def _reference(g, seeds):
    with st.SteinerGraph(g) as G:
        rc, cell, dist, pred = G.voronoi(seeds)
    assert rc == st.STEINER_OK
    return cell, dist, pred


def test_noalloc_matches_regular_entry_on_two_calls_in_a_row():
    g = wl.rmat(15, 16, wmax=100, seed=77)
    pool = wl.largest_cc(g)
    row_ptr, col, w = _dev(g.row_ptr), _dev(g.col), _dev(g.w)
    for call, (k, salt) in enumerate([(24, 1), (300, 2)]):
        seeds = np.sort(wl.sample_distinct(pool, k, salt))
        cell = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
        dist = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
        pred = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
        rc = st.steiner_voronoi_noalloc(row_ptr, col, w, _dev(seeds), cell, dist, pred)
        assert rc == st.STEINER_OK, st.last_error()
        ref_cell, ref_dist, ref_pred = _reference(g, seeds)
        np.testing.assert_array_equal(cell.cpu().numpy(), ref_cell, err_msg=f"call {call}")
        np.testing.assert_array_equal(dist.cpu().numpy().view(np.uint32), ref_dist)
        np.testing.assert_array_equal(pred.cpu().numpy(), ref_pred)


def test_noalloc_rejects_sizes_beyond_its_scratch_limit():
    lib = st.load_library()
    limit = 1048576
    small = torch.zeros(4, dtype=torch.int32, device="cuda")
    p = small.data_ptr()
    rc = lib.steiner_voronoi_noalloc(p, p, p, limit + 1, 2, p, 1, p, p, p, None)
    assert rc == st.STEINER_ENOMEM
    assert "limit" in st.last_error()


def test_noalloc_rejects_unsorted_seeds():
    g = wl.grid(40, 30, 9, seed=5)
    row_ptr, col, w = _dev(g.row_ptr), _dev(g.col), _dev(g.w)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    rc = st.steiner_voronoi_noalloc(row_ptr, col, w, _dev(np.array([50, 7], np.int32)), out, out, out)
    assert rc == st.STEINER_EINVAL
    seeds = np.array([7, 50, 1100], np.int32)
    cell = torch.empty(g.n, dtype=torch.int32, device="cuda")
    rc = st.steiner_voronoi_noalloc(row_ptr, col, w, _dev(seeds), cell, None, None)
    assert rc == st.STEINER_OK
    np.testing.assert_array_equal(cell.cpu().numpy(), _reference(g, seeds)[0])


def test_noalloc_rejects_bad_row_offsets_and_leaves_outputs_untouched():
    """Row offsets that decrease, or that do not end at the arc count, are
    caught before any arc is read; the outputs keep their contents; the
    next call with good offsets works."""
    g = wl.grid(40, 30, 9, seed=6)
    col, w = _dev(g.col), _dev(g.w)
    seeds = np.array([7, 50, 1100], np.int32)
    bad = g.row_ptr.copy()
    bad[100] = bad[102]                  # row 100 would start after its end
    for rp, c in ((bad, col), (g.row_ptr, col[:-2])):    # decreasing; row_ptr[n] != n_arcs
        cell = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
        rc = st.steiner_voronoi_noalloc(_dev(rp), c, w, _dev(seeds), cell, cell, cell)
        assert rc == st.STEINER_EINVAL
        assert "row_ptr" in st.last_error()
        assert bool((cell == -7).all())
    cell = torch.empty(g.n, dtype=torch.int32, device="cuda")
    rc = st.steiner_voronoi_noalloc(_dev(g.row_ptr), col, w, _dev(seeds), cell, None, None)
    assert rc == st.STEINER_OK
    np.testing.assert_array_equal(cell.cpu().numpy(), _reference(g, seeds)[0])
