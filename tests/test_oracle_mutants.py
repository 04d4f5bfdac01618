"""Planted mistakes in the CPU oracle must be caught by its pins.

Each mutant is a copy of ``oracle/steiner_oracle.c`` with one plausible
mistake (a dropped term, a wrong index, a reversed tie rule, a missing
step), compiled with gcc into a temporary library.  The pin battery of
``test_oracle_pins`` runs against it and at least one pin must fail.
Everything here runs on the CPU.  Each battery runs in a child process, so
a mutant that crashes the oracle (for instance by leaving a reached vertex
without a predecessor) also counts as caught.
"""
import json
import os
import subprocess
import sys

import pytest

import oracle
from tests import test_oracle_pins as pins

MUTANTS = {
    "bridge_drops_far_distance": (
        "uint64_t b = (uint64_t)dist[u] + w[e] + dist[v];",
        "uint64_t b = (uint64_t)dist[u] + w[e];"),
    "bridge_from_larger_rank": [
        ("rank[u] >= rank[v]) continue;", "rank[u] <= rank[v]) continue;"),
        ("pair_t *p = &tab[pair_slot(rank[u], rank[v], k)];",
         "pair_t *p = &tab[pair_slot(rank[v], rank[u], k)];"),
        ("p->ra = rank[u]; p->rb = rank[v];", "p->ra = rank[v]; p->rb = rank[u];")],
    "voronoi_tie_to_larger_rank": (
        "(a.dist == b.dist && a.rank < b.rank)",
        "(a.dist == b.dist && a.rank > b.rank)"),
    "relax_with_wrong_arc_weight": (
        "label_t cand = { lab[u].dist + w[e], lab[u].rank };",
        "label_t cand = { lab[u].dist + w[row_ptr[u]], lab[u].rank };"),
    "pred_takes_largest_id": (
        "pred[v] = (int32_t)u;      /* rows are sorted: first hit = smallest id */\n                break;",
        "pred[v] = (int32_t)u;"),
    "pred_ignores_cell": (
        "if (lab[u].rank == lab[v].rank && lab[u].dist + w[e] == lab[v].dist)",
        "if (lab[u].dist + w[e] == lab[v].dist)"),
    "seeds_not_ranked_by_id": (
        "qsort(s, k, sizeof(int32_t), cmp_i32);",
        ";"),
    "kruskal_heaviest_first": (
        "if (a->b != b->b) return a->b < b->b ? -1 : 1;",
        "if (a->b != b->b) return a->b > b->b ? -1 : 1;"),
    "kruskal_rank_tie_reversed": (
        "if (a->ra != b->ra) return a->ra < b->ra ? -1 : 1;",
        "if (a->ra != b->ra) return a->ra > b->ra ? -1 : 1;"),
    "tree_misses_bridge_edge": (
        "edges[ne++] = be;",
        "(void)be;"),
    "tree_walks_one_side_only": (
        "for (int side = 0; side < 2; ++side) {",
        "for (int side = 0; side < 1; ++side) {"),
    "tree_weight_of_wrong_edge": (
        "edge_weight(row_ptr, col, w, x, p)",
        "edge_weight(row_ptr, col, w, x, (uint32_t)col[row_ptr[x]])"),
    "no_disconnected_status": (
        "if (nm + 1 < k) rc = ORC_EDISCONNECTED;",
        ";"),
    "no_overflow_check_on_bridges": (
        "if (b >= DIST_INF) rc = ORC_EOVERFLOW;",
        ";"),
}


def _battery():
    """The pins, as (name, callable) pairs."""
    out = []
    for f in pins.WORKED:
        out.append((f"golden:{f}", lambda f=f: pins.test_golden_worked_example(f)))
    for name, g, k in pins.CASES[:6] + pins.CASES[7:8]:
        out.append((f"voronoi:{name}", lambda a=(name, g, k): pins.test_voronoi_equals_min_over_seed_dijkstra(*a)))
        out.append((f"pred:{name}", lambda a=(name, g, k): pins.test_pred_chains_are_shortest_paths_to_own_seed(*a)))
        out.append((f"mehlhorn:{name}", lambda a=(name, g, k): pins.test_mehlhorn_mst_weight_equals_kmb_mst_weight(*a)))
        out.append((f"tree:{name}", lambda a=(name, g, k): pins.test_tree_invariants_and_kmb_bound(*a)))
    out += [
        ("bridge_enum", pins.test_bridge_minimum_by_enumeration),
        ("k2_path", pins.test_two_seeds_give_a_shortest_path),
        ("s_eq_v", pins.test_seed_set_equal_to_vertex_set_gives_textbook_mst),
        ("tree_graph", pins.test_tree_shaped_graph_gives_the_exact_steiner_tree),
        ("dreyfus_wagner", pins.test_dreyfus_wagner_two_approximation_bound),
        ("disconnected", pins.test_disconnected_seeds_give_a_spanning_forest),
        ("overflow", pins.test_distance_overflow_is_reported),
    ]
    return out


def _run_battery_in_child(lib_path):
    """Failing pin names, or ["<crash: signal>"] if the child died."""
    code = ("import json, oracle; from tests import test_oracle_mutants as m; "
            f"print('RESULT' + json.dumps(m._failures(oracle._bind(__import__('ctypes').CDLL({lib_path!r})))))")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    p = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True,
                       timeout=600)
    for line in p.stdout.splitlines():
        if line.startswith("RESULT"):
            return json.loads(line[len("RESULT"):])
    return [f"<crash: returncode {p.returncode}>"]


def _failures(lib):
    failed = []
    pins.LIB = lib
    try:
        for name, fn in _battery():
            try:
                fn()
            except (AssertionError, IndexError, KeyError, ValueError):
                failed.append(name)
    finally:
        pins.LIB = None
    return failed


def test_unmutated_oracle_passes_the_battery():
    assert _failures(None) == []


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_planted_mistake_is_caught(mutant, tmp_path):
    edits = MUTANTS[mutant]
    if isinstance(edits, tuple):
        edits = [edits]
    src = oracle.source_text()
    for old, new in edits:
        assert src.count(old) == 1, f"mutation anchor for {mutant} not unique"
        src = src.replace(old, new)
    path = str(tmp_path / f"mut_{mutant}.so")
    oracle.compile_variant(src, path)
    failed = _run_battery_in_child(path)
    assert failed, f"no pin caught the planted mistake {mutant}"
