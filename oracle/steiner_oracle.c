/*
 * CPU oracle for the Voronoi-cell 2-approximation Steiner tree
 * (Mehlhorn's construction as parallelised in the paper, Algorithm 2).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously
 * correct reference that the CUDA path is checked against.  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load it;
 * the library's product path never does.  It shares no code, header,
 * table or helper with the CUDA path.
 *
 * Steps, in the paper's order (Algorithm 2):
 *   Step 1  Voronoi cells: every vertex u gets src(u), pred(u), d1(src(u),u)
 *           (Section "Preliminaries" defines N(s); Algorithm 4 computes it).
 *           Here: multi-source Dijkstra keyed by (distance, seed rank).
 *   Step 2  Distance graph G'_1: for every pair of adjacent cells (s,t),
 *           d'_1(s,t) = min d1(s,u) + d(u,v) + d1(v,t) over edges (u,v)
 *           with u in N(s), v in N(t) (Section "Preliminaries"; Algorithm 5).
 *   Step 3  MST G'_2 of G'_1 (sequential; the paper uses Prim, Kruskal here).
 *   Steps 4-7  keep only the bridge edge of every MST pair, add the
 *           predecessor paths from both bridge ends to their seeds
 *           (Algorithm 6), and sum the weights: D(G_S).
 *
 * Readings of points the paper leaves open (each listed in the design
 * notes as well):
 *   - Voronoi ties: a vertex equidistant from several seeds joins the seed
 *     with the smallest vertex id; labels compare as (distance, rank) where
 *     rank = position of the seed in the ascending seed list.
 *   - pred(v): the smallest-id neighbour u with cell(u) = cell(v) and
 *     d1(u) + d(u,v) = d1(v) (a tight edge inside the cell).
 *   - Bridge ties: per cell pair the minimum of (bridge distance, arc id),
 *     where the arc is the CSR arc leaving the endpoint whose cell has the
 *     smaller rank.
 *   - MST ties: Kruskal on the strict order (d'_1, rank a, rank b), so the
 *     MST is unique.
 *   - Distances and bridge sums are exact (64-bit); any reachable distance
 *     or bridge sum >= 2^32 - 1 is reported as ORC_EOVERFLOW.
 *   - Seeds in different components: ORC_EDISCONNECTED, and the output is
 *     the spanning forest.  Unreachable vertices: cell -1, dist 2^32-1,
 *     pred -1.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK            0
#define ORC_EINVAL       -1
#define ORC_ENOMEM       -2
#define ORC_EOVERFLOW    -3
#define ORC_EDISCONNECTED -4

#define DIST_INF 0xFFFFFFFFu
#define NO_VERTEX 0xFFFFFFFFu

/* ------------------------------------------------------------------ */
/* input validation                                                    */
/* ------------------------------------------------------------------ */

/* arc index of (u -> v) in u's sorted row, or -1 */
static int64_t find_arc(const uint32_t *row_ptr, const int32_t *col, uint32_t u, uint32_t v) {
    int64_t lo = row_ptr[u], hi = (int64_t)row_ptr[u + 1] - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if ((uint32_t)col[mid] == v) return mid;
        if ((uint32_t)col[mid] < v) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* The graph must be a simple symmetric graph with weights >= 1
 * (Table "preliminaries_notation": d maps E to positive integers). */
int oracle_check_graph(uint32_t n, const uint32_t *row_ptr, const int32_t *col, const uint32_t *w) {
    if (row_ptr[0] != 0) return ORC_EINVAL;
    for (uint32_t u = 0; u < n; ++u) {
        if (row_ptr[u + 1] < row_ptr[u]) return ORC_EINVAL;
        for (uint32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            if (col[e] < 0 || (uint32_t)col[e] >= n) return ORC_EINVAL;
            if ((uint32_t)col[e] == u) return ORC_EINVAL;
            if (w[e] == 0) return ORC_EINVAL;
            if (e > row_ptr[u] && col[e] <= col[e - 1]) return ORC_EINVAL;
            int64_t back = find_arc(row_ptr, col, (uint32_t)col[e], u);
            if (back < 0 || w[back] != w[e]) return ORC_EINVAL;
        }
    }
    return ORC_OK;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Copies the seeds, sorts them ascending (rank order) and validates them. */
static int sorted_seeds(uint32_t n, uint32_t k, const int32_t *seeds, int32_t **out) {
    if (k == 0) return ORC_EINVAL;
    int32_t *s = (int32_t *)malloc((size_t)k * sizeof(int32_t));
    if (!s) return ORC_ENOMEM;
    memcpy(s, seeds, (size_t)k * sizeof(int32_t));
    qsort(s, k, sizeof(int32_t), cmp_i32);
    for (uint32_t i = 0; i < k; ++i) {
        if (s[i] < 0 || (uint32_t)s[i] >= n || (i > 0 && s[i] == s[i - 1])) {
            free(s);
            return ORC_EINVAL;
        }
    }
    *out = s;
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Step 1: Voronoi cells by multi-source Dijkstra                      */
/* ------------------------------------------------------------------ */

/* A label is the pair (distance, seed rank), compared lexicographically. */
typedef struct { uint64_t dist; uint32_t rank; } label_t;

static int label_less(label_t a, label_t b) {
    return a.dist < b.dist || (a.dist == b.dist && a.rank < b.rank);
}

/* Indexed binary min-heap over vertices, keyed by their current label. */
typedef struct {
    uint32_t *heap;     /* heap[i] = vertex */
    uint32_t *pos;      /* pos[v] = index in heap, or NO_VERTEX */
    uint32_t size;
    const label_t *key;
} heap_t;

static void heap_swap(heap_t *h, uint32_t i, uint32_t j) {
    uint32_t a = h->heap[i], b = h->heap[j];
    h->heap[i] = b; h->heap[j] = a;
    h->pos[b] = i; h->pos[a] = j;
}

static void heap_up(heap_t *h, uint32_t i) {
    while (i > 0) {
        uint32_t p = (i - 1) / 2;
        if (!label_less(h->key[h->heap[i]], h->key[h->heap[p]])) break;
        heap_swap(h, i, p);
        i = p;
    }
}

static void heap_down(heap_t *h, uint32_t i) {
    for (;;) {
        uint32_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < h->size && label_less(h->key[h->heap[l]], h->key[h->heap[m]])) m = l;
        if (r < h->size && label_less(h->key[h->heap[r]], h->key[h->heap[m]])) m = r;
        if (m == i) break;
        heap_swap(h, i, m);
        i = m;
    }
}

static void heap_push_or_decrease(heap_t *h, uint32_t v) {
    if (h->pos[v] == NO_VERTEX) {
        h->heap[h->size] = v;
        h->pos[v] = h->size;
        h->size++;
    }
    heap_up(h, h->pos[v]);
}

static uint32_t heap_pop(heap_t *h) {
    uint32_t v = h->heap[0];
    h->size--;
    if (h->size > 0) {
        h->heap[0] = h->heap[h->size];
        h->pos[h->heap[0]] = 0;
        heap_down(h, 0);
    }
    h->pos[v] = NO_VERTEX;
    return v;
}

/*
 * Voronoi cells (Algorithm 2 Step 1).  Outputs per vertex:
 *   cell[v]   seed vertex id of v's cell, -1 if no seed reaches v
 *   dist[v]   d1(src(v), v), DIST_INF if unreached
 *   pred[v]   predecessor on a shortest path from src(v) (pred(s) = s for a
 *             seed), -1 if unreached
 *   rank_out  optional: rank of cell[v] (NO_VERTEX if unreached)
 * Returns ORC_OK, ORC_EINVAL or ORC_ENOMEM, or ORC_EOVERFLOW if some reached
 * distance does not fit below 2^32 - 1.
 */
static int voronoi_core(uint32_t n, const uint32_t *row_ptr, const int32_t *col, const uint32_t *w,
                        uint32_t k, const int32_t *seeds_sorted,
                        int32_t *cell, uint32_t *dist, int32_t *pred, uint32_t *rank_out) {
    label_t *lab = (label_t *)malloc((size_t)n * sizeof(label_t));
    uint32_t *hp = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    uint32_t *pos = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    if (!lab || !hp || !pos) { free(lab); free(hp); free(pos); return ORC_ENOMEM; }
    for (uint32_t v = 0; v < n; ++v) {
        lab[v].dist = UINT64_MAX; lab[v].rank = NO_VERTEX;
        pos[v] = NO_VERTEX;
    }
    heap_t h = { hp, pos, 0, lab };
    /* INITIALIZATION (Algorithm 3): seeds start at distance 0 in their own cell. */
    for (uint32_t r = 0; r < k; ++r) {
        uint32_t s = (uint32_t)seeds_sorted[r];
        lab[s].dist = 0; lab[s].rank = r;
        heap_push_or_decrease(&h, s);
    }
    while (h.size > 0) {
        uint32_t u = heap_pop(&h);
        for (uint32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            uint32_t v = (uint32_t)col[e];
            label_t cand = { lab[u].dist + w[e], lab[u].rank };
            /* strict improvement of v's (distance, rank) label */
            if (label_less(cand, lab[v])) {
                lab[v] = cand;
                heap_push_or_decrease(&h, v);
            }
        }
    }
    int rc = ORC_OK;
    for (uint32_t v = 0; v < n; ++v) {
        if (lab[v].rank == NO_VERTEX) {
            cell[v] = -1; dist[v] = DIST_INF;
            if (rank_out) rank_out[v] = NO_VERTEX;
        } else {
            if (lab[v].dist >= DIST_INF) rc = ORC_EOVERFLOW;
            cell[v] = seeds_sorted[lab[v].rank];
            dist[v] = lab[v].dist >= DIST_INF ? DIST_INF : (uint32_t)lab[v].dist;
            if (rank_out) rank_out[v] = lab[v].rank;
        }
    }
    /* pred(v): smallest-id neighbour on a tight edge inside v's cell */
    for (uint32_t v = 0; v < n; ++v) {
        pred[v] = -1;
        if (lab[v].rank == NO_VERTEX) continue;
        if (lab[v].dist == 0) { pred[v] = (int32_t)v; continue; }   /* a seed */
        for (uint32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
            uint32_t u = (uint32_t)col[e];
            if (lab[u].rank == lab[v].rank && lab[u].dist + w[e] == lab[v].dist) {
                pred[v] = (int32_t)u;      /* rows are sorted: first hit = smallest id */
                break;
            }
        }
    }
    free(lab); free(hp); free(pos);
    return rc;
}

int oracle_voronoi(uint32_t n, const uint32_t *row_ptr, const int32_t *col, const uint32_t *w,
                   uint32_t k, const int32_t *seeds, int32_t *cell, uint32_t *dist, int32_t *pred) {
    int32_t *ss = NULL;
    int rc = sorted_seeds(n, k, seeds, &ss);
    if (rc) return rc;
    rc = voronoi_core(n, row_ptr, col, w, k, ss, cell, dist, pred, NULL);
    free(ss);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Step 2: the distance graph G'_1 (minimum bridge per cell pair)      */
/* ------------------------------------------------------------------ */

typedef struct {
    uint32_t ra, rb;     /* cell ranks, ra < rb */
    uint64_t b;          /* d1(s,u) + d(u,v) + d1(v,t) */
    uint32_t arc;        /* CSR arc u -> v leaving the cell of rank ra */
} pair_t;

/* Upper-triangle slot of the pair (a, b), a < b < k. */
static uint64_t pair_slot(uint64_t a, uint64_t b, uint64_t k) {
    return a * k - a * (a + 1) / 2 + (b - a - 1);
}

/*
 * For every cross-cell edge {u, v} (taken as the arc leaving the smaller
 * rank), keep the minimum (b, arc) per cell pair.  Writes the pairs in
 * ascending (ra, rb) order into out (capacity cap) and their count.
 */
static int bridges_core(uint32_t n, const uint32_t *row_ptr, const int32_t *col, const uint32_t *w,
                        uint32_t k, const uint32_t *rank, const uint32_t *dist,
                        pair_t **out, uint64_t *count) {
    uint64_t slots = (uint64_t)k * (k - 1) / 2;
    if (slots > (1ull << 28)) return ORC_ENOMEM;          /* oracle keeps a dense table */
    pair_t *tab = (pair_t *)malloc((slots ? slots : 1) * sizeof(pair_t));
    if (!tab) return ORC_ENOMEM;
    for (uint64_t i = 0; i < slots; ++i) { tab[i].b = UINT64_MAX; tab[i].arc = NO_VERTEX; }
    int rc = ORC_OK;
    for (uint32_t u = 0; u < n; ++u) {
        if (rank[u] == NO_VERTEX) continue;
        for (uint32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            uint32_t v = (uint32_t)col[e];
            if (rank[v] == NO_VERTEX || rank[u] >= rank[v]) continue;   /* cross-cell, from smaller rank */
            uint64_t b = (uint64_t)dist[u] + w[e] + dist[v];
            if (b >= DIST_INF) rc = ORC_EOVERFLOW;
            pair_t *p = &tab[pair_slot(rank[u], rank[v], k)];
            if (b < p->b || (b == p->b && e < p->arc)) {
                p->ra = rank[u]; p->rb = rank[v]; p->b = b; p->arc = e;
            }
        }
    }
    uint64_t c = 0;
    for (uint64_t i = 0; i < slots; ++i)
        if (tab[i].arc != NO_VERTEX) tab[c++] = tab[i];
    *out = tab;
    *count = c;
    return rc;
}

/* ------------------------------------------------------------------ */
/* Step 3: Kruskal MST of G'_1 under the order (b, ra, rb)             */
/* ------------------------------------------------------------------ */

static int cmp_pair_weight(const void *x, const void *y) {
    const pair_t *a = (const pair_t *)x, *b = (const pair_t *)y;
    if (a->b != b->b) return a->b < b->b ? -1 : 1;
    if (a->ra != b->ra) return a->ra < b->ra ? -1 : 1;
    if (a->rb != b->rb) return a->rb < b->rb ? -1 : 1;
    return 0;
}

static uint32_t uf_root(uint32_t *p, uint32_t x) {
    while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
    return x;
}

/* Sorts pairs by weight and returns in *n_mst the count of MST pairs,
 * moved to the front of the array. */
static int kruskal_core(uint32_t k, pair_t *pairs, uint64_t count, uint64_t *n_mst) {
    qsort(pairs, count, sizeof(pair_t), cmp_pair_weight);
    uint32_t *p = (uint32_t *)malloc((size_t)k * sizeof(uint32_t));
    if (!p) return ORC_ENOMEM;
    for (uint32_t i = 0; i < k; ++i) p[i] = i;
    uint64_t m = 0;
    for (uint64_t i = 0; i < count; ++i) {
        uint32_t a = uf_root(p, pairs[i].ra), b = uf_root(p, pairs[i].rb);
        if (a == b) continue;
        p[a > b ? a : b] = a > b ? b : a;
        pairs[m++] = pairs[i];
    }
    free(p);
    *n_mst = m;
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Steps 4-7: expansion along predecessors, total distance             */
/* ------------------------------------------------------------------ */

typedef struct { uint32_t u, v, w; } edge_t;

static int cmp_edge(const void *x, const void *y) {
    const edge_t *a = (const edge_t *)x, *b = (const edge_t *)y;
    if (a->u != b->u) return a->u < b->u ? -1 : 1;
    if (a->v != b->v) return a->v < b->v ? -1 : 1;
    return 0;
}

static uint32_t owner_of_arc(const uint32_t *row_ptr, uint32_t n, uint32_t e) {
    uint32_t lo = 0, hi = n;              /* largest u with row_ptr[u] <= e */
    while (hi - lo > 1) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (row_ptr[mid] <= e) lo = mid; else hi = mid;
    }
    return lo;
}

/* weight of edge {a, b}; the edge exists by construction */
static uint32_t edge_weight(const uint32_t *row_ptr, const int32_t *col, const uint32_t *w,
                            uint32_t a, uint32_t b) {
    int64_t e = find_arc(row_ptr, col, a, b);
    return e < 0 ? 0 : w[e];
}

/*
 * The full pipeline.  Output buffers (any may be NULL except the edges):
 *   cell/dist/pred   per-vertex Voronoi state (n entries)
 *   pair_ra/rb/b/arc the distance graph G'_1 in ascending (ra, rb) order
 *                    (capacity pair_cap; *n_pairs receives the full count)
 *   mst_ra/rb/b/arc  the MST pairs in Kruskal order (capacity k)
 *   edge_u/v/w       tree edges, u < v, ascending (capacity n)
 * Returns the status; on ORC_OK or ORC_EDISCONNECTED the outputs are valid.
 */
int oracle_steiner(uint32_t n, const uint32_t *row_ptr, const int32_t *col, const uint32_t *w,
                   uint32_t k, const int32_t *seeds,
                   int32_t *cell, uint32_t *dist, int32_t *pred,
                   uint32_t *pair_ra, uint32_t *pair_rb, uint64_t *pair_b, uint32_t *pair_arc,
                   uint64_t pair_cap, uint64_t *n_pairs,
                   uint32_t *mst_ra, uint32_t *mst_rb, uint64_t *mst_b, uint32_t *mst_arc,
                   uint64_t *n_mst,
                   uint32_t *edge_u, uint32_t *edge_v, uint32_t *edge_w, uint64_t *n_edges,
                   uint64_t *total) {
    int32_t *ss = NULL;
    int rc = sorted_seeds(n, k, seeds, &ss);
    if (rc) return rc;
    int own_cell = 0, own_dist = 0, own_pred = 0;
    if (!cell) { cell = (int32_t *)malloc((size_t)n * 4); own_cell = 1; }
    if (!dist) { dist = (uint32_t *)malloc((size_t)n * 4); own_dist = 1; }
    if (!pred) { pred = (int32_t *)malloc((size_t)n * 4); own_pred = 1; }
    uint32_t *rank = (uint32_t *)malloc((size_t)n * 4);
    uint8_t *in_tree = (uint8_t *)calloc(n, 1);
    edge_t *edges = (edge_t *)malloc(((size_t)n + 1) * sizeof(edge_t));
    pair_t *pairs = NULL;
    uint64_t npairs = 0, nm = 0, ne = 0, tot = 0;
    if (!cell || !dist || !pred || !rank || !in_tree || !edges) { rc = ORC_ENOMEM; goto done; }

    rc = voronoi_core(n, row_ptr, col, w, k, ss, cell, dist, pred, rank);
    if (rc) goto done;
    rc = bridges_core(n, row_ptr, col, w, k, rank, dist, &pairs, &npairs);
    if (rc) goto done;
    if (n_pairs) *n_pairs = npairs;
    if (pair_ra)
        for (uint64_t i = 0; i < npairs && i < pair_cap; ++i) {
            pair_ra[i] = pairs[i].ra; pair_rb[i] = pairs[i].rb;
            pair_b[i] = pairs[i].b; pair_arc[i] = pairs[i].arc;
        }
    rc = kruskal_core(k, pairs, npairs, &nm);
    if (rc) goto done;
    if (n_mst) *n_mst = nm;
    if (mst_ra)
        for (uint64_t i = 0; i < nm; ++i) {
            mst_ra[i] = pairs[i].ra; mst_rb[i] = pairs[i].rb;
            mst_b[i] = pairs[i].b; mst_arc[i] = pairs[i].arc;
        }
    /* Algorithm 6: the bridge of every MST pair joins the tree, then each
     * end walks pred() up to its seed, adding (pred(x), x) once per x. */
    for (uint64_t i = 0; i < nm; ++i) {
        uint32_t e = pairs[i].arc;
        uint32_t u = owner_of_arc(row_ptr, n, e), v = (uint32_t)col[e];
        edge_t be = { u < v ? u : v, u < v ? v : u, w[e] };
        edges[ne++] = be;
        uint32_t ends[2] = { u, v };
        for (int side = 0; side < 2; ++side) {
            uint32_t x = ends[side];
            while ((uint32_t)pred[x] != x && !in_tree[x]) {
                in_tree[x] = 1;
                uint32_t p = (uint32_t)pred[x];
                edge_t pe = { p < x ? p : x, p < x ? x : p, edge_weight(row_ptr, col, w, x, p) };
                edges[ne++] = pe;
                x = p;
            }
        }
    }
    qsort(edges, ne, sizeof(edge_t), cmp_edge);
    for (uint64_t i = 0; i < ne; ++i) {
        edge_u[i] = edges[i].u; edge_v[i] = edges[i].v; edge_w[i] = edges[i].w;
        tot += edges[i].w;
    }
    *n_edges = ne;
    *total = tot;
    if (nm + 1 < k) rc = ORC_EDISCONNECTED;
done:
    if (own_cell) free(cell);
    if (own_dist) free(dist);
    if (own_pred) free(pred);
    free(rank); free(in_tree); free(edges); free(pairs); free(ss);
    return rc;
}
