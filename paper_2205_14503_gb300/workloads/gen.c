/*
 * Seeded synthetic workload generators: R-MAT and 2-D grid graphs as
 * symmetric weighted CSR, plus the largest connected component.
 *
 * This file holds input generation only; none of the Steiner-tree method's
 * arithmetic lives here.  It is shared by the CPU oracle's tests, the CUDA
 * path's tests and the benchmark, so both sides of every parity check see
 * the same bytes.
 *
 * Random numbers come from a counter-based generator: the splitmix64
 * output function (Steele, Lea and Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014) applied to seed + (ctr + 1) * golden.
 * Every draw is addressed by its counter, so the graphs are identical for
 * any thread count and on any host (x86_64 or aarch64).
 *
 * Graph conventions (the paper's datasets, Table "evaluation_datasets":
 * symmetric arcs, positive integer weights): self-loops are dropped,
 * parallel edges are merged keeping the minimum weight, both arcs of an
 * undirected edge carry the same weight, and each adjacency row is sorted
 * by neighbour id.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t sm64(uint64_t seed, uint64_t ctr) {
    uint64_t z = seed + (ctr + 1) * GOLDEN;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* uniform integer in [0, range) from the high 32 bits (multiply-shift) */
static inline uint32_t below32(uint64_t x, uint32_t range) {
    return (uint32_t)(((x >> 32) * (uint64_t)range) >> 32);
}

uint64_t wl_splitmix64(uint64_t seed, uint64_t ctr) { return sm64(seed, ctr); }

/* ------------------------------------------------------------------ */
/* edge sources                                                        */
/* ------------------------------------------------------------------ */

typedef struct {
    int kind;              /* 0 = R-MAT, 1 = grid, 2 = explicit list */
    uint64_t seed;
    uint64_t n_draws;
    uint32_t wmax;
    /* R-MAT */
    int scale;
    double t_a, t_ab, t_abc;   /* cumulative quadrant thresholds */
    int permute;
    uint64_t perm_mul[3], perm_add[3];
    /* grid */
    uint32_t gw, gh;
    /* explicit */
    const uint32_t *eu, *ev, *ew;
} source_t;

static inline uint32_t rmat_permute(const source_t *s, uint32_t x) {
    uint64_t mask = (s->scale >= 32) ? 0xFFFFFFFFull : ((1ull << s->scale) - 1);
    uint64_t y = x;
    int sh = s->scale / 2 + 1;
    for (int r = 0; r < 3; ++r) {
        y = (y * s->perm_mul[r] + s->perm_add[r]) & mask;   /* odd multiplier: bijection mod 2^scale */
        y ^= y >> sh;                                        /* xorshift: bijection on scale bits */
    }
    return (uint32_t)y;
}

/* Draw i of the source; returns 0 when the draw yields no edge (self-loop). */
static inline int draw_edge(const source_t *s, uint64_t i, uint32_t *u, uint32_t *v, uint32_t *w) {
    if (s->kind == 0) {
        uint32_t a = 0, b = 0;
        uint64_t x = 0;
        for (int l = 0; l < s->scale; ++l) {
            if ((l & 1) == 0) x = sm64(s->seed, i * 32 + (uint64_t)(l >> 1));
            uint32_t bits = (l & 1) ? (uint32_t)(x >> 32) : (uint32_t)x;
            double r = (double)bits * (1.0 / 4294967296.0);
            uint32_t bu, bv;
            if (r < s->t_a)        { bu = 0; bv = 0; }
            else if (r < s->t_ab)  { bu = 0; bv = 1; }
            else if (r < s->t_abc) { bu = 1; bv = 0; }
            else                   { bu = 1; bv = 1; }
            a = (a << 1) | bu;
            b = (b << 1) | bv;
        }
        if (s->permute) { a = rmat_permute(s, a); b = rmat_permute(s, b); }
        *u = a; *v = b;
        *w = 1 + below32(sm64(s->seed, i * 32 + 31), s->wmax);
        return a != b;
    } else if (s->kind == 1) {
        uint64_t nh = (uint64_t)s->gh * (s->gw - 1);
        uint32_t a, b;
        if (i < nh) {
            uint64_t r = i / (s->gw - 1), c = i % (s->gw - 1);
            a = (uint32_t)(r * s->gw + c); b = a + 1;
        } else {
            uint64_t j = i - nh;
            uint64_t r = j / s->gw, c = j % s->gw;
            a = (uint32_t)(r * s->gw + c); b = a + s->gw;
        }
        *u = a; *v = b;
        *w = 1 + below32(sm64(s->seed, i), s->wmax);
        return 1;
    } else {
        *u = s->eu[i]; *v = s->ev[i]; *w = s->ew[i];
        return s->eu[i] != s->ev[i];
    }
}

/* ------------------------------------------------------------------ */
/* parallel CSR build                                                  */
/* ------------------------------------------------------------------ */

typedef struct {
    const source_t *src;
    uint64_t lo, hi;          /* draw range */
    uint32_t n;
    uint64_t *deg;            /* pass 1: degree counters; pass 2: cursors */
    uint64_t *arcs;           /* (col << 32) | w, pre-dedup */
    int pass;
    /* row pass */
    const uint64_t *rp;
    uint64_t *cnt;
    uint32_t rlo, rhi;
} job_t;

static void *count_or_scatter(void *p) {
    job_t *j = (job_t *)p;
    for (uint64_t i = j->lo; i < j->hi; ++i) {
        uint32_t u, v, w;
        if (!draw_edge(j->src, i, &u, &v, &w)) continue;
        if (j->pass == 1) {
            __atomic_fetch_add(&j->deg[u], 1, __ATOMIC_RELAXED);
            __atomic_fetch_add(&j->deg[v], 1, __ATOMIC_RELAXED);
        } else {
            uint64_t pu = __atomic_fetch_add(&j->deg[u], 1, __ATOMIC_RELAXED);
            uint64_t pv = __atomic_fetch_add(&j->deg[v], 1, __ATOMIC_RELAXED);
            j->arcs[pu] = ((uint64_t)v << 32) | w;
            j->arcs[pv] = ((uint64_t)u << 32) | w;
        }
    }
    return NULL;
}

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

/* sort each row by (col, w) and count distinct cols */
static void *sort_rows(void *p) {
    job_t *j = (job_t *)p;
    for (uint32_t r = j->rlo; r < j->rhi; ++r) {
        uint64_t s = j->rp[r], e = j->rp[r + 1];
        uint64_t *a = j->arcs + s;
        uint64_t len = e - s;
        if (len > 1) {
            if (len <= 24) {               /* insertion sort for short rows */
                for (uint64_t x = 1; x < len; ++x) {
                    uint64_t key = a[x]; uint64_t y = x;
                    while (y > 0 && a[y - 1] > key) { a[y] = a[y - 1]; --y; }
                    a[y] = key;
                }
            } else {
                qsort(a, len, sizeof(uint64_t), cmp_u64);
            }
        }
        uint64_t c = 0;
        for (uint64_t x = 0; x < len; ++x)
            if (x == 0 || (a[x] >> 32) != (a[x - 1] >> 32)) ++c;
        j->cnt[r] = c;
    }
    return NULL;
}

typedef struct {
    const uint64_t *rp, *arcs;
    const uint64_t *newrp;
    int32_t *col; uint32_t *w;
    uint32_t rlo, rhi;
} emit_t;

static void *emit_rows(void *p) {
    emit_t *j = (emit_t *)p;
    for (uint32_t r = j->rlo; r < j->rhi; ++r) {
        uint64_t s = j->rp[r], e = j->rp[r + 1], o = j->newrp[r];
        for (uint64_t x = s; x < e; ++x) {
            if (x == s || (j->arcs[x] >> 32) != (j->arcs[x - 1] >> 32)) {
                j->col[o] = (int32_t)(j->arcs[x] >> 32);
                j->w[o] = (uint32_t)(j->arcs[x] & 0xFFFFFFFFu);   /* first = min weight */
                ++o;
            }
        }
    }
    return NULL;
}

static int run_jobs(void *(*fn)(void *), void *jobs, size_t job_size, int nt) {
    pthread_t th[256];
    for (int t = 0; t < nt; ++t)
        if (pthread_create(&th[t], NULL, fn, (char *)jobs + t * job_size)) {
            for (int q = 0; q < t; ++q) pthread_join(th[q], NULL);
            return -1;
        }
    for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);
    return 0;
}

/*
 * Phase A: count, scatter, sort and dedup.  Returns an opaque build handle
 * and the final arc count; phase B copies the CSR into caller arrays.
 */
typedef struct {
    uint32_t n;
    uint64_t *rp;       /* pre-dedup row offsets, n + 1 */
    uint64_t *arcs;
    uint64_t *newrp;    /* post-dedup row offsets, n + 1 */
    int nt;
} build_t;

static build_t *build_csr(const source_t *src, uint32_t n, int nt) {
    if (nt < 1) nt = 1;
    if (nt > 256) nt = 256;
    build_t *b = (build_t *)calloc(1, sizeof(build_t));
    if (!b) return NULL;
    b->n = n; b->nt = nt;
    uint64_t *deg = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    job_t *jobs = (job_t *)calloc((size_t)nt, sizeof(job_t));
    if (!deg || !jobs) { free(deg); free(jobs); free(b); return NULL; }
    for (int t = 0; t < nt; ++t) {
        jobs[t].src = src; jobs[t].n = n; jobs[t].deg = deg; jobs[t].pass = 1;
        jobs[t].lo = src->n_draws * (uint64_t)t / (uint64_t)nt;
        jobs[t].hi = src->n_draws * (uint64_t)(t + 1) / (uint64_t)nt;
    }
    run_jobs(count_or_scatter, jobs, sizeof(job_t), nt);
    uint64_t *rp = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    if (!rp) { free(deg); free(jobs); free(b); return NULL; }
    uint64_t acc = 0;
    for (uint32_t v = 0; v < n; ++v) { rp[v] = acc; acc += deg[v]; deg[v] = rp[v]; }
    rp[n] = acc;
    uint64_t *arcs = (uint64_t *)malloc((acc ? acc : 1) * sizeof(uint64_t));
    if (!arcs) { free(rp); free(deg); free(jobs); free(b); return NULL; }
    for (int t = 0; t < nt; ++t) { jobs[t].pass = 2; jobs[t].arcs = arcs; }
    run_jobs(count_or_scatter, jobs, sizeof(job_t), nt);
    free(deg);
    uint64_t *cnt = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    if (!cnt) { free(arcs); free(rp); free(jobs); free(b); return NULL; }
    for (int t = 0; t < nt; ++t) {
        jobs[t].rp = rp; jobs[t].cnt = cnt; jobs[t].arcs = arcs;
        jobs[t].rlo = (uint32_t)((uint64_t)n * t / nt);
        jobs[t].rhi = (uint32_t)((uint64_t)n * (t + 1) / nt);
    }
    run_jobs(sort_rows, jobs, sizeof(job_t), nt);
    free(jobs);
    acc = 0;
    for (uint32_t v = 0; v < n; ++v) { uint64_t c = cnt[v]; cnt[v] = acc; acc += c; }
    cnt[n] = acc;
    b->rp = rp; b->arcs = arcs; b->newrp = cnt;
    return b;
}

/* Returns the handle; *n_arcs receives the deduplicated arc count. */
static void *finish_source(source_t *src, uint32_t n, int nt, uint64_t *n_arcs) {
    source_t *keep = (source_t *)malloc(sizeof(source_t));
    if (!keep) return NULL;
    *keep = *src;
    build_t *b = build_csr(keep, n, nt);
    free(keep);
    if (!b) return NULL;
    *n_arcs = b->newrp[n];
    return b;
}

void *wl_rmat_begin(int scale, uint64_t edge_factor, double a, double b, double c,
                    uint32_t wmax, uint64_t seed, int permute, int nthreads, uint64_t *n_arcs) {
    if (scale < 1 || scale > 31 || wmax < 1) return NULL;
    source_t s; memset(&s, 0, sizeof s);
    s.kind = 0; s.seed = seed; s.scale = scale; s.wmax = wmax;
    s.n_draws = edge_factor << scale;
    s.t_a = a; s.t_ab = a + b; s.t_abc = a + b + c;
    s.permute = permute;
    for (int r = 0; r < 3; ++r) {
        s.perm_mul[r] = sm64(seed ^ 0xA5A5A5A5ull, 2 * (uint64_t)r) | 1ull;
        s.perm_add[r] = sm64(seed ^ 0xA5A5A5A5ull, 2 * (uint64_t)r + 1);
    }
    return finish_source(&s, (uint32_t)(1ull << scale), nthreads, n_arcs);
}

void *wl_grid_begin(uint32_t width, uint32_t height, uint32_t wmax, uint64_t seed,
                    int nthreads, uint64_t *n_arcs) {
    if (width < 1 || height < 1 || wmax < 1) return NULL;
    if ((uint64_t)width * height > 0xFFFFFFFFull) return NULL;
    source_t s; memset(&s, 0, sizeof s);
    s.kind = 1; s.seed = seed; s.wmax = wmax; s.gw = width; s.gh = height;
    s.n_draws = (uint64_t)height * (width - 1) + (uint64_t)(height - 1) * width;
    return finish_source(&s, width * height, nthreads, n_arcs);
}

void *wl_edges_begin(uint32_t n, uint64_t m, const uint32_t *u, const uint32_t *v,
                     const uint32_t *w, int nthreads, uint64_t *n_arcs) {
    for (uint64_t i = 0; i < m; ++i)
        if (u[i] >= n || v[i] >= n) return NULL;
    source_t s; memset(&s, 0, sizeof s);
    s.kind = 2; s.n_draws = m; s.eu = u; s.ev = v; s.ew = w;
    return finish_source(&s, n, nthreads, n_arcs);
}

/* Phase B: copy into caller arrays (row_ptr has n + 1 entries) and free. */
int wl_finish(void *handle, uint32_t *row_ptr, int32_t *col, uint32_t *w) {
    build_t *b = (build_t *)handle;
    uint32_t n = b->n;
    int rc = 0;
    if (b->newrp[n] > 0xFFFFFFFFull) rc = -1;   /* row offsets must fit 32 bits */
    if (rc == 0) {
        for (uint32_t v = 0; v <= n; ++v) row_ptr[v] = (uint32_t)b->newrp[v];
        int nt = b->nt;
        emit_t *jobs = (emit_t *)calloc((size_t)nt, sizeof(emit_t));
        if (!jobs) rc = -2;
        else {
            for (int t = 0; t < nt; ++t) {
                jobs[t].rp = b->rp; jobs[t].arcs = b->arcs; jobs[t].newrp = b->newrp;
                jobs[t].col = col; jobs[t].w = w;
                jobs[t].rlo = (uint32_t)((uint64_t)n * t / nt);
                jobs[t].rhi = (uint32_t)((uint64_t)n * (t + 1) / nt);
            }
            run_jobs(emit_rows, jobs, sizeof(emit_t), nt);
            free(jobs);
        }
    }
    free(b->rp); free(b->arcs); free(b->newrp); free(b);
    return rc;
}

void wl_abort(void *handle) {
    build_t *b = (build_t *)handle;
    if (!b) return;
    free(b->rp); free(b->arcs); free(b->newrp); free(b);
}

/* ------------------------------------------------------------------ */
/* connected components (concurrent union-find, parents point to       */
/* smaller ids, so path halving never breaks an ancestor chain)        */
/* ------------------------------------------------------------------ */

static inline uint32_t uf_find(uint32_t *p, uint32_t x) {
    for (;;) {
        uint32_t px = __atomic_load_n(&p[x], __ATOMIC_RELAXED);
        if (px == x) return x;
        uint32_t ppx = __atomic_load_n(&p[px], __ATOMIC_RELAXED);
        if (ppx != px) __atomic_store_n(&p[x], ppx, __ATOMIC_RELAXED);
        x = ppx;
    }
}

typedef struct {
    const uint32_t *row_ptr; const int32_t *col; uint32_t *parent;
    uint32_t lo, hi;
} cc_job_t;

static void *cc_unite(void *pp) {
    cc_job_t *j = (cc_job_t *)pp;
    for (uint32_t u = j->lo; u < j->hi; ++u) {
        for (uint32_t e = j->row_ptr[u]; e < j->row_ptr[u + 1]; ++e) {
            uint32_t v = (uint32_t)j->col[e];
            if (v <= u) continue;
            for (;;) {
                uint32_t ru = uf_find(j->parent, u), rv = uf_find(j->parent, v);
                if (ru == rv) break;
                uint32_t hi = ru > rv ? ru : rv, lo = ru > rv ? rv : ru;
                uint32_t expect = hi;
                if (__atomic_compare_exchange_n(&j->parent[hi], &expect, lo, 0,
                                                __ATOMIC_RELAXED, __ATOMIC_RELAXED))
                    break;
            }
        }
    }
    return NULL;
}

static void *cc_flatten(void *pp) {
    cc_job_t *j = (cc_job_t *)pp;
    for (uint32_t u = j->lo; u < j->hi; ++u) j->parent[u] = uf_find(j->parent, u);
    return NULL;
}

/*
 * comp[v] receives the smallest vertex id of v's component.  Returns the
 * representative of the largest component (ties: smallest representative)
 * and its size in *size.
 */
int64_t wl_components(uint32_t n, const uint32_t *row_ptr, const int32_t *col,
                      uint32_t *comp, int nthreads, uint64_t *size) {
    if (n == 0) { *size = 0; return -1; }
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    for (uint32_t v = 0; v < n; ++v) comp[v] = v;
    cc_job_t jobs[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].row_ptr = row_ptr; jobs[t].col = col; jobs[t].parent = comp;
        jobs[t].lo = (uint32_t)((uint64_t)n * t / nthreads);
        jobs[t].hi = (uint32_t)((uint64_t)n * (t + 1) / nthreads);
    }
    run_jobs(cc_unite, jobs, sizeof(cc_job_t), nthreads);
    run_jobs(cc_flatten, jobs, sizeof(cc_job_t), nthreads);
    uint64_t *cnt = (uint64_t *)calloc(n, sizeof(uint64_t));
    if (!cnt) return -2;
    for (uint32_t v = 0; v < n; ++v) cnt[comp[v]]++;
    uint64_t best = 0; int64_t rep = 0;
    for (uint32_t v = 0; v < n; ++v)
        if (cnt[v] > best) { best = cnt[v]; rep = v; }
    free(cnt);
    *size = best;
    return rep;
}

/*
 * Unweighted BFS levels from `root` (hop counts; UINT32_MAX where
 * unreachable), for the seed-selection workload variants.  Returns the
 * deepest level.
 */
int64_t wl_bfs_levels(uint32_t n, const uint32_t *row_ptr, const int32_t *col, uint32_t root,
                      uint32_t *level) {
    if (root >= n) return -1;
    uint32_t *queue = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    if (!queue) return -2;
    for (uint32_t v = 0; v < n; ++v) level[v] = UINT32_MAX;
    uint64_t head = 0, tail = 0;
    level[root] = 0;
    queue[tail++] = root;
    uint32_t deepest = 0;
    while (head < tail) {
        uint32_t u = queue[head++];
        uint32_t lu = level[u];
        if (lu > deepest) deepest = lu;
        for (uint32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            uint32_t v = (uint32_t)col[e];
            if (level[v] == UINT32_MAX) {
                level[v] = lu + 1;
                queue[tail++] = v;
            }
        }
    }
    free(queue);
    return deepest;
}
