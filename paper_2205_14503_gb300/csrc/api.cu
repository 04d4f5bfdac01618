// C ABI of the library (declared in include/steiner.h): graph upload,
// per-query device workspace, the single-query driver (Algorithm 2 end to
// end on one stream), the Voronoi export, and the batch/serving entries.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/steiner.h"
#include "internal.h"
#include "engine.h"

using namespace stn;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *where) {
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return STEINER_ECUDA;
}

#define CK(call)                                                     \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);          \
    } while (0)

template <class T>
cudaError_t dalloc(T *&p, uint64_t count) {
    if (p) cudaFree(p);
    p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void **)&p, count * sizeof(T));
}

uint32_t bit_length(uint32_t x) { return x ? 32u - (uint32_t)__builtin_clz(x) : 0u; }

uint32_t bits_for(uint32_t n) {
    uint32_t b = 1;
    while (b < 32 && (1ull << b) < (uint64_t)n) ++b;
    return b;
}

}  // namespace

struct steiner_graph {
    int device = 0;
    DevGraph g;
    Geometry geo;
    cudaStream_t stream = nullptr;
    std::mutex mu;
    Workspace ws;
    bool ws_ready = false;
    uint32_t nbits = 1;
    uint32_t delta = 0;
    uint32_t max_iters = 1u << 22;
    uint32_t local_rounds = 0;
    // Label width of the Voronoi phase: 0 chooses per query (32 bits when
    // the distance field leaves room for 256 largest weights and no query
    // with as few distance bits has overflowed it before), 32 or 64 force it.
    uint32_t label_bits = 0;
    // Band splits: -1 chooses (a scan of the labels while the light/heavy
    // split is on, else the far pile), 0 / 1 force the pile / the scan.
    int far_scan = -1;
    // Dense frontiers (bitmaps for large frontiers and band lists) wherever
    // the far scan runs without local rounds; 0 turns them off.
    uint32_t dense = 1;
    // Heavy-arc passes of the light/heavy split (with the far scan): 1
    // runs each in the push or the pull form, whichever reads fewer arcs;
    // 0 always pushes, 2 always pulls.
    uint32_t pull = 1;
    uint32_t last_pulls = 0;
    // After a heavy-arc pass in the pull form, the rest of the Voronoi phase
    // runs as one unbounded band (1, default) or keeps its bands (0).
    uint32_t tail = 1;
    uint32_t last_tail_it = 0;
    uint32_t narrow_fail_dbits = 0;   // most distance bits a narrow attempt ran out of
    uint32_t last_label_bits = 0;
    uint64_t narrow_reruns = 0;
    Control *h_ctl = nullptr;      // pinned
    cudaEvent_t ev[6] = {};
    BatchEngine *batch = nullptr;
    ServeEngine *serve = nullptr;
};

namespace {

int ensure_n_workspace(steiner_graph *G) {
    Workspace &ws = G->ws;
    if (G->ws_ready) return STEINER_OK;
    uint32_t n = G->g.n;
    ws.n = n;
    CK(dalloc(ws.label, n));
    CK(dalloc(ws.label32, n));
    CK(dalloc(ws.pred_arc, n));
    CK(dalloc(ws.stamp_near, n));
    CK(dalloc(ws.stamp_far, n));
    CK(dalloc(ws.stamp_band, n));
    CK(dalloc(ws.band_q, n));
    CK(dalloc(ws.band_hq, G->g.heavy_chunk_cap));
    CK(dalloc(ws.mark, n));
    const uint64_t words = ((uint64_t)n + 31) / 32;
    CK(dalloc(ws.nbm[0], words));
    CK(dalloc(ws.nbm[1], words));
    CK(dalloc(ws.bbm, words));
    CK(cudaMemsetAsync(ws.nbm[0], 0, words * 4, G->stream));
    CK(cudaMemsetAsync(ws.nbm[1], 0, words * 4, G->stream));
    CK(cudaMemsetAsync(ws.bbm, 0, words * 4, G->stream));
    CK(dalloc(ws.q[0], n));
    CK(dalloc(ws.q[1], n));
    CK(dalloc(ws.hq[0], G->g.heavy_chunk_cap));
    CK(dalloc(ws.hq[1], G->g.heavy_chunk_cap));
    CK(dalloc(ws.far[0], n));
    CK(dalloc(ws.far[1], n));
    CK(dalloc(ws.ctl, 1));
    uint64_t tcap = std::max<uint64_t>(n, 2);
    CK(dalloc(ws.tree_key, tcap));
    CK(dalloc(ws.tree_key2, tcap));
    CK(dalloc(ws.tree_w, tcap));
    CK(dalloc(ws.tree_w2, tcap));
    ws.tree_cap = (uint32_t)tcap;
    CK(cudaMemsetAsync(ws.stamp_near, 0, (size_t)n * 4, G->stream));
    CK(cudaMemsetAsync(ws.stamp_far, 0, (size_t)n * 4, G->stream));
    CK(cudaMemsetAsync(ws.stamp_band, 0, (size_t)n * 4, G->stream));
    CK(cudaMemsetAsync(ws.mark, 0, (size_t)n * 4, G->stream));
    ws.epoch_near = ws.epoch_far = ws.epoch_mark = ws.epoch_band = 1;
    G->ws_ready = true;
    return STEINER_OK;
}

int ensure_k_workspace(steiner_graph *G, uint32_t k, bool with_pairtab = true) {
    Workspace &ws = G->ws;
    if (k > ws.seeds_cap) {
        CK(dalloc(ws.seeds, k));
        ws.seeds_cap = k;
    }
    uint64_t slots = k > 1 ? (uint64_t)k * (k - 1) / 2 : 0;
    if (slots > (1ull << 28))
        return fail(STEINER_ENOMEM, "seed set too large for the pair table (k(k-1)/2 > 2^28)");
    if (with_pairtab && slots > ws.pairtab_cap) {
        CK(dalloc(ws.pairtab, slots));
        ws.pairtab_cap = slots;
    }
    uint64_t ecap = std::min<uint64_t>(slots, G->g.m / 2 + 1);
    if (ecap > ws.e_cap) {
        CK(dalloc(ws.e_key, ecap));
        CK(dalloc(ws.e_ra, ecap));
        CK(dalloc(ws.e_rb, ecap));
        CK(dalloc(ws.e_arc, ecap));
        CK(dalloc(ws.e_mst, ecap));
        ws.e_cap = ecap;
    }
    uint64_t tiles = std::max<uint64_t>((slots + 2047) / 2048, 64 * 256);
    if (tiles > ws.tile_cap) {
        CK(dalloc(ws.tile_off, tiles));
        ws.tile_cap = (uint32_t)tiles;
    }
    if (k > ws.comp_cap) {
        CK(dalloc(ws.comp, k));
        CK(dalloc(ws.hook, k));
        CK(dalloc(ws.best, k));
        ws.comp_cap = k;
    }
    return STEINER_OK;
}

int sorted_seed_list(const steiner_graph *G, const int32_t *seeds, uint32_t k,
                     std::vector<int32_t> &out) {
    if (k == 0) return fail(STEINER_EINVAL, "empty seed set");
    if (!seeds) return fail(STEINER_EINVAL, "null seed pointer");
    out.assign(seeds, seeds + k);
    std::sort(out.begin(), out.end());
    for (uint32_t i = 0; i < k; ++i) {
        if (out[i] < 0 || (uint32_t)out[i] >= G->g.n)
            return fail(STEINER_EINVAL, "seed id out of range");
        if (i && out[i] == out[i - 1]) return fail(STEINER_EINVAL, "duplicate seed id");
    }
    return STEINER_OK;
}

int status_from(const Control &c, uint32_t k, bool tree) {
    if (c.err & (ERR_BARRIER | ERR_TIMEOUT))
        return fail(STEINER_ETIMEOUT, "device loop or barrier hit its cap");
    if (c.err & ERR_OVERFLOW)
        return fail(STEINER_EOVERFLOW, "a distance or bridge sum reached 2^32 - 1");
    if (c.err & ERR_CAPACITY) return fail(STEINER_ENOMEM, "internal buffer capacity exceeded");
    if (tree && k > 1 && c.n_mst + 1 < k)
        return fail(STEINER_EDISCONNECTED, "seeds lie in more than one component");
    return STEINER_OK;
}

void advance_epochs(Workspace &ws, const Control &c, cudaStream_t s) {
    ws.epoch_near += c.iterations + 2;
    ws.epoch_far += c.phases + 2;
    ws.epoch_mark += 1;
    ws.epoch_band += c.bands + 2;
    if (c.err != 0 || ws.epoch_near > 0x7FFFFFFFu || ws.epoch_far > 0x7FFFFFFFu ||
        ws.epoch_mark > 0x7FFFFFFFu || ws.epoch_band > 0x7FFFFFFFu) {
        cudaMemsetAsync(ws.stamp_near, 0, (size_t)ws.n * 4, s);
        cudaMemsetAsync(ws.stamp_far, 0, (size_t)ws.n * 4, s);
        cudaMemsetAsync(ws.stamp_band, 0, (size_t)ws.n * 4, s);
        cudaMemsetAsync(ws.mark, 0, (size_t)ws.n * 4, s);
        // a run that stopped early may leave frontier bits set
        const size_t words = ((size_t)ws.n + 31) / 32;
        cudaMemsetAsync(ws.nbm[0], 0, words * 4, s);
        cudaMemsetAsync(ws.nbm[1], 0, words * 4, s);
        cudaMemsetAsync(ws.bbm, 0, words * 4, s);
        ws.epoch_near = ws.epoch_far = ws.epoch_mark = ws.epoch_band = 1;
    }
}

// Partition failures are not fatal: the kernels then filter arcs by weight
// on the id-sorted rows.
cudaError_t ensure_partition(steiner_graph *G, uint32_t delta) {
    if (ensure_partition_dev(G->g, delta, G->stream) != cudaSuccess) G->g.part_delta = 0;
    return cudaSuccess;
}

// Runs Steps 1 (and, with `full`, 2-7) of Algorithm 2 for one sorted seed
// list with the label width in G->ws.narrow.  Leaves the control block in
// G->h_ctl.
int run_pipeline_once(steiner_graph *G, const std::vector<int32_t> &ss, bool full, float *ms) {
    uint32_t k = (uint32_t)ss.size();
    int rc = ensure_n_workspace(G);
    if (rc) return rc;
    rc = ensure_k_workspace(G, k);
    if (rc) return rc;
    Workspace &ws = G->ws;
    cudaStream_t s = G->stream;
    CK(cudaMemcpyAsync(ws.seeds, ss.data(), (size_t)k * 4, cudaMemcpyHostToDevice, s));
    // far scan: by default wherever the light/heavy split is on (a band's
    // heavy-arc pass sends every proposal far, and the pile would cost a
    // stamp exchange and a queue slot per improvement)
    const bool split_on = G->delta <= G->g.max_w;
    const uint32_t far_scan = G->far_scan < 0 ? (split_on ? 1u : 0u) : (uint32_t)G->far_scan;
    static const bool trace = getenv("STEINER_TRACE") != nullptr;
    const uint32_t dense = (G->dense && far_scan && G->local_rounds == 0) ? 1u : 0u;
    SsspParams p{G->delta, G->max_iters, ws.epoch_near, ws.epoch_far, G->local_rounds,
                 ws.epoch_band, far_scan, trace ? 1u : 0u, dense, far_scan ? G->pull : 0u,
                 G->tail};
    CK(cudaEventRecord(G->ev[0], s));
    CK(ensure_partition(G, G->delta));
    CK(launch_init(G->g, ws, k, G->delta, s));
    CK(cudaEventRecord(G->ev[1], s));
    CK(launch_sssp(G->g, ws, G->geo, p, s));
    CK(cudaEventRecord(G->ev[2], s));
    CK(launch_scan(G->g, ws, k, full, s));
    uint32_t launches = 4;      // init labels, init seeds, SSSP, scan
    if (full) {
        CK(launch_compact_pairs(ws, k, s));
        CK(cudaEventRecord(G->ev[3], s));
        CK(launch_mst(ws, k, G->geo, s));
        CK(cudaEventRecord(G->ev[4], s));
        CK(launch_tree(G->g, ws, k, ws.epoch_mark, G->nbits, s));
        if (k > 1) launches += 3 + 1 + 2;   // compaction, MST, expansion + sort
    } else {
        CK(cudaEventRecord(G->ev[3], s));
        CK(cudaEventRecord(G->ev[4], s));
    }
    CK(cudaEventRecord(G->ev[5], s));
    CK(cudaMemcpyAsync(G->h_ctl, ws.ctl, sizeof(Control), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (ms) {
        for (int i = 0; i < 5; ++i) cudaEventElapsedTime(&ms[i], G->ev[i], G->ev[i + 1]);
        ms[5] = (float)launches;
    }
    advance_epochs(ws, *G->h_ctl, s);
    G->last_pulls = G->h_ctl->pulls;
    G->last_tail_it = G->h_ctl->tail_it;
    return STEINER_OK;
}

// As run_pipeline_once, choosing the label width: 32-bit labels hold
// (dist << rank bits) | rank; if a distance did not fit (ERR_NARROW) the
// query runs again with 64-bit labels, so the result never depends on the
// width.  ms[] (if given) sums both attempts.
int run_pipeline(steiner_graph *G, const std::vector<int32_t> &ss, bool full, float *ms) {
    const uint32_t k = (uint32_t)ss.size();
    const uint32_t rbits = bits_for(k);
    const uint32_t dbits = 32 - rbits;
    bool narrow;
    if (G->label_bits == 64) narrow = false;
    else if (G->label_bits == 32) narrow = true;
    else narrow = dbits >= bit_length(G->g.max_w) + 8 && dbits > G->narrow_fail_dbits;
    G->ws.narrow = narrow;
    G->ws.lshift = rbits;
    int rc = run_pipeline_once(G, ss, full, ms);
    G->last_label_bits = narrow ? 32 : 64;
    if (rc || !narrow || !(G->h_ctl->err & ERR_NARROW)) return rc;
    ++G->narrow_reruns;
    G->narrow_fail_dbits = std::max(G->narrow_fail_dbits, dbits);
    G->ws.narrow = false;
    G->last_label_bits = 64;
    float ms2[6] = {0, 0, 0, 0, 0, 0};
    rc = run_pipeline_once(G, ss, full, ms ? ms2 : nullptr);
    if (ms)
        for (int i = 0; i < 6; ++i) ms[i] += ms2[i];
    return rc;
}

int fetch_tree(steiner_graph *G, steiner_result_t *out) {
    const Control &c = *G->h_ctl;
    uint32_t nt = std::min(c.n_tree, G->ws.tree_cap);
    std::vector<uint64_t> keys(nt);
    std::vector<uint32_t> ws(nt);
    if (nt) {
        CK(cudaMemcpyAsync(keys.data(), G->ws.tree_key, (size_t)nt * 8, cudaMemcpyDeviceToHost,
                           G->stream));
        CK(cudaMemcpyAsync(ws.data(), G->ws.tree_w, (size_t)nt * 4, cudaMemcpyDeviceToHost,
                           G->stream));
        CK(cudaStreamSynchronize(G->stream));
    }
    out->edges = nt ? (steiner_edge_t *)malloc((size_t)nt * sizeof(steiner_edge_t)) : nullptr;
    if (nt && !out->edges) return fail(STEINER_ENOMEM, "host allocation of the result failed");
    uint64_t mask = (1ull << G->nbits) - 1;
    for (uint32_t i = 0; i < nt; ++i) {
        out->edges[i].u = (uint32_t)(keys[i] >> G->nbits);
        out->edges[i].v = (uint32_t)(keys[i] & mask);
        out->edges[i].w = ws[i];
    }
    out->n_edges = nt;
    out->total = c.total;
    return STEINER_OK;
}

int query_locked(steiner_graph *G, const int32_t *seeds, uint32_t k, steiner_result_t *out,
                 steiner_pair_t **pairs, uint64_t *n_pairs, steiner_stats_t *stats) {
    out->edges = nullptr;
    out->n_edges = 0;
    out->total = 0;
    std::vector<int32_t> ss;
    int rc = sorted_seed_list(G, seeds, k, ss);
    if (rc) return out->status = rc;
    float ms[6] = {0, 0, 0, 0, 0, 0};
    rc = run_pipeline(G, ss, true, ms);
    if (rc) return out->status = rc;
    const Control c = *G->h_ctl;
    rc = status_from(c, k, true);
    if (getenv("STEINER_TRACE")) {
        fprintf(stderr, "[steiner] err=0x%x exit=%u iterations=%u phases=%u attempts=%llu\n",
                c.err, c.exit_reason, c.iterations, c.phases, c.relax_attempts);
        const int nt = std::min<int>(TRACE_LEN, (int)c.iterations);
        for (int i = 0; i < nt; ++i) {
            // a far-pile split takes an iteration index of its own and is
            // not traced; its time counts with the iteration before it
            if (!c.trace_ns[i]) {
                fprintf(stderr, "[steiner]   it %d: far-pile split\n", i);
                continue;
            }
            unsigned long long t1 = (int)c.iterations <= TRACE_LEN ? c.end_ns : 0;
            for (int j = i + 1; j < nt; ++j)
                if (c.trace_ns[j]) {
                    t1 = c.trace_ns[j];
                    break;
                }
            double us = t1 > c.trace_ns[i] ? 1e-3 * (double)(t1 - c.trace_ns[i]) : -1.0;
            const double nw = (double)(G->geo.sssp_blocks * (G->geo.threads / 32));
            fprintf(stderr, "[steiner]   it %d: near %u heavy %u far %u T %u  %.1f us  relax %llu "
                    "improved %llu atomics %llu  warp busy mean %.1f max %.1f us\n",
                    i, c.trace[i][0], c.trace[i][1], c.trace[i][2], c.trace[i][3], us,
                    c.trace_relax[i][0], c.trace_relax[i][1], c.trace_relax[i][2],
                    1e-3 * (double)c.trace_busy[i][0] / nw, 1e-3 * (double)c.trace_busy[i][1]);
        }
    }
    if (rc == STEINER_OK || rc == STEINER_EDISCONNECTED) {
        int rc2 = fetch_tree(G, out);
        if (rc2) return out->status = rc2;
    }
    if (pairs && (rc == STEINER_OK || rc == STEINER_EDISCONNECTED)) {
        uint32_t np = k > 1 ? c.n_pairs : 0;
        std::vector<uint64_t> key(np);
        std::vector<uint32_t> ra(np), rb(np), arc(np), mst(np);
        if (np) {
            cudaStream_t s = G->stream;
            CK(cudaMemcpyAsync(key.data(), G->ws.e_key, (size_t)np * 8, cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(ra.data(), G->ws.e_ra, (size_t)np * 4, cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(rb.data(), G->ws.e_rb, (size_t)np * 4, cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(arc.data(), G->ws.e_arc, (size_t)np * 4, cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(mst.data(), G->ws.e_mst, (size_t)np * 4, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
        }
        steiner_pair_t *p = (steiner_pair_t *)malloc(std::max<size_t>(np, 1) * sizeof(steiner_pair_t));
        if (!p) return out->status = fail(STEINER_ENOMEM, "host allocation failed");
        for (uint32_t i = 0; i < np; ++i) {
            p[i].ra = ra[i];
            p[i].rb = rb[i];
            p[i].b = key[i] >> 32;
            p[i].arc = arc[i];
            p[i].in_mst = mst[i];
        }
        *pairs = p;
        if (n_pairs) *n_pairs = np;
    }
    if (stats) {
        stats->relax_attempts = c.relax_attempts;
        stats->relax_improved = c.relax_improved;
        stats->iterations = c.iterations;
        stats->phases = c.phases;
        stats->n_pairs = k > 1 ? c.n_pairs : 0;
        stats->n_tree_edges = c.n_tree;
        stats->gpu_launches = (uint32_t)ms[5];
        stats->ms_init = ms[0];
        stats->ms_voronoi = ms[1];
        stats->ms_bridges = ms[2];
        stats->ms_mst = ms[3];
        stats->ms_tree = ms[4];
    }
    return out->status = rc;
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

// ---------------------------------------------------------------------------
// exported entry points
// ---------------------------------------------------------------------------

extern "C" {

const char *steiner_last_error(void) { return g_last_error.c_str(); }

const char *steiner_version(void) { return "gb300-steiner 0.1 (sm_103a)"; }

int steiner_load_graph(const uint32_t *row_ptr, const int32_t *col, const uint32_t *w, uint32_t n,
                       uint64_t n_arcs, int device, steiner_graph_t *out) {
    if (!out) return fail(STEINER_EINVAL, "null output handle");
    *out = nullptr;
    if (!row_ptr || (n_arcs && (!col || !w))) return fail(STEINER_EINVAL, "null graph array");
    if (n == 0) return fail(STEINER_EINVAL, "graph has no vertices");
    if (n_arcs >= 0xFFFFFFFFull) return fail(STEINER_EINVAL, "arc count must be below 2^32");
    if (row_ptr[0] != 0 || row_ptr[n] != n_arcs)
        return fail(STEINER_EINVAL, "row_ptr[0] must be 0 and row_ptr[n] the arc count");
    for (uint32_t v = 0; v < n; ++v)
        if (row_ptr[v + 1] < row_ptr[v]) return fail(STEINER_EINVAL, "row_ptr not monotone");
    CK(cudaSetDevice(device));
    steiner_graph *G = new steiner_graph();
    G->device = device;
    G->g.n = n;
    G->g.m = n_arcs;
    G->nbits = bits_for(n);
    auto bail = [&](int rc) {
        steiner_free_graph(G);
        return rc;
    };
    cudaError_t e = cudaStreamCreateWithFlags(&G->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaStreamCreate"));
    for (auto &ev : G->ev)
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) return bail(cuda_fail(e, "cudaEventCreate"));
    if ((e = cudaMallocHost((void **)&G->h_ctl, sizeof(Control))) != cudaSuccess)
        return bail(cuda_fail(e, "cudaMallocHost"));
    // Internal vertex order: on a skewed degree distribution, descending
    // degree (ties by caller id), so the hubs' labels, which most arcs
    // point to, share L2 sectors.  STEINER_RELABEL=0/1 forces it off/on.
    uint32_t max_deg = 0;
    for (uint32_t v = 0; v < n; ++v) max_deg = std::max(max_deg, row_ptr[v + 1] - row_ptr[v]);
    const double avg_deg = n_arcs ? (double)n_arcs / n : 0.0;
    bool relabel = n_arcs > 0 && n >= 1024 && max_deg >= 16.0 * std::max(1.0, avg_deg);
    if (const char *env = getenv("STEINER_RELABEL")) relabel = n_arcs > 0 && atoi(env) != 0;
    std::vector<uint32_t> h_orig_of, h_new_of, h_new_rp;
    if (relabel) {
        std::vector<uint64_t> start((size_t)max_deg + 1, 0);
        for (uint32_t v = 0; v < n; ++v) ++start[row_ptr[v + 1] - row_ptr[v]];
        uint64_t pos = 0;
        for (int64_t d = max_deg; d >= 0; --d) {
            uint64_t c = start[d];
            start[d] = pos;
            pos += c;
        }
        h_orig_of.resize(n);
        h_new_of.resize(n);
        for (uint32_t v = 0; v < n; ++v) {
            uint32_t u = (uint32_t)start[row_ptr[v + 1] - row_ptr[v]]++;
            h_orig_of[u] = v;
            h_new_of[v] = u;
        }
        h_new_rp.resize((size_t)n + 1);
        h_new_rp[0] = 0;
        for (uint32_t u = 0; u < n; ++u)
            h_new_rp[u + 1] = h_new_rp[u] + (row_ptr[h_orig_of[u] + 1] - row_ptr[h_orig_of[u]]);
    }
    const uint32_t *irp = relabel ? h_new_rp.data() : row_ptr;     // internal row offsets
    // heavy rows, listed in CHUNK-arc pieces (internal ids)
    std::vector<uint64_t> chunks;
    uint64_t cap = 0;
    for (uint32_t v = 0; v < n; ++v) {
        uint32_t deg = irp[v + 1] - irp[v];
        if (deg >= HEAVY_DEG) {
            uint32_t nc = (deg + CHUNK - 1) / CHUNK;
            for (uint32_t c = 0; c < nc; ++c) chunks.push_back(((uint64_t)v << 32) | c);
            cap += nc;
        }
    }
    G->g.n_heavy_chunks = (uint32_t)chunks.size();
    // ids at or above n_big have fewer than HEAVY_DEG arcs: with the degree
    // order the hubs come first; without it no id is known to be light
    G->g.n_big = max_deg < HEAVY_DEG ? 0 : n;
    if (relabel && max_deg >= HEAVY_DEG) {
        uint32_t nb = 0;
        while (nb < n && irp[nb + 1] - irp[nb] >= HEAVY_DEG) ++nb;
        G->g.n_big = nb;
    }
    G->g.heavy_chunk_cap = (uint32_t)std::max<uint64_t>(cap, 1);
    if ((e = dalloc(G->g.row_ptr, (uint64_t)n + 1)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc"));
    if ((e = dalloc(G->g.adj, n_arcs)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc"));
    if ((e = dalloc(G->g.heavy_chunks, chunks.size())) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc"));
    if (relabel) {
        if ((e = dalloc(G->g.orig_row_ptr, (uint64_t)n + 1)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc"));
        if ((e = dalloc(G->g.orig_of, n)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc"));
        if ((e = dalloc(G->g.new_of, n)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc"));
    }
    int32_t *d_col = nullptr;
    uint32_t *d_w = nullptr, *d_bad = nullptr;
    if ((e = dalloc(d_col, n_arcs)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc"));
    if ((e = dalloc(d_w, n_arcs)) != cudaSuccess) {
        cudaFree(d_col);
        return bail(cuda_fail(e, "cudaMalloc"));
    }
    if ((e = dalloc(d_bad, 2)) != cudaSuccess) {
        cudaFree(d_col);
        cudaFree(d_w);
        return bail(cuda_fail(e, "cudaMalloc"));
    }
    cudaStream_t s = G->stream;
    uint32_t bad[2] = {0, 0};     // flags, largest weight
    e = cudaMemcpyAsync(G->g.row_ptr, irp, ((size_t)n + 1) * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && relabel)
        e = cudaMemcpyAsync(G->g.orig_row_ptr, row_ptr, ((size_t)n + 1) * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && relabel)
        e = cudaMemcpyAsync(G->g.orig_of, h_orig_of.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && relabel)
        e = cudaMemcpyAsync(G->g.new_of, h_new_of.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && n_arcs)
        e = cudaMemcpyAsync(d_col, col, (size_t)n_arcs * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && n_arcs)
        e = cudaMemcpyAsync(d_w, w, (size_t)n_arcs * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !chunks.empty())
        e = cudaMemcpyAsync(G->g.heavy_chunks, chunks.data(), chunks.size() * 8,
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0, 8, s);
    if (e == cudaSuccess)
        e = launch_validate_graph(relabel ? G->g.orig_row_ptr : G->g.row_ptr, d_col, d_w, n, n_arcs,
                                  G->g.adj, G->g.new_of, relabel ? G->g.row_ptr : nullptr, d_bad,
                                  d_bad + 1, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bad, d_bad, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_col);
    cudaFree(d_w);
    cudaFree(d_bad);
    if (e != cudaSuccess) return bail(cuda_fail(e, "graph upload"));
    if (bad[0]) {
        char msg[160];
        snprintf(msg, sizeof msg, "malformed graph (flags 0x%x: 1 range, 2 self-loop, 4 zero weight, "
                 "8 unsorted/duplicate, 16 asymmetric)", bad[0]);
        return bail(fail(STEINER_EINVAL, msg));
    }
    G->g.max_w = bad[1];
    // launch geometry of the persistent kernels
    cudaDeviceGetAttribute(&G->geo.sm_count, cudaDevAttrMultiProcessorCount, device);
    G->geo.threads = 256;
    int per_sm = sssp_occupancy(256);
    if (per_sm < 1) return bail(fail(STEINER_ECUDA, "SSSP kernel does not fit on an SM"));
    G->geo.sssp_blocks = per_sm * G->geo.sm_count;
    G->geo.sssp_max_blocks = G->geo.sssp_blocks;
    int mst_sm = mst_occupancy(512);
    G->geo.mst_blocks = std::max(1, mst_sm) * G->geo.sm_count;
    // default band width: ~32 average weights spread over the average degree
    double avg_w = 0;
    if (n_arcs) {
        uint64_t step = std::max<uint64_t>(1, n_arcs / 65536), cnt = 0;
        for (uint64_t i = 0; i < n_arcs; i += step, ++cnt) avg_w += w[i];
        avg_w /= (double)cnt;
    }
    double d = 32.0 * std::max(1.0, avg_w) / std::max(1.0, avg_deg);
    G->delta = (uint32_t)std::min(std::max(d, 1.0), 1.0e9);
    if (const char *env = getenv("STEINER_DELTA")) G->delta = (uint32_t)std::max(1L, atol(env));
    *out = G;
    return STEINER_OK;
}

void steiner_free_graph(steiner_graph_t G) {
    if (!G) return;
    if (G->serve) {
        steiner_serve_stop(G);
    }
    destroy_batch(G->batch);
    G->batch = nullptr;
    cudaSetDevice(G->device);
    if (G->stream) cudaStreamSynchronize(G->stream);
    Workspace &ws = G->ws;
    void *bufs[] = {ws.label, ws.label32, ws.nbm[0], ws.nbm[1], ws.bbm, ws.pred_arc, ws.stamp_near, ws.stamp_far, ws.stamp_band, ws.band_q,
                    ws.band_hq, ws.mark, ws.q[0], ws.q[1],
                    ws.hq[0], ws.hq[1], ws.far[0], ws.far[1], ws.ctl, ws.seeds, ws.pairtab,
                    ws.e_key, ws.e_ra, ws.e_rb, ws.e_arc, ws.e_mst, ws.tile_off, ws.comp, ws.hook,
                    ws.best, ws.tree_key, ws.tree_key2, ws.tree_w, ws.tree_w2, G->g.row_ptr,
                    G->g.adj, G->g.heavy_chunks, G->g.orig_row_ptr, G->g.orig_of, G->g.new_of,
                    G->g.adj_w, G->g.lend};
    for (void *p : bufs)
        if (p) cudaFree(p);
    for (auto &ev : G->ev)
        if (ev) cudaEventDestroy(ev);
    if (G->h_ctl) cudaFreeHost(G->h_ctl);
    if (G->stream) cudaStreamDestroy(G->stream);
    delete G;
}

int steiner_set_param(steiner_graph_t G, const char *key, int64_t value) {
    if (!G || !key) return fail(STEINER_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(G->mu);
    if (!strcmp(key, "delta")) {
        if (value < 1 || value > 0x7FFFFFFF) return fail(STEINER_EINVAL, "delta out of range");
        G->delta = (uint32_t)value;
    } else if (!strncmp(key, "batch_", 6)) {
        return batch_set_param(G, key, value);
    } else if (!strcmp(key, "sssp_blocks")) {
        // persistent grid size: 1 .. all co-resident blocks (0 = all)
        int maxb = G->geo.sssp_max_blocks;
        if (value < 0 || value > maxb) return fail(STEINER_EINVAL, "sssp_blocks out of range");
        G->geo.sssp_blocks = value ? (int)value : maxb;
    } else if (!strcmp(key, "local_rounds")) {
        if (value < 0 || value > 1024) return fail(STEINER_EINVAL, "local_rounds out of range");
        G->local_rounds = (uint32_t)value;
    } else if (!strcmp(key, "dense")) {
        if (value != 0 && value != 1) return fail(STEINER_EINVAL, "dense must be 0 or 1");
        G->dense = (uint32_t)value;
    } else if (!strcmp(key, "tail")) {
        if (value != 0 && value != 1) return fail(STEINER_EINVAL, "tail must be 0 or 1");
        G->tail = (uint32_t)value;
    } else if (!strcmp(key, "pull")) {
        if (value < 0 || value > 2) return fail(STEINER_EINVAL, "pull must be 0, 1 or 2");
        G->pull = (uint32_t)value;
    } else if (!strcmp(key, "far_scan")) {
        if (value < -1 || value > 1) return fail(STEINER_EINVAL, "far_scan must be -1, 0 or 1");
        G->far_scan = (int)value;
    } else if (!strcmp(key, "label_bits")) {
        if (value != 0 && value != 32 && value != 64)
            return fail(STEINER_EINVAL, "label_bits must be 0 (automatic), 32 or 64");
        G->label_bits = (uint32_t)value;
    } else if (!strcmp(key, "max_iters")) {
        if (value < 1 || value > 0x7FFFFFFF) return fail(STEINER_EINVAL, "max_iters out of range");
        G->max_iters = (uint32_t)value;
    } else {
        return fail(STEINER_EINVAL, std::string("unknown parameter ") + key);
    }
    return STEINER_OK;
}

int64_t steiner_get_param(steiner_graph_t G, const char *key) {
    if (!G || !key) return -1;
    if (!strcmp(key, "delta")) return G->delta;
    if (!strcmp(key, "max_iters")) return G->max_iters;
    if (!strcmp(key, "local_rounds")) return G->local_rounds;
    if (!strcmp(key, "sssp_blocks")) return G->geo.sssp_blocks;
    if (!strcmp(key, "sssp_max_blocks")) return G->geo.sssp_max_blocks;
    if (!strcmp(key, "sm_count")) return G->geo.sm_count;
    if (!strcmp(key, "heavy_chunks")) return G->g.n_heavy_chunks;
    if (!strcmp(key, "label_bits")) return G->label_bits;
    if (!strcmp(key, "far_scan")) return G->far_scan;
    if (!strcmp(key, "dense")) return G->dense;
    if (!strcmp(key, "pull")) return G->pull;
    if (!strcmp(key, "pull_passes_last")) return G->last_pulls;
    if (!strcmp(key, "tail")) return G->tail;
    if (!strcmp(key, "tail_iteration_last")) return G->last_tail_it;
    if (!strcmp(key, "label_bits_last")) return G->last_label_bits;
    if (!strcmp(key, "narrow_reruns")) return (int64_t)G->narrow_reruns;
    if (!strncmp(key, "batch_", 6)) return batch_counter(G->batch, key);
    return -1;
}

int steiner_query(steiner_graph_t G, const int32_t *seeds, uint32_t k, steiner_result_t *out) {
    return steiner_query_detail(G, seeds, k, out, nullptr, nullptr, nullptr);
}

int steiner_query_detail(steiner_graph_t G, const int32_t *seeds, uint32_t k,
                         steiner_result_t *out, steiner_pair_t **pairs, uint64_t *n_pairs,
                         steiner_stats_t *stats) {
    if (!G || !out) return fail(STEINER_EINVAL, "null argument");
    if (pairs) *pairs = nullptr;
    if (n_pairs) *n_pairs = 0;
    std::lock_guard<std::mutex> lk(G->mu);
    CK(cudaSetDevice(G->device));
    return query_locked(G, seeds, k, out, pairs, n_pairs, stats);
}

int steiner_voronoi(steiner_graph_t G, const int32_t *seeds, uint32_t k, int32_t *cell,
                    uint32_t *dist, int32_t *pred) {
    if (!G) return fail(STEINER_EINVAL, "null graph");
    std::lock_guard<std::mutex> lk(G->mu);
    CK(cudaSetDevice(G->device));
    std::vector<int32_t> ss;
    int rc = sorted_seed_list(G, seeds, k, ss);
    if (rc) return rc;
    rc = run_pipeline(G, ss, false, nullptr);
    if (rc) return rc;
    Control c = *G->h_ctl;
    rc = status_from(c, k, false);
    if (rc) return rc;
    uint32_t n = G->g.n;
    cudaStream_t s = G->stream;
    // device outputs are written in place; host outputs go through the
    // (idle) tree buffers and are copied back
    int32_t *d_cell = cell, *d_pred = pred;
    uint32_t *d_dist = dist;
    bool hc = cell && !is_device_ptr(cell), hd = dist && !is_device_ptr(dist),
         hp = pred && !is_device_ptr(pred);
    if (hc) d_cell = reinterpret_cast<int32_t *>(G->ws.tree_key);
    if (hd) d_dist = reinterpret_cast<uint32_t *>(G->ws.tree_key2);
    if (hp) d_pred = reinterpret_cast<int32_t *>(G->ws.tree_w);
    CK(launch_export(G->g, G->ws, k, d_cell, d_dist, d_pred, s));
    if (hc) CK(cudaMemcpyAsync(cell, d_cell, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
    if (hd) CK(cudaMemcpyAsync(dist, d_dist, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
    if (hp) CK(cudaMemcpyAsync(pred, d_pred, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return STEINER_OK;
}

void steiner_result_free(steiner_result_t *r) {
    if (!r) return;
    free(r->edges);
    r->edges = nullptr;
    r->n_edges = 0;
}

void steiner_pairs_free(steiner_pair_t *p) { free(p); }

}  // extern "C"

// ---------------------------------------------------------------------------
// helpers used by the batch and serving engines
// ---------------------------------------------------------------------------

namespace stn {

int api_query_locked(steiner_graph *G, const int32_t *seeds, uint32_t k, steiner_result_t *out) {
    return query_locked(G, seeds, k, out, nullptr, nullptr, nullptr);
}

// Steps 3-7 of Algorithm 2 for one slot of the multi-query engine: the
// slot's pair table and strided predecessor column feed the single-query
// compaction, MST, expansion and sort kernels.  Caller holds G->mu.
int api_run_tail(steiner_graph *G, uint64_t *pairtab, uint32_t *pred_base, uint32_t pred_stride,
                 uint32_t k, bool overflow, steiner_result_t *out) {
    out->edges = nullptr;
    out->n_edges = 0;
    out->total = 0;
    if (overflow)
        return out->status = fail(STEINER_EOVERFLOW, "a distance or bridge sum reached 2^32 - 1");
    int rc = ensure_n_workspace(G);
    if (!rc) rc = ensure_k_workspace(G, k, false);
    if (rc) return out->status = rc;
    Workspace v = G->ws;
    v.pairtab = pairtab;
    v.pred_arc = pred_base;
    v.pred_stride = pred_stride;
    cudaStream_t s = G->stream;
    CK(cudaMemsetAsync(v.ctl, 0, sizeof(Control), s));
    CK(launch_compact_pairs(v, k, s));
    CK(launch_mst(v, k, G->geo, s));
    CK(launch_tree(G->g, v, k, G->ws.epoch_mark, G->nbits, s));
    CK(cudaMemcpyAsync(G->h_ctl, v.ctl, sizeof(Control), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    G->ws.epoch_mark += 1;
    if (G->ws.epoch_mark > 0x7FFFFFFFu) {
        CK(cudaMemsetAsync(G->ws.mark, 0, (size_t)G->ws.n * 4, s));
        G->ws.epoch_mark = 1;
    }
    const Control c = *G->h_ctl;
    rc = status_from(c, k, true);
    if (rc == STEINER_OK || rc == STEINER_EDISCONNECTED) {
        int rc2 = fetch_tree(G, out);
        if (rc2) return out->status = rc2;
    }
    return out->status = rc;
}

int api_sorted_seeds(steiner_graph *G, const int32_t *seeds, uint32_t k, std::vector<int32_t> &out) {
    return sorted_seed_list(G, seeds, k, out);
}

cudaStream_t api_stream(steiner_graph *G) { return G->stream; }

uint32_t api_reserve_mark_tags(steiner_graph *G, uint32_t count, uint32_t **mark) {
    *mark = nullptr;
    if (ensure_n_workspace(G) != STEINER_OK) return 0;
    Workspace &ws = G->ws;
    if ((uint64_t)ws.epoch_mark + count > 0x7FFFFFFFull) {
        if (cudaMemsetAsync(ws.mark, 0, (size_t)ws.n * 4, G->stream) != cudaSuccess) return 0;
        ws.epoch_mark = 1;
    }
    const uint32_t tag0 = ws.epoch_mark;
    ws.epoch_mark += count;
    *mark = ws.mark;
    return tag0;
}

std::mutex &api_mutex(steiner_graph *G) { return G->mu; }
const DevGraph &api_graph(steiner_graph *G) { return G->g; }
int api_device(steiner_graph *G) { return G->device; }
BatchEngine *&api_batch(steiner_graph *G) { return G->batch; }
ServeEngine *&api_serve(steiner_graph *G) { return G->serve; }
uint32_t api_delta(steiner_graph *G) { return G->delta; }
void api_ensure_partition(steiner_graph *G, uint32_t delta) {
    ensure_partition_dev(G->g, delta, G->stream);
}
uint32_t api_nbits(steiner_graph *G) { return G->nbits; }
const Geometry &api_geometry(steiner_graph *G) { return G->geo; }
void api_set_error(const std::string &msg) { g_last_error = msg; }

}  // namespace stn
