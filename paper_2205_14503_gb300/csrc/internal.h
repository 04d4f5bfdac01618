// Internal interfaces between the C ABI (api.cu) and the kernel files.
// Host-visible structs describe device buffers; launchers enqueue work on
// a caller stream and never synchronise.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace stn {

// Degree at or above which a vertex's adjacency is processed in chunks of
// CHUNK arcs (one warp per chunk) instead of inside a 32-vertex batch.
constexpr uint32_t HEAVY_DEG = 256;
constexpr uint32_t CHUNK = 512;

// Resident graph: row offsets and interleaved (neighbour, weight) arcs.
struct DevGraph {
    uint32_t n = 0;
    uint64_t m = 0;                 // arcs
    uint32_t *row_ptr = nullptr;    // n + 1
    uint2 *adj = nullptr;           // m: {col, w}
    uint64_t *heavy_chunks = nullptr;   // (v << 32) | chunk index, for deg >= HEAVY_DEG
    uint32_t n_heavy_chunks = 0;
    uint32_t heavy_chunk_cap = 0;   // bound on chunk entries a frontier can hold
    uint32_t max_w = 0;             // largest arc weight
    // Internal vertex order.  On a skewed degree distribution the vertices
    // are renumbered by descending degree (ties by id), so the labels of
    // the hubs that most arcs point to share L2 sectors; rows keep the
    // caller's order of neighbours (ascending caller id).  All results are
    // reported in the caller's ids and arc indices.  Null: identity.
    uint32_t *orig_of = nullptr;     // internal id -> caller id, n
    uint32_t *new_of = nullptr;      // caller id -> internal id, n
    uint32_t *orig_row_ptr = nullptr;   // the caller's row offsets, n + 1
    // Weight-partitioned copy of adj for the Voronoi kernels (built for one
    // band width at a time): row v holds its arcs lighter than part_delta
    // in [row_ptr[v], lend[v]) and the rest in [lend[v], row_ptr[v + 1]).
    // The id-sorted adj stays the reference for pred, bridges and the tree.
    uint2 *adj_w = nullptr;
    uint32_t *lend = nullptr;
    uint32_t part_delta = 0;        // 0: not built
    // Vertices with ids at or above n_big have fewer than HEAVY_DEG arcs
    // (the descending-degree order puts the hubs first; n without it).
    uint32_t n_big = 0;
};

// The weight-partitioned rows to use for band width delta: built for that
// width and the split on (delta at or below the largest weight), else null.
inline const uint32_t *active_lend(const DevGraph &g, uint32_t delta) {
    return (delta <= g.max_w && g.adj_w && g.lend && g.part_delta == delta) ? g.lend : nullptr;
}

// Offset from internal to caller arc indices along internal row v (which
// starts at rs): the caller's index of internal arc `arc` of the row is
// caller_arc_base(...) + arc, modulo 2^32.
__device__ __forceinline__ uint32_t caller_arc_base(const uint32_t *orig_of,
                                                    const uint32_t *orig_row_ptr, uint32_t v,
                                                    uint32_t rs) {
    return orig_of ? orig_row_ptr[orig_of[v]] - rs : 0u;
}

__device__ __forceinline__ uint32_t caller_id(const uint32_t *orig_of, uint32_t v) {
    return orig_of ? orig_of[v] : v;
}

__device__ __forceinline__ uint32_t internal_id(const uint32_t *new_of, uint32_t v) {
    return new_of ? new_of[v] : v;
}

constexpr int TRACE_LEN = 128;

// Device control block of one query.
struct Control {
    GridBarrier bar;
    uint32_t err;
    uint32_t near_count[3];
    uint32_t heavy_count[3];
    uint32_t far_count[2];
    uint32_t far_min[2];
    uint32_t iterations;
    uint32_t phases;
    unsigned long long relax_attempts;
    unsigned long long relax_improved;
    // bridge / tree phases
    uint32_t n_pairs;
    uint32_t n_mst;
    uint32_t n_tree;
    uint32_t pad;
    unsigned long long total;
    GridBarrier bar2;
    uint32_t mst_any;
    uint32_t exit_reason;        // 1 converged, 2 iteration cap, 3/4 barrier gave up
    // band lists of the light/heavy arc split: vertices relaxed in the
    // current band (light items, heavy-row chunks) and the passes run
    uint32_t band_count;
    uint32_t band_hcount;
    uint32_t bands;
    uint32_t pulls;              // heavy-arc passes run in the pull form
    uint32_t tail_it;            // iteration the unbounded tail band began at (0: none)
    // heavy arcs of the vertices listed in the current band (a vertex
    // listed twice counts twice), and of the vertices a pull pass found
    // unsettled: the push and pull costs of a band's heavy-arc pass
    unsigned long long band_hsum;
    unsigned long long pull_hsum;
    uint32_t trace[TRACE_LEN][4];  // first iterations: near items, heavy chunks, far pile, T
    unsigned long long trace_ns[TRACE_LEN];   // their start times (global timer, ns)
    unsigned long long trace_relax[TRACE_LEN][3];   // relaxations, improvements, atomics (traced)
    unsigned long long trace_busy[TRACE_LEN][2];    // warps' relaxation time: sum, max (ns)
    unsigned long long end_ns;                // end of the last iteration
};

// Per-query device workspace for the single-query path.
struct Workspace {
    uint32_t n = 0;
    uint64_t *label = nullptr;      // (dist << 32) | rank
    // Narrow labels (dist << lshift) | rank, used instead of `label` by the
    // Voronoi, scan and export kernels of a query with `narrow` set.
    uint32_t *label32 = nullptr;
    uint32_t lshift = 0;
    bool narrow = false;
    uint32_t *pred_arc = nullptr;   // arc of the pred edge in v's row; SEED_ARC; INF32
    uint32_t pred_stride = 1;       // pred of v at pred_arc[v * pred_stride]
    uint32_t *stamp_near = nullptr;
    uint32_t *stamp_far = nullptr;
    uint32_t *stamp_band = nullptr;  // band-list membership tags
    uint32_t *band_q = nullptr;      // vertices relaxed in the current band, n
    uint64_t *band_hq = nullptr;     // their heavy-row chunks, heavy_chunk_cap
    uint32_t *mark = nullptr;       // tree-walk stamps
    // dense frontiers: near bitmaps (alternating by iteration) and the band
    // bitmap, ceil(n / 32) words each, all zero between queries
    uint32_t *nbm[2] = {nullptr, nullptr};
    uint32_t *bbm = nullptr;
    uint32_t *q[2] = {nullptr, nullptr};      // light frontier
    uint64_t *hq[2] = {nullptr, nullptr};     // heavy-chunk frontier
    uint32_t *far[2] = {nullptr, nullptr};
    Control *ctl = nullptr;
    int32_t *seeds = nullptr;       // sorted seed ids (rank order)
    uint32_t seeds_cap = 0;
    uint64_t *pairtab = nullptr;    // k (k - 1) / 2 packed (b << 32 | arc)
    uint64_t pairtab_cap = 0;
    // compacted distance graph
    uint64_t *e_key = nullptr;      // (b << 32) | slot
    uint32_t *e_ra = nullptr, *e_rb = nullptr, *e_arc = nullptr;
    uint32_t *e_mst = nullptr;
    uint32_t *tile_off = nullptr;
    uint64_t e_cap = 0;
    uint32_t tile_cap = 0;
    // MST scratch (k entries)
    uint32_t *comp = nullptr, *hook = nullptr;
    unsigned long long *best = nullptr;
    uint32_t comp_cap = 0;
    // tree output
    uint64_t *tree_key = nullptr, *tree_key2 = nullptr;   // (min << 32) | max
    uint32_t *tree_w = nullptr, *tree_w2 = nullptr;
    uint32_t tree_cap = 0;
    // tags that avoid clearing the stamp arrays between queries
    uint32_t epoch_near = 0, epoch_far = 0, epoch_mark = 0, epoch_band = 0;
};

// Launch geometry of the persistent kernels (from the occupancy API).
struct Geometry {
    int sm_count = 0;
    int sssp_blocks = 0;        // persistent grid size in use
    int sssp_max_blocks = 0;    // co-resident limit (occupancy x SMs)
    int mst_blocks = 0;
    int threads = 256;
};

struct SsspParams {
    uint32_t delta;          // near/far band width
    uint32_t max_iters;      // loop cap -> ERR_TIMEOUT
    uint32_t base_near;      // first near tag of this query
    uint32_t base_far;       // first far tag of this query
    uint32_t local_rounds;   // warp-local relaxation rounds per iteration
    uint32_t base_band;      // first band-list tag of this query
    uint32_t far_scan;       // splits scan the labels instead of a far pile
    uint32_t trace;          // per-iteration relaxation counts into Control::trace_relax
    uint32_t dense;          // dense frontiers (needs far_scan and no local rounds)
    uint32_t pull;           // heavy-arc passes: 0 push, 1 push or pull by cost, 2 pull (far_scan)
    uint32_t tail;           // after a pull pass, the rest as one unbounded band (1) or not (0)
};

// SM count of the current device (queried once per device, then cached);
// the launchers size their grids in multiples of it.
int current_sm_count();

// voronoi.cu
cudaError_t launch_init(const DevGraph &g, Workspace &ws, uint32_t k, uint32_t delta,
                        cudaStream_t s);
cudaError_t launch_sssp(const DevGraph &g, Workspace &ws, const Geometry &geo,
                        const SsspParams &p, cudaStream_t s);
cudaError_t launch_export(const DevGraph &g, Workspace &ws, uint32_t k, int32_t *cell,
                          uint32_t *dist, int32_t *pred, cudaStream_t s);
int sssp_occupancy(int threads);

// bridge.cu
cudaError_t launch_scan(const DevGraph &g, Workspace &ws, uint32_t k, bool pairs,
                        cudaStream_t s);
cudaError_t launch_compact_pairs(Workspace &ws, uint32_t k, cudaStream_t s);

// tree.cu
cudaError_t launch_mst(Workspace &ws, uint32_t k, const Geometry &geo, cudaStream_t s);
cudaError_t launch_tree(const DevGraph &g, Workspace &ws, uint32_t k, uint32_t tag,
                        uint32_t n_bits, cudaStream_t s);
int mst_occupancy(int threads);
cudaError_t launch_sort_keys(uint64_t *key0, uint64_t *key1, uint32_t *w0, uint32_t *w1,
                             uint32_t *blk_hist, uint32_t cap, uint32_t key_bits, Control *ctl,
                             cudaStream_t s);

// graph.cu
// Builds g.adj_w / g.lend for band width delta (both allocated by the caller).
cudaError_t launch_partition(const DevGraph &g, uint32_t delta, cudaStream_t s);
// With the light/heavy split on for band width delta (delta at or below the
// largest weight), the Voronoi kernels read rows partitioned by weight
// class: allocates and builds (or rebuilds, after a change of delta) that
// copy.  On failure part_delta is 0 and the kernels filter arcs by weight
// on the id-sorted rows instead.
cudaError_t ensure_partition_dev(DevGraph &g, uint32_t delta, cudaStream_t s);
// Validates the caller's CSR (row_ptr, col, w) and writes the interleaved
// internal adjacency: arc e of caller row u goes to
// new_row_ptr[new_of[u]] + (e - row_ptr[u]) with neighbour new_of[col[e]]
// (new_of / new_row_ptr null: the identity).
cudaError_t launch_validate_graph(const uint32_t *row_ptr, const int32_t *col,
                                  const uint32_t *w, uint32_t n, uint64_t m, uint2 *adj,
                                  const uint32_t *new_of, const uint32_t *new_row_ptr,
                                  uint32_t *bad, uint32_t *max_w, cudaStream_t s);

}  // namespace stn
