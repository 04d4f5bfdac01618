// Voronoi cells of all seeds at once (Algorithm 2 Step 1; Algorithm 4 is the
// paper's asynchronous vertex-centric form of the same fixed point).
//
// Every vertex v holds one packed label (d1(src(v), v) << 32) | rank(src(v)).
// Relaxing an arc u -> v proposes (d(u) + d(u,v)) << 32 | rank(u) and keeps
// the minimum with a 64-bit atomicMin, so the fixed point is, per vertex,
// the lexicographic minimum over seeds of (distance, seed rank): the
// nearest seed, ties to the smallest seed id.  The fixed point does not
// depend on the order in which relaxations land.
//
// Order of work: a near/far frontier (a two-bucket delta-stepping).  The
// paper prioritises low-distance messages in its message queue (Section
// "Distributed Implementation"); on the GPU the same effect comes from
// relaxing only vertices whose distance is below a threshold T (near) and
// parking the rest (far) until the near frontier drains, then raising T by
// delta.  One persistent cooperative kernel runs all iterations with a
// bounded grid barrier between them.
//
// Light and heavy arcs (the edge classes of delta-stepping): while a band
// [T - delta, T) iterates, only arcs lighter than delta are relaxed, since
// a heavier arc out of the band cannot land inside it.  Every vertex
// relaxed in the band is listed once; when the band's frontier drains, one
// extra pass relaxes the heavy arcs of the listed vertices with their final
// labels, so a vertex improved several times inside its band (a hub reached
// by many light paths) scans its heavy arcs once.  All of its proposals land
// at or above T, in the far pile.  The split is on only when some arc
// weight reaches delta.
//
// Pull form of the heavy-arc pass (with the far scan): once a band has
// drained, every label below T is final, and a heavy proposal can only
// change a vertex still at or above T.  So instead of pushing the heavy
// arcs of the band's vertices, every unsettled vertex may read its own
// heavy arcs and the labels at their other ends, keeping the best proposal
// from those below T.  Both forms reach the same labels; the pass takes
// the form that reads fewer arcs.  On a small-world graph the first band
// holds most of the vertices and nearly all heavy arcs, while the vertices
// left unsettled have few (direction-optimising search, Beamer et al.,
// applied to delta-stepping's heavy-arc phase).
#include "internal.h"

namespace stn {

struct SsspArgs {
    const uint32_t *__restrict__ row_ptr;
    const uint2 *__restrict__ adj;
    uint32_t n;
    uint64_t *label;         // 64-bit labels (the wide kernel)
    uint32_t *label32;       // narrow labels (the narrow kernel)
    uint32_t lshift;         // rank bits of a narrow label
    uint32_t ldmax;          // largest distance a narrow label holds
    uint32_t *stamp_near;
    uint32_t *stamp_far;
    uint32_t *q0, *q1;
    uint64_t *hq0, *hq1;
    uint32_t *far0, *far1;
    Control *ctl;
    uint32_t delta;
    uint32_t max_iters;
    uint32_t base_near;
    uint32_t base_far;
    uint32_t heavy_cap;
    uint32_t local_rounds;   // warp-local relaxation rounds per iteration (0 = off)
    uint32_t *stamp_band;    // band-list membership tags
    uint32_t *band_q;        // vertices relaxed in the current band
    uint64_t *band_hq;       // heavy-row chunks of listed high-degree vertices
    uint32_t base_band;
    uint32_t defer;          // light/heavy arc split on
    uint32_t far_scan;       // no far pile: splits find far vertices by scanning the labels
    uint32_t trace;          // record per-iteration relaxation counts
    // Dense frontiers (with the far scan, without local rounds): a large
    // frontier is a bitmap (one bit per vertex, set with a fire-and-forget
    // atomicOr) read in id order by the next iteration, and the band list
    // of the light/heavy split is a bitmap too; hubs keep their chunk
    // queues.  Ids below n_big may have HEAVY_DEG arcs or more, ids at or
    // above it have fewer (the degree order makes this a bound).
    uint32_t dense;
    uint32_t pull;           // heavy-arc passes: 0 push, 1 by cost, 2 pull
    uint32_t tail;           // 1: after a pull pass the rest runs as one unbounded band
    uint64_t m;              // arcs (the first bound on a pull pass's cost)
    uint32_t n_big;
    uint32_t n_words;        // bitmap words, ceil(n / 32)
    uint32_t *nbm0, *nbm1;   // near bitmaps, alternating by iteration
    uint32_t *bbm;           // band bitmap
    // with the split: end of each row's light part in the weight-partitioned
    // adjacency `adj` (null: rows are unpartitioned and arcs are filtered)
    const uint32_t *lend;
};

// ---------------------------------------------------------------------------
// init (Algorithm 3, INITIALIZATION): every label at infinity, then each
// seed at distance 0 in its own cell and on the first frontier.
// ---------------------------------------------------------------------------

__global__ void init_labels_kernel(uint32_t n, uint64_t *__restrict__ label,
                                   uint32_t *__restrict__ label32,
                                   uint32_t *__restrict__ pred_arc) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (label32) label32[v] = INF32;
        else label[v] = INF64;
        pred_arc[v] = INF32;
    }
}

__global__ void init_seeds_kernel(const uint32_t *__restrict__ row_ptr,
                                  const uint32_t *__restrict__ lend, const int32_t *seeds,
                                  const uint32_t *__restrict__ new_of,
                                  uint32_t k, uint64_t *label, uint32_t *label32,
                                  uint32_t *pred_arc,
                                  uint32_t *stamp_near, uint32_t tag0, uint32_t *q0,
                                  uint64_t *hq0, uint32_t heavy_cap, uint32_t n, Control *ctl) {
    uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r == 0) {
        ctl->far_min[0] = INF32;
        ctl->far_min[1] = INF32;
    }
    if (r >= k) return;
    uint32_t s = internal_id(new_of, (uint32_t)seeds[r]);
    if (label32) label32[s] = r;          // distance 0, cell = rank r
    else label[s] = (uint64_t)r;
    pred_arc[s] = SEED_ARC;
    stamp_near[s] = tag0;
    uint32_t rs = row_ptr[s], deg = (lend ? lend[s] : row_ptr[s + 1]) - rs;   // near part
    if (deg >= HEAVY_DEG) {
        uint32_t nc = (deg + CHUNK - 1) / CHUNK;
        uint32_t base = atomicAdd(&ctl->heavy_count[0], nc);
        if (base + nc > heavy_cap) { atomicOr(&ctl->err, ERR_CAPACITY); return; }
        for (uint32_t c = 0; c < nc; ++c) hq0[base + c] = ((uint64_t)s << 32) | c;
    } else {
        uint32_t slot = atomicAdd(&ctl->near_count[0], 1u);
        if (slot >= n) { atomicOr(&ctl->err, ERR_CAPACITY); return; }
        q0[slot] = s;
    }
}

// ---------------------------------------------------------------------------
// relaxation: U arcs in flight per lane; frontier appends staged per block
// ---------------------------------------------------------------------------

constexpr int ILP = 4;                 // arcs per lane per round group (relax_group's
                                       // early exit tests imp[0..3] by name: keep 4)
constexpr uint32_t NEAR_STAGE = 4096;  // block staging capacity (near items)
constexpr uint32_t SSSP_WARPS = 8;     // warps per block (256 threads)
constexpr uint32_t NEAR_REGION = NEAR_STAGE / SSSP_WARPS;   // one region per warp
constexpr uint32_t FAR_STAGE = 1024;   // block staging capacity (far items)
constexpr uint32_t BAND_STAGE = 2048;  // block staging capacity (band-list items)
constexpr uint32_t BAND_REGION = BAND_STAGE / SSSP_WARPS;
constexpr int SPLIT_ILP = 4;           // 32-vertex chunks per warp step in a band split
constexpr uint32_t DENSE_WORDS = 8;    // bitmap words per dense work item (light arcs)
constexpr uint32_t DENSE_WORDS_HP = 8; // the same in a heavy-arc pass
constexpr int PULL_ILP = 4;            // 32-vertex chunks per warp step in a pull pass

// Where the appends of one processing segment go.
struct PushTargets {
    uint32_t *qn;        // light queue of the next iteration
    uint32_t *qn_count;
    uint64_t *hqn;       // heavy-chunk queue of the next iteration
    uint32_t *hqn_count;
    uint32_t *farq;      // far pile of the current phase
    uint32_t *far_count;
    uint32_t *far_min;
    uint32_t *bandq;     // band list and its fill counter
    uint32_t *band_count;
    uint32_t tag_next;
    uint32_t tag_far;
    uint64_t T;
    // A full warp region may move to the global queue mid-segment (not
    // during the warp-local rounds, which index into the region).
    bool flush;
    // Near pushes of light vertices set bits of nbm (the next iteration
    // reads the bitmap) instead of going through the queue.
    bool dense;
    uint32_t *nbm;
    // With warp-local rounds: every improvement appends its vertex to the
    // improving warp's region with no stamp (a region may hold a vertex
    // twice, and a warp-local round simply reads the current label); the
    // near stamps deduplicate items only on their way to the global queue.
    bool nostamp;
    uint32_t *nostamp_stamp;     // the near stamps (for the deduplication)
    unsigned long long *hsum;    // receives the warps' heavy-arc sums (null: none)
    // end of each row's part relaxed by a near vertex (the light part while
    // the light/heavy split is on); null: whole rows
    const uint32_t *lend;
};

// Per-block staging buffers.  Near and band-list appends go to one region
// per warp, which only that warp touches: a full region moves to the global
// queue with one global atomicAdd (one per region, not one per append: a
// single queue counter that every warp bumps on every append serialises the
// whole grid on one L2 address), and the rest moves at the end of the
// segment (flush_stage).  In the local rounds a warp relaxes its own near
// region.  Far appends share one block buffer (shared-memory atomics).
struct Stage {
    uint32_t near_buf[NEAR_STAGE];
    uint32_t far_buf[FAR_STAGE];
    uint32_t band_buf[BAND_STAGE];
    uint32_t band_n[SSSP_WARPS];    // items staged per band region
    uint32_t dn_near[SSSP_WARPS];   // bits set in the near bitmap by each warp
    uint32_t dn_band[SSSP_WARPS];   // bits set in the band bitmap by each warp
    uint32_t hs[SSSP_WARPS];        // heavy arcs listed (or pulled) by each warp
    uint32_t near_n[SSSP_WARPS];    // items staged per warp region
    uint32_t local_lo[SSSP_WARPS];  // region[0, local_lo) was relaxed by its warp already
    uint32_t near_off[SSSP_WARPS];  // flush: offset of each region's rest
    uint32_t far_n, far_min;
    uint32_t base_near, base_far;
};

__device__ __forceinline__ void stage_reset(Stage &st) {
    if (threadIdx.x == 0) {
        st.far_n = 0;
        st.far_min = INF32;
    }
    if (threadIdx.x < SSSP_WARPS) {
        st.near_n[threadIdx.x] = 0;
        st.band_n[threadIdx.x] = 0;
        st.dn_near[threadIdx.x] = 0;
        st.dn_band[threadIdx.x] = 0;
        st.hs[threadIdx.x] = 0;
        st.local_lo[threadIdx.x] = 0;
    }
    __syncthreads();
}

// Moves the block's staged appends to the global queues.  Called by all
// threads of the block; ends with the staging buffers still holding data
// (stage_reset clears them at the next segment).
__device__ __forceinline__ void flush_stage(Stage &st, const PushTargets &t, uint32_t n,
                                            uint32_t *err) {
    __syncthreads();
    const uint32_t nf = min(st.far_n, FAR_STAGE);
    if (threadIdx.x == 0) {
        uint32_t nn = 0;
        for (uint32_t w = 0; w < SSSP_WARPS; ++w) {
            const uint32_t hi = min(st.near_n[w], NEAR_REGION), lo = st.local_lo[w];
            st.near_off[w] = nn;
            if (!t.nostamp) nn += hi > lo ? hi - lo : 0;
        }
        st.base_near = nn ? atomicAdd(t.qn_count, nn) : 0;
        st.base_far = nf ? atomicAdd(t.far_count, nf) : 0;
        if (st.far_min != INF32) atomicMin(t.far_min, st.far_min);
        // bits set in the bitmaps count as items (a vertex set twice counts
        // twice): the counts only size the next iteration and show that a
        // frontier or band list is non-empty
        uint32_t dnn = 0, dnb = 0;
        for (uint32_t w = 0; w < SSSP_WARPS; ++w) {
            dnn += st.dn_near[w];
            dnb += st.dn_band[w];
        }
        if (dnn) atomicAdd(t.qn_count, dnn);
        if (dnb) atomicAdd(t.band_count, dnb);
        if (t.hsum) {
            unsigned long long hs = 0;
            for (uint32_t w = 0; w < SSSP_WARPS; ++w) hs += st.hs[w];
            if (hs) atomicAdd(t.hsum, hs);
        }
    }
    __syncthreads();
    {   // each warp moves the rest of its own regions
        const uint32_t w = threadIdx.x >> 5;
        const uint32_t hi = min(st.near_n[w], NEAR_REGION), lo = st.local_lo[w];
        if (t.nostamp) {            // deduplicated on the way
            for (uint32_t i0 = lo; i0 < hi; i0 += 32) {
                const uint32_t i = i0 + lane_id();
                queue_append(i < hi, i < hi ? st.near_buf[w * NEAR_REGION + i] : 0u, t.qn,
                             t.qn_count, n, err, t.nostamp_stamp, t.tag_next);
            }
        } else {
            for (uint32_t i = lo + lane_id(); i < hi; i += 32) {
                uint32_t slot = st.base_near + st.near_off[w] + (i - lo);
                if (slot < n) t.qn[slot] = st.near_buf[w * NEAR_REGION + i];
                else atomicOr(err, ERR_CAPACITY);
            }
        }
        const uint32_t nb = min(st.band_n[w], BAND_REGION);
        if (nb) {
            uint32_t base = 0;
            if (lane_id() == 0) base = atomicAdd(t.band_count, nb);
            base = __shfl_sync(FULL, base, 0);
            for (uint32_t i = lane_id(); i < nb; i += 32) {
                if (base + i < n) t.bandq[base + i] = st.band_buf[w * BAND_REGION + i];
                else atomicOr(err, ERR_CAPACITY);
            }
        }
    }
    for (uint32_t i = threadIdx.x; i < nf; i += blockDim.x) {
        uint32_t slot = st.base_far + i;
        if (slot < n) t.farq[slot] = st.far_buf[i];
        else atomicOr(err, ERR_CAPACITY);
    }
}

// Near appends: high-degree vertices become CHUNK-arc items of the heavy
// queue (per-lane atomics; rare), the rest go through the staging buffer.
__device__ __forceinline__ void push_near(const SsspArgs &a, Stage &st, const PushTargets &t,
                                          bool want, uint32_t v, uint32_t deg) {
    bool heavy = want && deg >= HEAVY_DEG;
    const uint32_t w = threadIdx.x >> 5;
    region_append(want && !heavy, v, st.near_buf + w * NEAR_REGION, &st.near_n[w], NEAR_REGION,
                  t.flush, t.qn, t.qn_count, a.n, &a.ctl->err,
                  t.nostamp ? a.stamp_near : nullptr, t.tag_next);
    if (heavy) {
        uint32_t nc = (deg + CHUNK - 1) / CHUNK;
        uint32_t base = atomicAdd(t.hqn_count, nc);
        if (base + nc > a.heavy_cap) {
            atomicOr(&a.ctl->err, ERR_CAPACITY);
        } else {
            for (uint32_t c = 0; c < nc; ++c) t.hqn[base + c] = ((uint64_t)v << 32) | c;
        }
    }
}

// Far appends: `want` appends v to the pile (first time this phase);
// `cand` marks every far proposal, so far_min bounds the pile from below
// even for vertices already in it.
__device__ __forceinline__ void push_far(const SsspArgs &a, Stage &st, const PushTargets &t,
                                         bool want, bool cand, uint32_t v, uint32_t d) {
    stage_append(want, v, st.far_buf, &st.far_n, FAR_STAGE, t.farq, t.far_count, a.n, &a.ctl->err);
    if (__any_sync(FULL, cand)) {
        uint32_t m = cand ? d : INF32;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) m = min(m, __shfl_xor_sync(FULL, m, o));
        if (lane_id() == 0 && m != INF32) atomicMin(&st.far_min, m);
    }
}

// Label of v in the 64-bit form (read past L1: other blocks write it).
template <bool NARROW>
__device__ __forceinline__ uint64_t sssp_label(const SsspArgs &a, uint32_t v) {
    if (NARROW) return widen_label(ldcg_u32(&a.label32[v]), a.lshift);
    return ldcg_u64(&a.label[v]);
}

// Relaxes up to ILP arcs per lane.  For arc u of this lane: valid[u], the
// arc index and the tail's label; only arcs with wlo <= weight < whi are
// relaxed.  The loads and atomics of the ILP arcs are issued back to back
// so their latencies overlap.
// With `precheck` a plain load of the head's label comes first and only
// improving proposals issue the atomic: right for thick frontiers, where
// L2 atomic throughput is the limit; thin frontiers are latency-bound and
// skip the extra dependent load.
// The tail labels lab[] are in the 64-bit form; NARROW kernels keep the
// head labels in 32 bits and flag (narrow_miss) any proposal whose distance
// does not fit one, which the host answers with a 64-bit rerun.
template <bool NARROW>
__device__ __forceinline__ void relax_group(const SsspArgs &a, Stage &st, const PushTargets &t,
                                            const bool (&valid)[ILP], const uint32_t (&arc)[ILP],
                                            const uint64_t (&lab)[ILP], bool precheck,
                                            bool stream, uint32_t wlo, uint32_t whi,
                                            unsigned long long &attempts,
                                            unsigned long long &improved, bool &narrow_miss,
                                            unsigned long long &atomics) {
    uint2 e[ILP];
#pragma unroll
    for (int u = 0; u < ILP; ++u) {
        e[u] = make_uint2(0, 0);
        // heavy-row chunks are streamed (evict first); short rows may be
        // re-read by later hops and stay cacheable
        if (valid[u]) e[u] = stream ? __ldcs(&a.adj[arc[u]]) : __ldg(&a.adj[arc[u]]);
    }
    uint64_t nd[ILP];
    bool imp[ILP], fr[ILP];
#pragma unroll
    for (int u = 0; u < ILP; ++u) {
        imp[u] = fr[u] = false;
        nd[u] = INF32;
        if (valid[u] && e[u].y >= wlo && e[u].y < whi) {
            ++attempts;
            nd[u] = (lab[u] >> 32) + (uint64_t)e[u].y;
            if (NARROW) {
                if (nd[u] > a.ldmax) {
                    narrow_miss = true;
                } else {
                    const uint32_t nl = ((uint32_t)nd[u] << a.lshift) | (uint32_t)lab[u];
                    if (!precheck || nl < ldcg_u32(&a.label32[e[u].x])) {
                        ++atomics;
                        if (a.far_scan && nd[u] >= t.T) {
                            // a far proposal needs no answer (nothing is queued
                            // for it): a fire-and-forget reduction
                            atomicMin(&a.label32[e[u].x], nl);
                            fr[u] = true;
                        } else {
                            const uint32_t old = atomicMin(&a.label32[e[u].x], nl);
                            imp[u] = nl < old;
                        }
                    }
                }
            } else if (nd[u] < INF32) {
                // proposals at or above 2^32 - 1 are skipped; the scan reports the overflow
                uint64_t nl = (nd[u] << 32) | (lab[u] & 0xFFFFFFFFull);
                if (!precheck || nl < ldcg_u64(&a.label[e[u].x])) {
                    ++atomics;
                    if (a.far_scan && nd[u] >= t.T) {
                        atomicMin(reinterpret_cast<unsigned long long *>(&a.label[e[u].x]),
                                  (unsigned long long)nl);
                        fr[u] = true;
                    } else {
                        uint64_t old = atomicMin(reinterpret_cast<unsigned long long *>(&a.label[e[u].x]),
                                                 (unsigned long long)nl);
                        imp[u] = nl < old;
                    }
                }
            }
        }
    }
    // rounds that improve nothing skip the append machinery
    if (!__any_sync(FULL, imp[0] | imp[1] | imp[2] | imp[3] | fr[0] | fr[1] | fr[2] | fr[3])) return;
    bool to_near[ILP], to_far[ILP], cand[ILP], dn[ILP];
    uint32_t deg[ILP];
#pragma unroll
    for (int u = 0; u < ILP; ++u) {
        to_near[u] = to_far[u] = dn[u] = false;
        cand[u] = fr[u];         // a fire-and-forget far proposal still bounds far_min
        deg[u] = 0;
        if (!imp[u]) continue;
        ++improved;
        uint32_t v = e[u].x;
        if (nd[u] < t.T && t.dense) {
            // a light vertex sets its bit; a possible hub (id below n_big)
            // reads its degree first and, if it is one, joins the chunk queue
            if (v < a.n_big) {
                const uint32_t r0 = a.row_ptr[v];
                deg[u] = (t.lend ? t.lend[v] : a.row_ptr[v + 1]) - r0;
            }
            if (deg[u] >= HEAVY_DEG) {
                to_near[u] = atomicExch(&a.stamp_near[v], t.tag_next) != t.tag_next;
            } else {
                atomicOr(&t.nbm[v >> 5], 1u << (v & 31));
                dn[u] = true;
            }
        } else if (nd[u] < t.T && t.nostamp) {
            // ids at or above n_big cannot be hubs: no look at the row
            if (v < a.n_big) {
                const uint32_t r0 = a.row_ptr[v];
                deg[u] = (t.lend ? t.lend[v] : a.row_ptr[v + 1]) - r0;
            }
            to_near[u] = deg[u] < HEAVY_DEG ||     // hubs join the chunk queue once
                         atomicExch(&a.stamp_near[v], t.tag_next) != t.tag_next;
        } else if (nd[u] < t.T) {
            uint32_t r0 = a.row_ptr[v];                           // independent of the exchange
            uint32_t r1 = t.lend ? t.lend[v] : a.row_ptr[v + 1];  // end of the part relaxed near
            to_near[u] = atomicExch(&a.stamp_near[v], t.tag_next) != t.tag_next;
            deg[u] = r1 - r0;
        } else {
            cand[u] = true;      // bounds far_min
            // with the far scan, the split finds far vertices by their labels
            if (!a.far_scan) to_far[u] = atomicExch(&a.stamp_far[v], t.tag_far) != t.tag_far;
        }
    }
#pragma unroll
    for (int u = 0; u < ILP; ++u) {
        push_near(a, st, t, to_near[u], e[u].x, deg[u]);
        push_far(a, st, t, to_far[u], cand[u], e[u].x, (uint32_t)nd[u]);
    }
    if (t.dense) {
        uint32_t c = 0;
#pragma unroll
        for (int u = 0; u < ILP; ++u) c += (uint32_t)__popc(__ballot_sync(FULL, dn[u]));
        if (lane_id() == 0 && c) st.dn_near[threadIdx.x >> 5] += c;
    }
}

// Lists vertex u (lanes with `want`; hdeg arcs in its heavy part) in the
// current band once: as one item, or as CHUNK-arc pieces when the heavy
// part is long.  A vertex without heavy arcs needs no listing.
__device__ __forceinline__ void band_track(const SsspArgs &a, Stage &st, bool want, uint32_t u,
                                           uint32_t hdeg, uint32_t tag) {
    uint32_t listed = 0;     // heavy arcs this lane lists
    if (a.dense) {
        // dense band list: a bit per listed vertex (the pass reads the
        // bitmap), so only the hubs need the stamp that lists them once
        const bool small = want && hdeg > 0 && hdeg < HEAVY_DEG;
        if (small) atomicOr(&a.bbm[u >> 5], 1u << (u & 31));
        const uint32_t c = (uint32_t)__popc(__ballot_sync(FULL, small));
        if (lane_id() == 0 && c) st.dn_band[threadIdx.x >> 5] += c;
        if (small) listed = hdeg;
        want = want && hdeg >= HEAVY_DEG;
    }
    bool add = want && hdeg > 0 && atomicExch(&a.stamp_band[u], tag) != tag;
    const bool big = add && hdeg >= HEAVY_DEG;
    const uint32_t w = threadIdx.x >> 5;
    if (add) listed = hdeg;
    listed = __reduce_add_sync(FULL, listed);
    if (lane_id() == 0 && listed) st.hs[w] += listed;
    region_append(add && !big, u, st.band_buf + w * BAND_REGION, &st.band_n[w], BAND_REGION, true,
                  a.band_q, &a.ctl->band_count, a.n, &a.ctl->err);
    if (big) {
        const uint32_t nc = (hdeg + CHUNK - 1) / CHUNK;
        const uint32_t base = atomicAdd(&a.ctl->band_hcount, nc);
        if (base + nc > a.heavy_cap || base + nc < base) {
            atomicOr(&a.ctl->err, ERR_CAPACITY);
        } else {
            for (uint32_t c = 0; c < nc; ++c) a.band_hq[base + c] = ((uint64_t)u << 32) | c;
        }
    }
}

// Lists high-degree vertex u (warp-uniform; deg arcs in its heavy part) in
// the current band once, as its CHUNK-arc pieces.
__device__ __forceinline__ void band_track_heavy(const SsspArgs &a, Stage &st, uint32_t u,
                                                 uint32_t deg, uint32_t tag) {
    const uint32_t lane = lane_id();
    if (deg == 0) return;
    uint32_t add = 0;
    if (lane == 0) add = atomicExch(&a.stamp_band[u], tag) != tag;
    if (!__shfl_sync(FULL, add, 0)) return;
    if (lane == 0) st.hs[threadIdx.x >> 5] += deg;
    const uint32_t nc = (deg + CHUNK - 1) / CHUNK;
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&a.ctl->band_hcount, nc);
    base = __shfl_sync(FULL, base, 0);
    if (base + nc > a.heavy_cap || base + nc < base) {
        if (lane == 0) atomicOr(&a.ctl->err, ERR_CAPACITY);
        return;
    }
    for (uint32_t c = lane; c < nc; c += 32) a.band_hq[base + c] = ((uint64_t)u << 32) | c;
}

// Relaxes the arcs of up to 32 frontier vertices, one per lane (has, u),
// flattened over the lanes: their light parts (their heavy parts in a
// band's closing pass, hp), listing them for the band when tracked.
template <bool NARROW>
__device__ __forceinline__ void relax_vertices(const SsspArgs &a, Stage &st, const PushTargets &t,
                                               bool has, uint32_t u, bool hp, bool track,
                                               uint32_t tag_band, uint32_t wlo, uint32_t whi,
                                               bool precheck, unsigned long long &attempts,
                                               unsigned long long &improved, bool &narrow_miss,
                                               unsigned long long &atomics) {
    const uint32_t lane = lane_id();
    uint32_t s = 0, deg = 0, hdeg = 0;
    uint64_t lab = INF64;
    if (has) {
        const uint32_t r0 = a.row_ptr[u], r1 = a.row_ptr[u + 1];
        const uint32_t le = t.lend ? t.lend[u] : r1;
        if (hp) {                       // the heavy part (or the whole row)
            s = t.lend ? le : r0;
            deg = r1 - s;
        } else {                        // the light part
            s = r0;
            deg = le - r0;
            hdeg = t.lend ? r1 - le : r1 - r0;
        }
        lab = sssp_label<NARROW>(a, u);
        if (lab == INF64) deg = 0;
    }
    if (track) band_track(a, st, has, u, hdeg, tag_band);
    const uint32_t incl = warp_inclusive_scan(deg);
    const uint32_t excl = incl - deg;
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    for (uint32_t b = 0; b < total; b += 32 * ILP) {
        bool valid[ILP];
        uint32_t arc[ILP];
        uint64_t labs[ILP];
#pragma unroll
        for (int q = 0; q < ILP; ++q) {
            const uint32_t j = b + lane + 32 * q;
            valid[q] = j < total;
            const uint32_t owner = warp_owner_search(excl, valid[q] ? j : 0);
            const uint32_t so = __shfl_sync(FULL, s, owner);
            const uint32_t eo = __shfl_sync(FULL, excl, owner);
            labs[q] = __shfl_sync(FULL, lab, owner);
            arc[q] = so + (j - eo);
        }
        relax_group<NARROW>(a, st, t, valid, arc, labs, precheck, false, wlo, whi, attempts,
                            improved, narrow_miss, atomics);
    }
}

// Index of the t-th set bit (0-based) of a 32-bit word.
__device__ __forceinline__ uint32_t nth_set_bit(uint32_t x, uint32_t t) {
    uint32_t pos = 0;
#pragma unroll
    for (uint32_t w = 16; w >= 1; w >>= 1) {
        const uint32_t c = (uint32_t)__popc(x & ((1u << w) - 1u));
        if (t >= c) {
            t -= c;
            x >>= w;
            pos += w;
        }
    }
    return pos;
}

// Pull form of a band's heavy-arc pass (threshold T, every label below T
// final).  Warps sweep the vertex ids 32 at a time (coalesced labels), or
// the candidate list; a vertex at or above T (unreached included) reads
// the arcs of its heavy part, flattened over the warp, and the labels at
// their other ends.  The best proposal (d(u) + w, rank(u)) from a settled
// neighbour u is gathered per vertex in shared memory (pmin: one slot per
// vertex of the warp's step) and, if it beats the vertex's label, sent as
// one fire-and-forget atomicMin; it bounds far_min as a far push proposal
// does.  The sweep also clears the band bitmap that the push form would
// have read.  The warps' sums of the heavy arcs met go to st.hs (the pass's
// cost).
// `out` (sweep of every id, no tail): the unsettled vertices with arcs are
// listed there, the candidates of the split that follows.
// `tail`: the pass starts the unbounded tail band: every unsettled vertex
// whose label is now finite joins the next frontier (t), with its whole row.
template <bool NARROW>
__device__ __noinline__ void pull_pass(const SsspArgs &a, Stage &st,
                                       unsigned long long (*pmin)[32 * PULL_ILP], uint64_t T,
                                       const uint32_t *list, uint32_t count, uint32_t *out,
                                       uint32_t *out_count, bool tail, uint32_t *nbm,
                                       uint32_t *qn, uint32_t *qn_count, uint64_t *hqn,
                                       uint32_t *hqn_count, unsigned long long &attempts,
                                       unsigned long long &improved, bool &narrow_miss,
                                       unsigned long long &atomics) {
    const uint32_t lane = lane_id();
    const uint32_t wib = threadIdx.x >> 5;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    unsigned long long *pm = pmin[wib];
    // where the tail's first frontier goes (light vertices as bits when dense)
    PushTargets t;
    t.qn = qn;
    t.qn_count = qn_count;
    t.hqn = hqn;
    t.hqn_count = hqn_count;
    t.flush = true;
    t.dense = a.dense != 0;
    t.nbm = nbm;
    t.nostamp = false;
    t.nostamp_stamp = nullptr;
    t.tag_next = 0;
    t.hsum = nullptr;
    t.lend = nullptr;
    uint32_t met = 0;
    uint32_t fmin = INF32;
    // the vertices: every id, or the candidate list (then the band bitmap
    // is cleared by a sweep of its own)
    if (list && a.dense)
        for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n_words;
             i += gridDim.x * blockDim.x)
            if (ldcg_u32(&a.bbm[i])) a.bbm[i] = 0;
    const uint32_t nv = list ? count : a.n;
    // PULL_ILP chunks of 32 vertices per warp step, their loads issued together
    for (uint32_t b = warp * 32 * PULL_ILP; b < nv; b += nwarps * 32 * PULL_ILP) {
        if (!list && a.dense && lane < PULL_ILP && (b >> 5) + lane < a.n_words &&
            ldcg_u32(&a.bbm[(b >> 5) + lane]))
            a.bbm[(b >> 5) + lane] = 0;
        uint32_t vs[PULL_ILP];
        uint64_t lab[PULL_ILP];
        uint32_t s[PULL_ILP], r1[PULL_ILP], r0[PULL_ILP];
#pragma unroll
        for (int c = 0; c < PULL_ILP; ++c) {
            const uint32_t i = b + 32u * c + lane;
            vs[c] = i < nv ? (list ? ldcg_u32(&list[i]) : i) : INF32;
            pm[32 * c + lane] = INF64;
        }
#pragma unroll
        for (int c = 0; c < PULL_ILP; ++c)    // past the end: taken as settled
            lab[c] = vs[c] != INF32 ? sssp_label<NARROW>(a, vs[c]) : 0ull;
        bool uns[PULL_ILP];
#pragma unroll
        for (int c = 0; c < PULL_ILP; ++c) {
            const uint32_t v = vs[c];
            s[c] = r1[c] = r0[c] = 0;
            uns[c] = lab[c] == INF64 || (lab[c] >> 32) >= T;
            if (uns[c]) {
                r1[c] = a.row_ptr[v + 1];
                r0[c] = a.row_ptr[v];
                s[c] = a.lend ? a.lend[v] : r0[c];
            }
        }
        if (out) {
            // the sweep over every id lists the unsettled vertices with arcs
            // (the candidates of the split that follows), staged in the band
            // regions, which a heavy-arc pass does not use
#pragma unroll
            for (int c = 0; c < PULL_ILP; ++c)
                region_append(uns[c] && r1[c] != r0[c], vs[c], st.band_buf + wib * BAND_REGION,
                              &st.band_n[wib], BAND_REGION, true, out, out_count, a.n,
                              &a.ctl->err);
        }
        __syncwarp();
#pragma unroll
        for (int c = 0; c < PULL_ILP; ++c) {
            const uint32_t deg = r1[c] - s[c];
            met += deg;
            const uint32_t incl = warp_inclusive_scan(deg);
            const uint32_t excl = incl - deg;
            const uint32_t total = __shfl_sync(FULL, incl, 31);
            for (uint32_t j0 = 0; j0 < total; j0 += 32 * ILP) {
                bool valid[ILP];
                uint32_t slot[ILP];
                uint64_t hl[ILP];
                uint2 e[ILP];
#pragma unroll
                for (int q = 0; q < ILP; ++q) {
                    const uint32_t j = j0 + lane + 32 * q;
                    valid[q] = j < total;
                    const uint32_t owner = warp_owner_search(excl, valid[q] ? j : 0);
                    const uint32_t so = __shfl_sync(FULL, s[c], owner);
                    const uint32_t eo = __shfl_sync(FULL, excl, owner);
                    hl[q] = __shfl_sync(FULL, lab[c], owner);
                    slot[q] = 32u * c + owner;
                    e[q] = make_uint2(0, 0);
                    // the unsettled rows are read once per pass: streamed
                    if (valid[q]) e[q] = __ldcs(&a.adj[so + (j - eo)]);
                }
                uint64_t tl[ILP];
#pragma unroll
                for (int q = 0; q < ILP; ++q) {
                    tl[q] = INF64;
                    if (valid[q] && e[q].y >= a.delta) tl[q] = sssp_label<NARROW>(a, e[q].x);
                }
#pragma unroll
                for (int q = 0; q < ILP; ++q) {
                    // an unsettled (or unreached) neighbour proposes nothing yet
                    if (!valid[q] || tl[q] == INF64 || (tl[q] >> 32) >= T) continue;
                    ++attempts;
                    const uint64_t nd = (tl[q] >> 32) + (uint64_t)e[q].y;
                    if (NARROW && nd > a.ldmax) {
                        // only an unreached vertex could take it (a narrow
                        // label's distance is at most ldmax): the host
                        // reruns the query with 64-bit labels
                        if (hl[q] == INF64) narrow_miss = true;
                        continue;
                    }
                    if (nd >= INF32) continue;         // the scan reports the overflow
                    const uint64_t nl64 = (nd << 32) | (tl[q] & 0xFFFFFFFFull);
                    if (nl64 < hl[q]) atomicMin(&pm[slot[q]], (unsigned long long)nl64);
                }
            }
        }
        __syncwarp();
        // each lane settles its own vertices: one atomic per improved one
#pragma unroll
        for (int c = 0; c < PULL_ILP; ++c) {
            const uint64_t best = pm[32 * c + lane];
            uint64_t now = lab[c];
            if (uns[c] && best < lab[c]) {
                if (NARROW)
                    atomicMin(&a.label32[vs[c]],
                              ((uint32_t)(best >> 32) << a.lshift) | (uint32_t)best);
                else
                    atomicMin(reinterpret_cast<unsigned long long *>(&a.label[vs[c]]),
                              (unsigned long long)best);
                ++atomics;
                ++improved;
                fmin = min(fmin, (uint32_t)(best >> 32));
                now = best;
            }
            if (tail) {
                // reached and unsettled: the tail's first frontier, whole rows
                const bool want = uns[c] && now != INF64 && r1[c] != r0[c];
                const uint32_t deg = r1[c] - r0[c];
                const bool bit = t.dense && want && deg < HEAVY_DEG;
                const uint32_t word = __ballot_sync(FULL, bit);
                if (!list) {
                    if (lane == 0 && word) t.nbm[(b + 32u * c) >> 5] = word;
                } else if (bit) {
                    atomicOr(&t.nbm[vs[c] >> 5], 1u << (vs[c] & 31));
                }
                if (lane == 0 && word) st.dn_near[wib] += (uint32_t)__popc(word);
                push_near(a, st, t, want && !bit, vs[c], deg);
            }
        }
        __syncwarp();
    }
    met = __reduce_add_sync(FULL, met);
    fmin = __reduce_min_sync(FULL, fmin);
    if (lane == 0) {
        st.hs[wib] += met;
        if (fmin != INF32) atomicMin(&st.far_min, fmin);
    }
}

// ---------------------------------------------------------------------------
// the persistent near/far kernel
// ---------------------------------------------------------------------------

template <bool NARROW>
__global__ void __launch_bounds__(256, 3) sssp_kernel(SsspArgs a) {
    __shared__ Stage st;
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    Control *ctl = a.ctl;
    unsigned long long attempts = 0, improved = 0;
    bool narrow_miss = false;
    unsigned long long atomics = 0;
    // trace: each warp's counter sums at the start of the iteration (lane 0
    // keeps them in shared memory, off the registers of the hot loops)
    __shared__ unsigned long long trace_snap[SSSP_WARPS][4];
    if (threadIdx.x < SSSP_WARPS * 4) (&trace_snap[0][0])[threadIdx.x] = 0;
    uint32_t it = 0, phase = 0, bands = 0;
    uint64_t T = a.delta;
    bool first = (blockIdx.x == 0 && threadIdx.x == 0);
    bool hp = false;               // this iteration is a band's heavy-arc pass
    bool pull = false;             // ... in the pull form
    // With the far scan, the first split lists every vertex left unsettled
    // (those with arcs); later splits and pull passes visit that list,
    // which each split shrinks, instead of every id.
    bool listed = false;
    // Tail: after a band whose heavy-arc pass ran in the pull form (it
    // settled most of the graph's heavy arcs), the rest runs as one
    // unbounded band, a frontier Bellman-Ford over whole rows: on a
    // small-world graph the unsettled vertices hang off the settled core
    // by short chains, and a few iterations reach the fixed point that a
    // band per delta would approach in many splits.
    bool tail = false;
    __shared__ unsigned long long pmin[SSSP_WARPS][32 * PULL_ILP];   // pull pass minima
    // heavy arcs a pull pass would read now, bounded from above: all arcs
    // at first, then what the last pull pass met (the unsettled set only
    // shrinks)
    __shared__ unsigned long long pull_bound;
    if (threadIdx.x == 0) pull_bound = a.m;
    bool cur_dense = false;        // this iteration's light items are the bits of a near bitmap

    for (;;) {
        const uint32_t cs = it % 3, ns = (it + 1) % 3;
        uint32_t n_light, n_heavy;
        if (hp) {
            n_light = min(ldcg_u32(&ctl->band_count), a.n);
            n_heavy = min(ldcg_u32(&ctl->band_hcount), a.heavy_cap);
        } else {
            n_light = min(ldcg_u32(&ctl->near_count[cs]), a.n);
            n_heavy = min(ldcg_u32(&ctl->heavy_count[cs]), a.heavy_cap);
        }
        if (first) {
            ctl->near_count[(it + 2) % 3] = 0;
            ctl->heavy_count[(it + 2) % 3] = 0;
            if (hp && pull) ++ctl->pulls;
            if (it < TRACE_LEN) {
                ctl->trace[it][0] = n_light;
                ctl->trace[it][1] = n_heavy;
                ctl->trace[it][2] = ldcg_u32(&ctl->far_count[phase & 1]);
                ctl->trace[it][3] = (uint32_t)T;
                ctl->trace_ns[it] = global_ns();
            }
        }
        stage_reset(st);
        const bool odd = it & 1;
        const uint32_t *qc = hp ? a.band_q : (odd ? a.q1 : a.q0);
        const uint64_t *hqc = hp ? a.band_hq : (odd ? a.hq1 : a.hq0);
        const uint32_t fc = phase & 1;
        PushTargets t;
        t.qn = odd ? a.q0 : a.q1;
        t.qn_count = &ctl->near_count[ns];
        t.hqn = odd ? a.hq0 : a.hq1;
        t.hqn_count = &ctl->heavy_count[ns];
        t.farq = fc ? a.far1 : a.far0;
        t.far_count = &ctl->far_count[fc];
        t.far_min = &ctl->far_min[fc];
        t.bandq = a.band_q;
        t.band_count = &ctl->band_count;
        t.tag_next = a.base_near + it + 1;
        t.tag_far = a.base_far + phase;
        t.T = T;
        t.flush = true;
        // dense in: light items from this iteration's near bitmap (or, in a
        // dense heavy-arc pass, the band bitmap); dense out: a large
        // frontier (a fraction of the graph, or many hub chunks) pushes its
        // light vertices as bits for the next iteration.  Every block reads
        // the same counts, so all agree.
        const bool dense_in = hp ? a.dense != 0 : cur_dense;
        const bool push_dense =
            a.dense && !hp && (n_light >= a.n / 128 || n_heavy >= a.n / 4096);
        uint32_t *bm_in = hp ? a.bbm : ((it & 1) ? a.nbm1 : a.nbm0);
        t.dense = push_dense;
        t.nbm = (it & 1) ? a.nbm0 : a.nbm1;
        t.nostamp = a.local_rounds != 0 && !hp;
        t.nostamp_stamp = a.stamp_near;
        // arcs relaxed by this iteration: all; light ones while a band
        // iterates under the split; heavy ones in the band's closing pass
        // (in the tail every relaxation covers whole rows)
        const uint32_t wlo = hp ? a.delta : 0u;
        const uint32_t whi = (a.defer && !hp && !tail) ? a.delta : 0xFFFFFFFFu;
        const bool track = a.defer && !hp && !tail;
        t.lend = tail ? nullptr : a.lend;
        const uint32_t tag_band = a.base_band + bands;
        t.hsum = track ? &ctl->band_hsum : (hp && pull ? &ctl->pull_hsum : nullptr);

        // Vertices per warp batch: a thin frontier is spread over all warps
        // (fewer sequential rounds per warp), a thick one packs 32 per warp.
        uint32_t per = (n_light + nwarps - 1) / nwarps;
        uint32_t bsz = per <= 1 ? 1 : per <= 2 ? 2 : per <= 4 ? 4 : per <= 8 ? 8 : per <= 16 ? 16 : 32;
        // A dense work item is one bitmap word (32 vertices) where vertices
        // may have many arcs (ids below n_big, in the degree order the high
        // degrees), else DENSE_WORDS words: balanced work per warp.  A
        // sparse bitmap (under one set bit per two words) is read 32 words
        // per item: the sweep itself is then the cost.
        const uint32_t cw = n_light < a.n_words / 2 ? 32u : hp ? DENSE_WORDS_HP : DENSE_WORDS;
        const uint32_t fine = min(a.n_words, (a.n_big + 1023) / 1024 * 32);
        const uint32_t n_work = n_heavy + (dense_in ? fine + (a.n_words - fine + cw - 1) / cw
                                                    : (n_light + bsz - 1) / bsz);
        if (a.trace && lane == 0) trace_snap[threadIdx.x >> 5][3] = global_ns();
        if (hp && pull) {
            // without a list yet, the pass sweeps every id and lists the
            // unsettled ones as this phase's pile (empty with the far scan)
            uint32_t *pile = fc ? a.far1 : a.far0;
            t.bandq = pile;
            t.band_count = &ctl->far_count[fc];
            // with the tail to follow, the pass pushes its first frontier
            pull_pass<NARROW>(a, st, pmin, T, listed ? pile : nullptr,
                              listed ? min(ldcg_u32(&ctl->far_count[fc]), a.n) : a.n,
                              (listed || a.tail) ? nullptr : pile, &ctl->far_count[fc],
                              a.tail != 0, t.nbm, t.qn, t.qn_count, t.hqn, t.hqn_count,
                              attempts, improved, narrow_miss, atomics);
        } else
        for (uint32_t wi = warp; wi < n_work; wi += nwarps) {
            if (wi < n_heavy) {
                // one CHUNK of a high-degree vertex per warp
                uint64_t item = __ldcg(reinterpret_cast<const unsigned long long *>(&hqc[wi]));
                uint32_t u = (uint32_t)(item >> 32), c = (uint32_t)item;
                uint32_t r0 = a.row_ptr[u], r1 = a.row_ptr[u + 1];
                const uint32_t le = t.lend ? t.lend[u] : r1;      // light part [r0, le)
                // a band's heavy pass covers the heavy part, else the light one
                const uint32_t base = hp && t.lend ? le : r0, end = hp ? r1 : le;
                uint32_t s = base + c * CHUNK;
                uint32_t e = min(end, s + CHUNK);
                uint64_t lab = sssp_label<NARROW>(a, u);
                if (track && c == 0) band_track_heavy(a, st, u, t.lend ? r1 - le : r1 - r0, tag_band);
                for (uint32_t b = s; b < e; b += 32 * ILP) {
                    bool valid[ILP];
                    uint32_t arc[ILP];
                    uint64_t labs[ILP];
#pragma unroll
                    for (int q = 0; q < ILP; ++q) {
                        arc[q] = b + lane + 32 * q;
                        valid[q] = arc[q] < e;
                        labs[q] = lab;
                    }
                    relax_group<NARROW>(a, st, t, valid, arc, labs, true, true, wlo, whi, attempts,
                                improved, narrow_miss, atomics);
                }
            } else if (dense_in) {
                // 1 or 32 words of the bitmap, one per lane (read and
                // cleared); their set bits, 32 at a time, are the vertices
                const uint32_t di = wi - n_heavy;
                const uint32_t w0 = di < fine ? di : fine + (di - fine) * cw;
                const uint32_t nw = di < fine ? 1u : cw;
                uint32_t word = 0;
                if (lane < nw && w0 + lane < a.n_words) {
                    word = ldcg_u32(&bm_in[w0 + lane]);
                    if (word) bm_in[w0 + lane] = 0;
                }
                const uint32_t cnt = (uint32_t)__popc(word);
                const uint32_t incl = warp_inclusive_scan(cnt);
                const uint32_t excl = incl - cnt;
                const uint32_t total = __shfl_sync(FULL, incl, 31);
                for (uint32_t b = 0; b < total; b += 32) {
                    const uint32_t j = b + lane;
                    const bool has = j < total;
                    const uint32_t owner = warp_owner_search(excl, has ? j : 0);
                    const uint32_t wo = __shfl_sync(FULL, word, owner);
                    const uint32_t eo = __shfl_sync(FULL, excl, owner);
                    const uint32_t u = has ? (w0 + owner) * 32 + nth_set_bit(wo, j - eo) : 0;
                    relax_vertices<NARROW>(a, st, t, has, u, hp, track, tag_band, wlo, whi, true,
                                           attempts, improved, narrow_miss, atomics);
                }
            } else {
                // bsz frontier vertices per warp, their arcs flattened over the lanes
                const uint32_t i = (wi - n_heavy) * bsz + lane;
                const bool has = lane < bsz && i < n_light;
                const uint32_t u = has ? ldcg_u32(&qc[i]) : 0;
                relax_vertices<NARROW>(a, st, t, has, u, hp, track, tag_band, wlo, whi, bsz == 32,
                                       attempts, improved, narrow_miss, atomics);
            }
        }
        // Local rounds: relax the vertices just staged for the next
        // iteration right away, a hop further per round, instead of waiting
        // for the grid barrier; what is left is flushed.  (A heavy-arc pass
        // stages nothing near.)
        if (a.local_rounds && !hp) {
            // Warp-local rounds: each warp relaxes the vertices it staged
            // itself, a hop per round, with no block barrier between hops.
            const uint32_t wib = threadIdx.x >> 5;
            t.flush = false;            // the loop below indexes into the region
            uint32_t *region = st.near_buf + wib * NEAR_REGION;
            uint32_t lo = 0;
            for (uint32_t r = 0; r < a.local_rounds; ++r) {
                __syncwarp();
                const uint32_t hi = min(*(volatile uint32_t *)&st.near_n[wib], NEAR_REGION);
                if (lo >= hi) break;
                for (uint32_t b0 = lo; b0 < hi; b0 += 32) {
                    const uint32_t i = b0 + lane;
                    const bool has = i < hi;
                    uint32_t s = 0, deg = 0, u = 0, hdeg = 0;
                    uint64_t lab = INF64;
                    if (has) {
                        u = region[i];
                        // row offsets and the label in one round trip: every
                        // later improvement of u appends u again (to the
                        // improving warp's region), so the current label is
                        // all a round needs
                        s = a.row_ptr[u];
                        const uint32_t r1 = a.row_ptr[u + 1];
                        const uint32_t le = t.lend ? t.lend[u] : r1;
                        deg = le - s;
                        hdeg = t.lend ? r1 - le : r1 - s;
                        lab = sssp_label<NARROW>(a, u);
                    }
                    if (track) band_track(a, st, has, u, hdeg, tag_band);
                    uint32_t incl = warp_inclusive_scan(deg);
                    uint32_t excl = incl - deg;
                    uint32_t total = __shfl_sync(FULL, incl, 31);
                    for (uint32_t b = 0; b < total; b += 32 * ILP) {
                        bool valid[ILP];
                        uint32_t arc[ILP];
                        uint64_t labs[ILP];
#pragma unroll
                        for (int q = 0; q < ILP; ++q) {
                            uint32_t j = b + lane + 32 * q;
                            valid[q] = j < total;
                            uint32_t owner = warp_owner_search(excl, valid[q] ? j : 0);
                            uint32_t so = __shfl_sync(FULL, s, owner);
                            uint32_t eo = __shfl_sync(FULL, excl, owner);
                            labs[q] = __shfl_sync(FULL, lab, owner);
                            arc[q] = so + (j - eo);
                        }
                        relax_group<NARROW>(a, st, t, valid, arc, labs, false, false, wlo, whi,
                                    attempts, improved, narrow_miss, atomics);
                    }
                }
                lo = hi;
            }
            if (lane == 0) st.local_lo[wib] = lo;
        }
        if (a.trace && it < TRACE_LEN) {
            // per warp: busy time of this iteration's relaxation (sum, max)
            unsigned long long da = attempts, di = improved, dm = atomics;
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                da += __shfl_xor_sync(FULL, da, o);
                di += __shfl_xor_sync(FULL, di, o);
                dm += __shfl_xor_sync(FULL, dm, o);
            }
            if (lane == 0) {
                unsigned long long *snap = trace_snap[threadIdx.x >> 5];
                const unsigned long long busy = global_ns() - snap[3];
                const unsigned long long sa = da, si = di, sm = dm;
                da -= snap[0];
                di -= snap[1];
                dm -= snap[2];
                snap[0] = sa;
                snap[1] = si;
                snap[2] = sm;
                if (da | di) {
                    atomicAdd(&ctl->trace_relax[it][0], da);
                    atomicAdd(&ctl->trace_relax[it][1], di);
                    atomicAdd(&ctl->trace_relax[it][2], dm);
                }
                atomicAdd(&ctl->trace_busy[it][0], busy);
                atomicMax(&ctl->trace_busy[it][1], busy);
            }
        }
        flush_stage(st, t, a.n, &ctl->err);
        if (!grid_sync(&ctl->bar, &ctl->err)) {
            if (first) ctl->exit_reason = 3;
            break;
        }
        // a pull pass that starts the tail set its frontier's bits (dense)
        cur_dense = (hp && pull && a.tail) ? a.dense != 0 : push_dense;
        ++it;
        const bool was_hp = hp;
        if (hp) {
            ++bands;               // later listings use a fresh tag
            hp = false;
            if (pull && a.tail) {
                // the tail band: no threshold, whole rows, no more splits
                tail = true;
                T = INF32;
                if (first) ctl->tail_it = it;
            }
            if (pull) {
                // every thread has read pull_bound at the decision, a
                // barrier ago; one writes the new bound, read at the next
                if (threadIdx.x == 0)
                    pull_bound = ldcg_u64(reinterpret_cast<const uint64_t *>(&ctl->pull_hsum));
                listed = true;     // the pass listed the candidates (or used the list)
            }
            pull = false;
        }
        if (it >= a.max_iters) {
            if (first) {
                atomicOr(&ctl->err, ERR_TIMEOUT);
                ctl->exit_reason = 2;
            }
            break;
        }
        uint32_t next = ldcg_u32(&ctl->near_count[ns]) + ldcg_u32(&ctl->heavy_count[ns]);
        if (next != 0) continue;
        if (tail) {                    // the tail's frontier drained: converged
            if (first) ctl->exit_reason = 1;
            break;
        }
        // Band drained: its heavy arcs first (one more iteration), then the
        // split.  The band lists are cleared in the split, so no block can
        // still be reading their counts here.
        // The pull form when the band listed more heavy arcs than a pull
        // would read: the heavy arcs of the vertices unsettled before the
        // band less the band's own, plus the sweep over every label (taken
        // as n / 8 arcs: coalesced, against one random label per arc).
        // Listings count a vertex once per relaxation, which leans to the
        // pull only when the band is large.
        if (a.defer && !was_hp && !tail &&
            (ldcg_u32(&ctl->band_count) | ldcg_u32(&ctl->band_hcount)) != 0) {
            hp = true;
            const unsigned long long listed_hs =
                ldcg_u64(reinterpret_cast<const uint64_t *>(&ctl->band_hsum));
            const unsigned long long rest = pull_bound > listed_hs ? pull_bound - listed_hs : 0ull;
            const uint32_t sweep =
                listed ? min(ldcg_u32(&ctl->far_count[phase & 1]), a.n) : a.n;
            pull = a.pull == 2 || (a.pull == 1 && listed_hs > rest + sweep / 8);
            continue;
        }

        // Near frontier drained: raise the threshold and split the far pile.
        // Every block has just read near_count[it % 3] to take this branch,
        // so the split must not push there: it fills the slot (and queue)
        // of iteration it + 1, and the loop resumes at it + 1.  That slot was
        // cleared at the top of iteration it - 1 and nothing reads it before
        // the barrier that ends the split.  Iteration it + 1 will push into
        // slot (it + 2) % 3, which the skipped top of iteration it would
        // have cleared: clear it here (its last reader was iteration it - 1).
        // With the far scan there is no pile: every label at or above the
        // threshold came from a proposal (or a split) that lowered far_min,
        // so an infinite far_min means no vertex is left unsettled.
        uint32_t nf = min(ldcg_u32(&ctl->far_count[fc]), a.n);
        uint32_t fmin = ldcg_u32(&ctl->far_min[fc]);
        if (a.far_scan ? fmin == INF32 : nf == 0) {           // converged
            if (first) ctl->exit_reason = 1;
            break;
        }
        uint64_t T_old = T;
        T = (fmin != INF32 && (uint64_t)fmin > T ? (uint64_t)fmin : T) + a.delta;
        ++phase;
        const uint32_t *fs = fc ? a.far1 : a.far0;
        const uint32_t its = it + 1;
        if (first) {
            ctl->near_count[(its + 1) % 3] = 0;
            ctl->heavy_count[(its + 1) % 3] = 0;
            ctl->band_count = 0;
            ctl->band_hcount = 0;
            ctl->band_hsum = 0;
        }
        stage_reset(st);
        PushTargets u;
        u.qn = (its & 1) ? a.q1 : a.q0;
        u.qn_count = &ctl->near_count[its % 3];
        u.hqn = (its & 1) ? a.hq1 : a.hq0;
        u.hqn_count = &ctl->heavy_count[its % 3];
        u.farq = fc ? a.far0 : a.far1;
        u.far_count = &ctl->far_count[fc ^ 1];
        u.far_min = &ctl->far_min[fc ^ 1];
        // With the far scan the split rebuilds the pile as the candidate
        // list: every vertex at or above T_old (the new band's frontier and
        // all later ones; unreached vertices with arcs too), staged in the
        // band regions, which no band listing uses during a split.
        u.bandq = a.far_scan ? (fc ? a.far0 : a.far1) : a.band_q;
        u.band_count = a.far_scan ? &ctl->far_count[fc ^ 1] : &ctl->band_count;
        u.tag_next = a.base_near + its;
        u.tag_far = a.base_far + phase;
        u.T = T;
        u.flush = true;
        // the first split sweeps every id, and sets whole bitmap words;
        // a split over the list sets bits, and only for a list long enough
        // that the next iteration's sweep of the bitmap pays
        const bool from_list = a.far_scan && listed;
        const bool dense_out = a.dense && (!from_list || nf >= a.n / 64);
        u.dense = dense_out;
        u.nbm = (its & 1) ? a.nbm1 : a.nbm0;
        u.nostamp = false;             // the split visits each vertex once
        u.nostamp_stamp = a.stamp_near;
        u.hsum = nullptr;
        u.lend = tail ? nullptr : a.lend;
        // the far pile (or list), or with the far scan first every vertex
        const uint32_t n_split = (a.far_scan && !from_list) ? a.n : nf;
        // SPLIT_ILP chunks of 32 per warp step, their loads issued together.
        // A vertex is met once here (the pile holds it once, the scan visits
        // each id once) and nothing relaxes during the split, so its near
        // stamp is a plain store.
        for (uint32_t b = warp * 32 * SPLIT_ILP; b < n_split; b += nwarps * 32 * SPLIT_ILP) {
            uint32_t v[SPLIT_ILP], deg[SPLIT_ILP];
            uint64_t d[SPLIT_ILP];
            bool to_near[SPLIT_ILP], cand[SPLIT_ILP], keep[SPLIT_ILP], in[SPLIT_ILP];
#pragma unroll
            for (int c = 0; c < SPLIT_ILP; ++c) {
                const uint32_t i = b + 32u * c + lane;
                in[c] = i < n_split;
                v[c] = 0;
                d[c] = INF32;
                if (in[c]) v[c] = (a.far_scan && !from_list) ? i : ldcg_u32(&fs[i]);
            }
#pragma unroll
            for (int c = 0; c < SPLIT_ILP; ++c)
                if (in[c]) d[c] = sssp_label<NARROW>(a, v[c]) >> 32;
#pragma unroll
            for (int c = 0; c < SPLIT_ILP; ++c) {
                const bool valid = d[c] != INF32;                  // unreached or past the end
                to_near[c] = valid && d[c] >= T_old && d[c] < T;   // below T_old: already settled
                cand[c] = valid && d[c] >= T;
                deg[c] = 0;
                // dense: ids at or above n_big are light without a look at the row
                if (to_near[c] && (!a.dense || v[c] < a.n_big)) {
                    const uint32_t r0 = a.row_ptr[v[c]];
                    const uint32_t r1 = u.lend ? u.lend[v[c]] : a.row_ptr[v[c] + 1];
                    a.stamp_near[v[c]] = u.tag_next;
                    deg[c] = r1 - r0;
                }
                if (a.far_scan) {
                    // the list keeps to_near and cand vertices, and unreached
                    // ones with arcs (isolated vertices are never reached)
                    keep[c] = to_near[c] || cand[c];
                    if (in[c] && !valid)
                        keep[c] = from_list || a.row_ptr[v[c] + 1] != a.row_ptr[v[c]];
                } else {
                    keep[c] = cand[c] &&
                              atomicExch(&a.stamp_far[v[c]], u.tag_far) != u.tag_far;
                }
            }
#pragma unroll
            for (int c = 0; c < SPLIT_ILP; ++c) {
                // dense: light vertices as bits; from the id sweep a chunk is
                // one bitmap word (empty since the band drained), so one store
                const bool bit = dense_out && to_near[c] && deg[c] < HEAVY_DEG;
                const uint32_t word = __ballot_sync(FULL, bit);
                if (from_list) {
                    if (bit) atomicOr(&u.nbm[v[c] >> 5], 1u << (v[c] & 31));
                } else if (lane == 0 && word) {
                    u.nbm[(b + 32u * c) >> 5] = word;
                }
                if (lane == 0 && word) st.dn_near[threadIdx.x >> 5] += (uint32_t)__popc(word);
                push_near(a, st, u, to_near[c] && !bit, v[c], deg[c]);
                if (a.far_scan) {
                    const uint32_t w = threadIdx.x >> 5;
                    region_append(keep[c], v[c], st.band_buf + w * BAND_REGION, &st.band_n[w],
                                  BAND_REGION, true, u.bandq, u.band_count, a.n, &ctl->err);
                }
                push_far(a, st, u, keep[c] && !a.far_scan, cand[c], v[c], (uint32_t)d[c]);
            }
        }
        flush_stage(st, u, a.n, &ctl->err);
        if (!grid_sync(&ctl->bar, &ctl->err)) {
            if (first) ctl->exit_reason = 4;
            break;
        }
        if (first) {
            ctl->far_count[fc] = 0;
            ctl->far_min[fc] = INF32;
            ctl->pull_hsum = 0;      // read after the pass's barrier, before this one
        }
        it = its;
        cur_dense = dense_out;        // the split set the next frontier's bits
        listed = a.far_scan != 0;
        if (it >= a.max_iters) {
            if (first) {
                atomicOr(&ctl->err, ERR_TIMEOUT);
                ctl->exit_reason = 2;
            }
            break;
        }
    }
    // counters
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        attempts += __shfl_xor_sync(FULL, attempts, o);
        improved += __shfl_xor_sync(FULL, improved, o);
    }
    if (lane == 0) {
        atomicAdd(&ctl->relax_attempts, attempts);
        atomicAdd(&ctl->relax_improved, improved);
    }
    if (NARROW && __any_sync(FULL, narrow_miss) && lane == 0) atomicOr(&ctl->err, ERR_NARROW);
    if (first) {
        ctl->iterations = it;
        ctl->phases = phase;
        ctl->bands = bands;
        ctl->end_ns = global_ns();
    }
}
// ---------------------------------------------------------------------------
// export: packed labels -> (cell seed id, distance, predecessor id)
// ---------------------------------------------------------------------------

__global__ void export_kernel(uint32_t n, const uint2 *__restrict__ adj,
                              const uint64_t *__restrict__ label,
                              const uint32_t *__restrict__ label32, uint32_t lshift,
                              const uint32_t *__restrict__ pred_arc,
                              const int32_t *__restrict__ seeds,
                              const uint32_t *__restrict__ orig_of, int32_t *cell, uint32_t *dist,
                              int32_t *pred) {
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const uint32_t v = caller_id(orig_of, u);       // outputs are in the caller's ids
        uint64_t lab = label32 ? widen_label(label32[u], lshift) : label[u];
        if (lab == INF64) {
            if (cell) cell[v] = -1;
            if (dist) dist[v] = INF32;
            if (pred) pred[v] = -1;
            continue;
        }
        if (cell) cell[v] = seeds[(uint32_t)lab];
        if (dist) dist[v] = (uint32_t)(lab >> 32);
        if (pred) {
            uint32_t pa = pred_arc[u];
            pred[v] = pa == SEED_ARC ? (int32_t)v
                                     : (pa == INF32 ? -1 : (int32_t)caller_id(orig_of, adj[pa].x));
        }
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

static int grid_for(uint64_t items, int threads) {
    uint64_t b = (items + threads - 1) / threads;
    if (b < 1) b = 1;
    const uint64_t cap = (uint64_t)current_sm_count() * 16;
    if (b > cap) b = cap;
    return (int)b;
}

cudaError_t launch_init(const DevGraph &g, Workspace &ws, uint32_t k, uint32_t delta,
                        cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(ws.ctl, 0, sizeof(Control), s);
    if (e != cudaSuccess) return e;
    uint32_t *l32 = ws.narrow ? ws.label32 : nullptr;
    init_labels_kernel<<<grid_for(g.n, 256), 256, 0, s>>>(g.n, ws.label, l32, ws.pred_arc);
    init_seeds_kernel<<<(k + 255) / 256, 256, 0, s>>>(g.row_ptr, active_lend(g, delta), ws.seeds,
                                                       g.new_of, k, ws.label, l32,
                                                       ws.pred_arc, ws.stamp_near,
                                                       ws.epoch_near, ws.q[0], ws.hq[0],
                                                       g.heavy_chunk_cap, g.n, ws.ctl);
    return cudaGetLastError();
}

// Co-resident blocks per SM that both label widths of the kernel reach.
int sssp_occupancy(int threads) {
    int nw = 0, nn = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nw, sssp_kernel<false>, threads, 0) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nn, sssp_kernel<true>, threads, 0) !=
            cudaSuccess)
        return 0;
    return nw < nn ? nw : nn;
}

cudaError_t launch_sssp(const DevGraph &g, Workspace &ws, const Geometry &geo,
                        const SsspParams &p, cudaStream_t s) {
    SsspArgs a;
    a.row_ptr = g.row_ptr;
    a.adj = g.adj;
    a.n = g.n;
    a.label = ws.label;
    a.label32 = ws.label32;
    a.lshift = ws.lshift;
    a.ldmax = (uint32_t)((1ull << (32 - ws.lshift)) - 2);
    a.stamp_near = ws.stamp_near;
    a.stamp_far = ws.stamp_far;
    a.q0 = ws.q[0];
    a.q1 = ws.q[1];
    a.hq0 = ws.hq[0];
    a.hq1 = ws.hq[1];
    a.far0 = ws.far[0];
    a.far1 = ws.far[1];
    a.ctl = ws.ctl;
    a.delta = p.delta;
    a.max_iters = p.max_iters;
    a.base_near = p.base_near;
    a.base_far = p.base_far;
    a.heavy_cap = g.heavy_chunk_cap;
    a.local_rounds = p.local_rounds;
    a.stamp_band = ws.stamp_band;
    a.band_q = ws.band_q;
    a.band_hq = ws.band_hq;
    a.base_band = p.base_band;
    a.defer = p.delta <= g.max_w ? 1u : 0u;
    a.far_scan = p.far_scan;
    a.trace = p.trace;
    a.dense = p.dense;
    a.pull = p.far_scan ? p.pull : 0u;
    a.tail = p.tail;
    a.m = g.m;
    a.n_big = g.n_big;
    a.n_words = (g.n + 31) / 32;
    a.nbm0 = ws.nbm[0];
    a.nbm1 = ws.nbm[1];
    a.bbm = ws.bbm;
    a.lend = active_lend(g, p.delta);
    if (a.lend) a.adj = g.adj_w;        // rows partitioned by weight class
    void *args[] = {&a};
    const void *fn = ws.narrow ? (const void *)sssp_kernel<true> : (const void *)sssp_kernel<false>;
    return cudaLaunchCooperativeKernel(fn, dim3(geo.sssp_blocks), dim3(geo.threads), args, 0, s);
}

cudaError_t launch_export(const DevGraph &g, Workspace &ws, uint32_t k, int32_t *cell,
                          uint32_t *dist, int32_t *pred, cudaStream_t s) {
    (void)k;
    export_kernel<<<grid_for(g.n, 256), 256, 0, s>>>(g.n, g.adj, ws.label,
                                                      ws.narrow ? ws.label32 : nullptr, ws.lshift,
                                                      ws.pred_arc, ws.seeds, g.orig_of, cell,
                                                      dist, pred);
    return cudaGetLastError();
}

}  // namespace stn
