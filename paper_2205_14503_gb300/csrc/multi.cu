// Multi-query Voronoi cells and bridge scan (the batched and serving modes).
//
// The arithmetic per query is exactly the single-query path's (Algorithm 2
// Steps 1-2 with the same packed (distance, rank) atomicMin fixed point and
// the same tie rules); what changes is how the work of up to 64 queries is
// shared:
//  * labels are vertex-major, label[v * 64 + q], so relaxing one arc for all
//    pending slots is one contiguous 256-byte run of atomics; a label is 32
//    bits, (distance << b) | rank with b the bits of the slot's largest rank
//    (ordered by (distance, rank) as the 64-bit form), and a slot whose
//    distances do not fit is answered by the single-query path instead;
//  * a frontier entry is a vertex; nmask[v] says which slots must relax
//    v's arcs, so a CSR row is read once for all of them;
//  * each slot has its own near/far threshold T[q] and far accounting, so a
//    slot admitted mid-run starts its own bands (continuous batching);
//  * the persistent kernel can yield at an iteration boundary (a slot
//    converged, or the host rang the doorbell), keeping all state in device
//    memory, and resume later with more slots;
//  * light and heavy arcs are split per slot as in the single-query kernel:
//    while a slot's band iterates only arcs lighter than delta are relaxed,
//    a per-vertex mask records which slots relaxed the vertex in their
//    current band (vertices with any bit set are kept in a band list), and
//    when a slot's near work drains its heavy arcs are relaxed once, in the
//    next shared iteration, for the listed vertices with its bit.
#include "multi.h"

namespace stn {

// (arc, slot) pairs in flight per lane.  Two, at six 256-thread blocks per
// SM (40 registers), beat four at four blocks (64 registers): the kernel is
// bound by the latency of each item's chain of L2 round trips, so more
// resident warps pay more than more pairs per warp.
constexpr int MQ_ILP = 2;
constexpr uint32_t MQ_NEAR_STAGE = 1024;
constexpr uint32_t MQ_FAR_STAGE = 512;

struct MqArgs {
    const uint32_t *__restrict__ row_ptr;
    const uint2 *__restrict__ adj;
    uint32_t n;
    uint32_t *label;
    unsigned long long *nmask, *fmask;
    uint32_t *stamp_near, *in_far;
    uint32_t *q0, *q1;
    unsigned long long *item_mask;   // per frontier item: the slots it relaxes
    uint64_t *item_pre;              // per item: (arc, slot) pairs before it in its block segment
    uint64_t *bsum;                  // per block: pairs in its segment
    uint32_t *far0, *far1;
    unsigned long long *bmask;       // per vertex: slots that relaxed it in their current band
    uint32_t *bl0, *bl1, *bl2;       // band lists
    MqControl *ctl;
    const uint32_t *doorbell;
    uint32_t delta;
    uint32_t base_near;
    uint32_t max_iters;
    uint32_t yield;          // leave once this many slots converged (0: only when all did)
    uint32_t defer;          // light/heavy arc split on (some weight >= delta)
    // with the split: end of each row's light part in the weight-partitioned
    // adjacency `adj` (null: rows are unpartitioned and arcs are filtered)
    const uint32_t *lend;
    uint32_t pull;           // first heavy-arc pass of a slot in the pull form
};

__device__ __forceinline__ uint32_t *band_list(const MqArgs &a, uint32_t i) {
    return i == 0 ? a.bl0 : (i == 1 ? a.bl1 : a.bl2);
}

constexpr int MQ_WARPS = 256 / 32;
constexpr int MQ_MAX_BLOCKS = 1024;

struct MqStage {
    uint64_t boff[MQ_MAX_BLOCKS];          // pair offset of each block's frontier segment
    uint64_t wtot[MQ_WARPS];
    uint64_t carry, W;
    uint32_t near_buf[MQ_NEAR_STAGE];
    uint32_t far_buf[MQ_FAR_STAGE];
    uint32_t near_n, far_n, base_near, base_far;
    unsigned long long act;
    unsigned long long T[MQ_SLOTS];        // current thresholds (block copy)
    unsigned long long Tnew[MQ_SLOTS];     // thresholds after a split
    uint32_t fmin[MQ_SLOTS];               // far-distance minimum of this segment
    int32_t fpend[MQ_SLOTS];               // change of far_pending in this segment
    unsigned long long mag[MQ_SLOTS + 1];  // ceil(2^40 / c) for c = 2..64 (divmod by c)
    uint32_t lshift[MQ_SLOTS];             // rank bits of each slot's labels
};

// Slot q's label of v in the 64-bit form (dist << 32) | rank.
__device__ __forceinline__ uint64_t mq_label(const uint32_t *label, uint64_t v, uint32_t q,
                                             uint32_t shift) {
    return widen_label(ldcg_u32(&label[v * MQ_SLOTS + q]), shift);
}

struct MqTargets {
    uint32_t *qn, *qn_count;
    unsigned long long *act;
    uint32_t *farq, *far_count;
    uint32_t *fmin;          // ctl->fmin[pile]
    uint32_t tag_next;
};

__device__ __forceinline__ int popc64(unsigned long long x) { return __popcll(x); }

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Inclusive scan of one 64-bit value per thread over a 256-thread block;
// wtot[] receives the per-warp inclusive totals (wtot[MQ_WARPS-1] = block
// total after the call).  Every thread of the block must call it.
__device__ __forceinline__ uint64_t block_inclusive_scan64(uint64_t x, uint64_t *wtot) {
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= (uint32_t)o) x += y;
    }
    if (lane == 31) wtot[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t acc = 0;
        for (int i = 0; i < MQ_WARPS; ++i) {
            acc += wtot[i];
            wtot[i] = acc;
        }
    }
    __syncthreads();
    return x + (w ? wtot[w - 1] : 0);
}

// Index of the t-th set bit (0-based) of a 32-bit word.
__device__ __forceinline__ uint32_t nth_bit32(uint32_t x, uint32_t t) {
    uint32_t pos = 0;
#pragma unroll
    for (uint32_t w = 16; w >= 1; w >>= 1) {
        uint32_t c = __popc(x & ((1u << w) - 1u));
        if (t >= c) {
            t -= c;
            x >>= w;
            pos += w;
        }
    }
    return pos;
}

__device__ __forceinline__ uint32_t nth_bit64(unsigned long long m, uint32_t t) {
    uint32_t lo = (uint32_t)m, pl = (uint32_t)__popc(lo);
    return t < pl ? nth_bit32(lo, t) : 32 + nth_bit32((uint32_t)(m >> 32), t - pl);
}

__device__ __forceinline__ unsigned long long warp_or64(unsigned long long x) {
    uint32_t lo = __reduce_or_sync(FULL, (uint32_t)x);
    uint32_t hi = __reduce_or_sync(FULL, (uint32_t)(x >> 32));
    return ((unsigned long long)hi << 32) | lo;
}

__device__ __forceinline__ void seg_reset(MqStage &st) {
    if (threadIdx.x == 0) {
        st.near_n = 0;
        st.far_n = 0;
        st.act = 0;
    }
    if (threadIdx.x < MQ_SLOTS) {
        st.fmin[threadIdx.x] = INF32;
        st.fpend[threadIdx.x] = 0;
    }
    __syncthreads();
}

__device__ __forceinline__ void seg_flush(MqStage &st, const MqTargets &t, MqControl *ctl,
                                          uint32_t n) {
    __syncthreads();
    uint32_t nn = min(st.near_n, MQ_NEAR_STAGE), nf = min(st.far_n, MQ_FAR_STAGE);
    if (threadIdx.x == 0) {
        st.base_near = nn ? atomicAdd(t.qn_count, nn) : 0;
        st.base_far = nf ? atomicAdd(t.far_count, nf) : 0;
        if (st.act) atomicOr(t.act, st.act);
    }
    if (threadIdx.x < MQ_SLOTS) {
        uint32_t q = threadIdx.x;
        if (st.fmin[q] != INF32) atomicMin(&t.fmin[q], st.fmin[q]);
        if (st.fpend[q]) atomicAdd(&ctl->far_pending[q], st.fpend[q]);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nn; i += blockDim.x) {
        uint32_t slot = st.base_near + i;
        if (slot < n) t.qn[slot] = st.near_buf[i];
        else atomicOr(&ctl->err, ERR_CAPACITY);
    }
    for (uint32_t i = threadIdx.x; i < nf; i += blockDim.x) {
        uint32_t slot = st.base_far + i;
        if (slot < n) t.farq[slot] = st.far_buf[i];
        else atomicOr(&ctl->err, ERR_CAPACITY);
    }
}

// A vertex with near work joins the next frontier through the staging
// buffer.  (Hubs need no special handling: work is split by pairs.)
__device__ __forceinline__ void mq_push_near(const MqArgs &a, MqStage &st, const MqTargets &t,
                                             bool want, uint32_t v) {
    stage_append(want, v, st.near_buf, &st.near_n, MQ_NEAR_STAGE, t.qn, t.qn_count, a.n,
                 &a.ctl->err);
}

// Relaxes up to MQ_ILP (arc, slot) pairs per lane.
// Pair i is arc arc[i] for slot qs[i]; heavy[i] marks a heavy-arc pass
// item (only arcs of weight >= delta), else only lighter arcs are relaxed
// when the split is on.
__device__ __forceinline__ void mq_relax(const MqArgs &a, MqStage &st, const MqTargets &t,
                                         const bool (&valid)[MQ_ILP],
                                         const uint32_t (&arc)[MQ_ILP],
                                         const uint32_t (&qs)[MQ_ILP],
                                         const uint64_t (&lab)[MQ_ILP],
                                         const bool (&heavy)[MQ_ILP],
                                         unsigned long long &attempts,
                                         unsigned long long &improved,
                                         unsigned long long &narrow_miss) {
    uint2 e[MQ_ILP];
#pragma unroll
    for (int i = 0; i < MQ_ILP; ++i) {
        e[i] = make_uint2(0, 0);
        if (valid[i]) e[i] = __ldg(&a.adj[arc[i]]);
    }
    uint64_t nd[MQ_ILP];
    bool imp[MQ_ILP];
#pragma unroll
    for (int i = 0; i < MQ_ILP; ++i) {
        imp[i] = false;
        nd[i] = INF32;
        if (!valid[i] || lab[i] == INF64) continue;
        if (heavy[i] ? e[i].y < a.delta : (a.defer && e[i].y >= a.delta)) continue;
        ++attempts;
        nd[i] = (lab[i] >> 32) + (uint64_t)e[i].y;
        const uint32_t sh = st.lshift[qs[i]];
        if (nd[i] > (uint64_t)((1ull << (32 - sh)) - 2)) {
            narrow_miss |= 1ull << qs[i];        // the slot is answered by the single-query path
        } else {
            // read first: most proposals do not improve, and a load costs far
            // less L2 throughput than an atomic
            const uint32_t nl = ((uint32_t)nd[i] << sh) | (uint32_t)lab[i];
            uint32_t *dst = &a.label[(uint64_t)e[i].x * MQ_SLOTS + qs[i]];
            if (nl < ldcg_u32(dst)) {
                const uint32_t old = atomicMin(dst, nl);
                imp[i] = nl < old;
            }
        }
    }
    // most rounds improve nothing: skip the append machinery then
    bool any_imp = false;
#pragma unroll
    for (int i = 0; i < MQ_ILP; ++i) any_imp |= imp[i];
    if (!__any_sync(FULL, any_imp)) return;
    bool to_near[MQ_ILP], to_far[MQ_ILP];
    unsigned long long act = 0;
#pragma unroll
    for (int i = 0; i < MQ_ILP; ++i) {
        to_near[i] = to_far[i] = false;
        if (!imp[i]) continue;
        ++improved;
        uint32_t v = e[i].x, q = qs[i];
        unsigned long long bit = 1ull << q;
        if (nd[i] < st.T[q]) {
            atomicOr(&a.nmask[v], bit);
            to_near[i] = atomicExch(&a.stamp_near[v], t.tag_next) != t.tag_next;
            act |= bit;
        } else {
            unsigned long long old = atomicOr(&a.fmask[v], bit);
            if (!(old & bit)) atomicAdd(&st.fpend[q], 1);
            atomicMin(&st.fmin[q], (uint32_t)nd[i]);
            to_far[i] = atomicExch(&a.in_far[v], 1u) == 0;
        }
    }
    act = warp_or64(act);
    if (lane_id() == 0 && act) atomicOr(&st.act, act);
#pragma unroll
    for (int i = 0; i < MQ_ILP; ++i) {
        mq_push_near(a, st, t, to_near[i], e[i].x);
        stage_append(to_far[i], e[i].x, st.far_buf, &st.far_n, MQ_FAR_STAGE, t.farq, t.far_count,
                     a.n, &a.ctl->err);
    }
}

// Pull form of the first heavy-arc pass of the slots in P.  A slot in its
// first band has threshold delta; once its near work drained, every label
// below it is final, and a heavy arc (weight delta or more) brings a vertex
// still at or above it only a proposal at or above it.  So instead of
// pushing the heavy arcs of the band's vertices, every vertex unsettled in
// some slot of P reads its own heavy arcs and, per arc, the label run of the
// other end.  Warps sweep the vertices one at a time, lane l serving slots
// l and l + 32; each lane keeps its slots' best proposal from settled ends
// in registers and, after the row, sends one atomicMin per improved
// (vertex, slot) and does the bookkeeping of mq_relax for it (a far
// proposal: far mask, far pending count, far minimum, far pile).  Only
// this warp writes these labels during the iteration: the band items of
// the iteration leave out the slots of P, and those slots have no near
// work.
__device__ __noinline__ void mq_pull_sweep(const MqArgs &a, MqStage &st, unsigned long long P,
                                           uint32_t *qn, uint32_t *qn_count, uint32_t *farq,
                                           uint32_t *far_count, uint32_t tag_next,
                                           unsigned long long &attempts,
                                           unsigned long long &improved,
                                           unsigned long long &narrow_miss) {
    MqTargets t;
    t.qn = qn;
    t.qn_count = qn_count;
    t.act = nullptr;
    t.farq = farq;
    t.far_count = far_count;
    t.fmin = nullptr;
    t.tag_next = tag_next;
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t q0 = lane, q1 = lane + 32;
    const bool p0 = (P >> q0) & 1ull, p1 = (P >> q1) & 1ull;
    const uint32_t sh0 = st.lshift[q0], sh1 = st.lshift[q1];
    const unsigned long long T0 = st.T[q0], T1 = st.T[q1];
    const uint64_t lm0 = (1ull << (32 - sh0)) - 2, lm1 = (1ull << (32 - sh1)) - 2;
    for (uint32_t v = warp; v < a.n; v += nwarps) {
        const uint64_t base = (uint64_t)v * MQ_SLOTS;
        const uint64_t la = p0 ? widen_label(ldcg_u32(&a.label[base + q0]), sh0) : 0ull;
        const uint64_t lb = p1 ? widen_label(ldcg_u32(&a.label[base + q1]), sh1) : 0ull;
        const bool ua = p0 && (la == INF64 || (la >> 32) >= T0);
        const bool ub = p1 && (lb == INF64 || (lb >> 32) >= T1);
        if (!__any_sync(FULL, ua || ub)) continue;
        const uint32_t r1 = a.row_ptr[v + 1];
        const uint32_t s = a.lend ? a.lend[v] : a.row_ptr[v];
        uint64_t ba = INF64, bb = INF64;
        for (uint32_t j = s; j < r1; ++j) {
            const uint2 e = a.adj[j];                  // one record, every lane
            if (e.y < a.delta) continue;               // light (unpartitioned rows only)
            const uint64_t ub_ = (uint64_t)e.x * MQ_SLOTS;
            const uint32_t xa = ua ? ldcg_u32(&a.label[ub_ + q0]) : INF32;
            const uint32_t xb = ub ? ldcg_u32(&a.label[ub_ + q1]) : INF32;
            if (xa != INF32) {
                const uint64_t lu = widen_label(xa, sh0);
                if ((lu >> 32) < T0) {                 // a settled end proposes
                    ++attempts;
                    const uint64_t nd = (lu >> 32) + (uint64_t)e.y;
                    if (nd > lm0) {
                        if (la == INF64) narrow_miss |= 1ull << q0;
                    } else {
                        ba = min(ba, (uint64_t)((nd << 32) | (lu & 0xFFFFFFFFull)));
                    }
                }
            }
            if (xb != INF32) {
                const uint64_t lu = widen_label(xb, sh1);
                if ((lu >> 32) < T1) {
                    ++attempts;
                    const uint64_t nd = (lu >> 32) + (uint64_t)e.y;
                    if (nd > lm1) {
                        if (lb == INF64) narrow_miss |= 1ull << q1;
                    } else {
                        bb = min(bb, (uint64_t)((nd << 32) | (lu & 0xFFFFFFFFull)));
                    }
                }
            }
        }
        const bool ia = ua && ba < la, ib = ub && bb < lb;
        if (ia) atomicMin(&a.label[base + q0], ((uint32_t)(ba >> 32) << sh0) | (uint32_t)ba);
        if (ib) atomicMin(&a.label[base + q1], ((uint32_t)(bb >> 32) << sh1) | (uint32_t)bb);
        const bool fa = ia && (ba >> 32) >= T0, fb = ib && (bb >> 32) >= T1;
        unsigned long long nbits = (ia && !fa ? 1ull << q0 : 0ull) | (ib && !fb ? 1ull << q1 : 0ull);
        unsigned long long fbits = (fa ? 1ull << q0 : 0ull) | (fb ? 1ull << q1 : 0ull);
        nbits = warp_or64(nbits);
        fbits = warp_or64(fbits);
        if (!(nbits | fbits)) continue;
        improved += (ia ? 1u : 0u) + (ib ? 1u : 0u);
        unsigned long long fold = 0;
        bool to_far = false, to_near = false;
        if (lane == 0) {
            if (fbits) {
                fold = atomicOr(&a.fmask[v], fbits);
                to_far = atomicExch(&a.in_far[v], 1u) == 0;
            }
            if (nbits) {
                atomicOr(&a.nmask[v], nbits);
                to_near = atomicExch(&a.stamp_near[v], tag_next) != tag_next;
                atomicOr(&st.act, nbits);
            }
        }
        fold = __shfl_sync(FULL, fold, 0);
        if (fa) {
            if (!((fold >> q0) & 1ull)) atomicAdd(&st.fpend[q0], 1);
            atomicMin(&st.fmin[q0], (uint32_t)(ba >> 32));
        }
        if (fb) {
            if (!((fold >> q1) & 1ull)) atomicAdd(&st.fpend[q1], 1);
            atomicMin(&st.fmin[q1], (uint32_t)(bb >> 32));
        }
        mq_push_near(a, st, t, to_near, v);
        stage_append(to_far, v, st.far_buf, &st.far_n, MQ_FAR_STAGE, t.farq, t.far_count, a.n,
                     &a.ctl->err);
    }
}

__global__ void __launch_bounds__(256, 6) mq_sssp_kernel(MqArgs a) {
    __shared__ MqStage st;
    MqControl *ctl = a.ctl;
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const bool first = gtid == 0;
    unsigned long long attempts = 0, improved = 0, narrow_miss = 0;
    uint32_t it = ldcg_u32(&ctl->it), fc = ldcg_u32(&ctl->fc);
    unsigned long long infl = __ldcg(&ctl->inflight) & ~__ldcg(&ctl->converged);
    unsigned long long conv_total = 0;
    // heavy-arc passes: H = slots whose pass runs in this iteration
    unsigned long long H = __ldcg(&ctl->hpass) & infl;
    unsigned long long hp_done = __ldcg(&ctl->hp_done);
    unsigned long long band0 = __ldcg(&ctl->band0);
    uint32_t pull_sweeps = 0;
    uint32_t bc = ldcg_u32(&ctl->blist);
    if (threadIdx.x < MQ_SLOTS) {
        st.T[threadIdx.x] = __ldcg(&ctl->T[threadIdx.x]);
        st.lshift[threadIdx.x] = ldcg_u32(&ctl->lshift[threadIdx.x]);
    }
    if (threadIdx.x <= MQ_SLOTS) {
        const uint32_t c = threadIdx.x;
        st.mag[c] = c > 1 ? ((1ull << 40) + c - 1) / c : 0ull;
    }
    __syncthreads();
    uint32_t iters = 0, reason = 0;

    while (infl) {
        const uint32_t cs = it % 3, ns = (it + 1) % 3;
        const bool odd = it & 1;
        const uint32_t n_items = min(ldcg_u32(&ctl->near_count[cs]), a.n);
        // Work items: the near frontier, then (when some slots run their
        // heavy-arc pass) the band list.  A pass reads list bc and moves the
        // survivors, with this iteration's new listings, to list bc + 1;
        // list bc + 2 (read by the previous pass) is cleared for the next.
        // slots of H in their first band run the pass in the pull form
        const unsigned long long P = a.pull ? (H & band0) : 0ull;
        const uint32_t n_band = H ? min(ldcg_u32(&ctl->bcount[bc]), a.n) : 0u;
        const uint32_t n_all = n_items + n_band;
        const uint32_t tgt = H ? (bc + 1) % 3 : bc;
        const uint32_t *blo = band_list(a, bc);
        uint32_t *bln = band_list(a, tgt);
        if (first) {
            uint32_t r = (it + 2) % 3;
            ctl->near_count[r] = 0;
            ctl->act[r] = 0;
            if (H) ctl->bcount[(bc + 2) % 3] = 0;
        }
        const uint32_t *qc = odd ? a.q1 : a.q0;

        unsigned long long tm0 = first ? gtimer() : 0;
        // Phase A: every frontier vertex takes its pending slot mask; its
        // work is deg x |mask| (arc, slot) pairs; prefix sums per block
        // segment of the frontier.
        const uint32_t seg = (n_all + gridDim.x - 1) / gridDim.x;
        const uint32_t seg_lo = min(n_all, blockIdx.x * seg);
        const uint32_t seg_hi = min(n_all, seg_lo + seg);
        if (threadIdx.x == 0) st.carry = 0;
        __syncthreads();
        for (uint32_t b0 = seg_lo; b0 < seg_hi; b0 += blockDim.x) {
            uint32_t i = b0 + threadIdx.x;
            uint64_t w = 0;
            bool listed = false;
            uint32_t u = 0;
            if (i < seg_hi) {
                unsigned long long M;
                if (i < n_items) {
                    u = ldcg_u32(&qc[i]);
                    M = atomicExch(&a.nmask[u], 0ull);
                    // first slot to relax u in its band lists u
                    if (a.defer && M) listed = atomicOr(&a.bmask[u], M) == 0ull;
                } else {
                    u = ldcg_u32(&blo[i - n_items]);
                    const unsigned long long old = atomicAnd(&a.bmask[u], ~H);
                    M = old & H & ~P;            // the slots whose band closes now (pushed)
                    listed = (old & ~H) != 0ull; // still in other slots' bands
                }
                a.item_mask[i] = M;
                // frontier items relax the light part, band items the heavy one
                const uint32_t r0 = a.row_ptr[u], r1 = a.row_ptr[u + 1];
                const uint32_t le = a.lend ? a.lend[u] : r1;
                const uint32_t deg = i < n_items ? le - r0 : (a.lend ? r1 - le : r1 - r0);
                w = (uint64_t)deg * (uint64_t)popc64(M);
            }
            const uint32_t ls = warp_append(listed, &ctl->bcount[tgt], a.n, &ctl->err);
            if (ls != INF32) bln[ls] = u;
            uint64_t incl = block_inclusive_scan64(w, st.wtot);
            if (i < seg_hi) a.item_pre[i] = st.carry + incl - w;
            __syncthreads();
            if (threadIdx.x == blockDim.x - 1) st.carry += incl;
            __syncthreads();
        }
        if (threadIdx.x == 0) a.bsum[blockIdx.x] = st.carry;
        unsigned long long tm1 = first ? gtimer() : 0;
        if (!grid_sync(&ctl->bar, &ctl->err)) { reason = 5; break; }
        unsigned long long tm2 = first ? gtimer() : 0;
        // block offsets and the total
        {
            uint64_t carry = 0;
            for (uint32_t b0 = 0; b0 < gridDim.x; b0 += blockDim.x) {
                uint32_t b = b0 + threadIdx.x;
                uint64_t x = b < gridDim.x ? __ldcg(reinterpret_cast<const unsigned long long *>(&a.bsum[b])) : 0;
                uint64_t incl = block_inclusive_scan64(x, st.wtot);
                if (b < gridDim.x) st.boff[b] = carry + incl - x;
                __syncthreads();
                carry += st.wtot[MQ_WARPS - 1];
                __syncthreads();
            }
            if (threadIdx.x == 0) st.W = carry;
            __syncthreads();
        }
        seg_reset(st);
        MqTargets t;
        t.qn = odd ? a.q0 : a.q1;
        t.qn_count = &ctl->near_count[ns];
        t.act = &ctl->act[ns];
        t.farq = fc ? a.far1 : a.far0;
        t.far_count = &ctl->far_count[fc];
        t.fmin = ctl->fmin[fc];
        t.tag_next = a.base_near + it + 1;

        // Phase B: the W (arc, slot) pairs, numbered arc-major inside each
        // item (arc j, slot t -> j * |mask| + t), are cut into 32 chunks per
        // warp, and warp w takes chunks w, w + nw, w + 2 nw, ... spread over
        // the whole pair space, so a costly region (many improving pairs) is
        // shared by many warps.  Lane i finds the first item of the warp's
        // i-th chunk (all 32 searches at once).  Inside a chunk the warp
        // slides a window of 32 consecutive items (one per lane, loaded in
        // parallel) and spreads the window's pairs over its lanes, MQ_ILP per
        // lane in flight.
        const uint64_t W = st.W;
        auto gpre = [&](uint32_t i) -> uint64_t {
            return st.boff[i / seg] + __ldcg(reinterpret_cast<const unsigned long long *>(&a.item_pre[i]));
        };
        const uint64_t n_chunks = (uint64_t)nwarps * 32;
        const uint64_t my_chunk = warp + (uint64_t)lane * nwarps;
        const uint64_t my_p = (uint64_t)((unsigned __int128)W * my_chunk / n_chunks);
        const uint64_t my_p1 = (uint64_t)((unsigned __int128)W * (my_chunk + 1) / n_chunks);
        uint32_t my_i0 = 0;
        if (my_p < my_p1) {
            uint32_t lo = 0, hi = n_all;            // first item: largest i with gpre(i) <= p
            while (hi - lo > 1) {
                uint32_t mid = lo + (hi - lo) / 2;
                if (gpre(mid) <= my_p) lo = mid; else hi = mid;
            }
            my_i0 = lo;
        }
        for (uint32_t ch = 0; ch < 32; ++ch) {
            uint64_t p = __shfl_sync(FULL, my_p, ch);
            const uint64_t p1 = __shfl_sync(FULL, my_p1, ch);
            uint32_t i0 = __shfl_sync(FULL, my_i0, ch);
            while (p < p1) {
                uint32_t idx = i0 + lane;
                uint64_t pre = ~0ull;
                uint32_t u = 0, s0 = 0, c = 0;
                unsigned long long M = 0;
                if (idx < n_all) {
                    pre = gpre(idx);
                    u = idx < n_items ? ldcg_u32(&qc[idx]) : ldcg_u32(&blo[idx - n_items]);
                    M = __ldcg(&a.item_mask[idx]);
                    s0 = (idx >= n_items && a.lend) ? a.lend[u] : a.row_ptr[u];
                    c = (uint32_t)popc64(M);
                }
                const bool hv = idx >= n_items;        // heavy-arc pass item
                const uint64_t wend = i0 + 32 < n_all ? gpre(i0 + 32) : W;
                const uint64_t stop = min(p1, wend);
                // The window's items one after another: an item's pairs are
                // (arc j, slot t) -> j * c + t; the lanes take fixed slots
                // (and, for c <= 16, several arcs per step), so a lane finds
                // its slot and loads the tail's label once per item and then
                // steps over the arcs with one broadcast arc load per arc.
                for (uint32_t w = 0; w < 32; ++w) {
                    const uint64_t pre_w = __shfl_sync(FULL, pre, w);
                    if (pre_w >= stop) break;
                    uint64_t end_w = w < 31 ? __shfl_sync(FULL, pre, w + 1) : wend;
                    end_w = min(end_w, stop);
                    const uint32_t cw = __shfl_sync(FULL, c, w);
                    if (cw == 0 || end_w <= p || end_w <= pre_w) continue;
                    const uint32_t uw = __shfl_sync(FULL, u, w);
                    const uint32_t sw = __shfl_sync(FULL, s0, w);
                    const unsigned long long Mw = __shfl_sync(FULL, M, w);
                    const bool hw = __shfl_sync(FULL, hv, w);
                    // the item's pairs inside this chunk: [lo, hi)
                    const uint32_t lo = (uint32_t)((p > pre_w ? p : pre_w) - pre_w);
                    const uint32_t hi = (uint32_t)(end_w - pre_w);
                    const uint64_t mw = st.mag[cw];
                    const uint32_t jlo = cw > 1 ? (uint32_t)__umul64hi((uint64_t)lo, mw << 24) : lo;
                    const uint32_t jhi = cw > 1 ? (uint32_t)__umul64hi((uint64_t)(hi - 1), mw << 24) : hi - 1;
                    if (cw <= 32) {
                        // g lanes per arc (g = c rounded up to a power of two),
                        // 32 / g arcs per step
                        const uint32_t gsh = cw <= 1 ? 0u : 32u - __clz(cw - 1);
                        const uint32_t A = 32u >> gsh;
                        const uint32_t tq = lane & ((1u << gsh) - 1u), aoff = lane >> gsh;
                        const bool tok = tq < cw;
                        const uint32_t q = tok ? nth_bit64(Mw, tq) : 0u;
                        const uint64_t lab = tok ? mq_label(a.label, uw, q, st.lshift[q]) : INF64;
                        for (uint32_t j0 = jlo; j0 <= jhi; j0 += MQ_ILP * A) {
                            bool valid[MQ_ILP], heavy[MQ_ILP];
                            uint32_t arc[MQ_ILP], qs[MQ_ILP];
                            uint64_t labs[MQ_ILP];
#pragma unroll
                            for (int k = 0; k < MQ_ILP; ++k) {
                                const uint32_t jj = j0 + (uint32_t)k * A + aoff;
                                const uint32_t l = jj * cw + tq;
                                valid[k] = tok && jj <= jhi && l >= lo && l < hi;
                                heavy[k] = hw;
                                arc[k] = sw + jj;
                                qs[k] = q;
                                labs[k] = lab;
                            }
                            mq_relax(a, st, t, valid, arc, qs, labs, heavy, attempts, improved, narrow_miss);
                        }
                    } else {
                        // 33..64 slots: each lane takes slots lane and lane + 32
                        const uint32_t t1 = lane + 32;
                        const bool tok1 = t1 < cw;
                        const uint32_t q0 = cw == MQ_SLOTS ? lane : nth_bit64(Mw, lane);
                        const uint32_t q1 = tok1 ? (cw == MQ_SLOTS ? t1 : nth_bit64(Mw, t1)) : 0u;
                        const uint64_t lab0 = mq_label(a.label, uw, q0, st.lshift[q0]);
                        const uint64_t lab1 = tok1 ? mq_label(a.label, uw, q1, st.lshift[q1]) : INF64;
                        for (uint32_t j0 = jlo; j0 <= jhi; j0 += MQ_ILP / 2) {
                            bool valid[MQ_ILP], heavy[MQ_ILP];
                            uint32_t arc[MQ_ILP], qs[MQ_ILP];
                            uint64_t labs[MQ_ILP];
#pragma unroll
                            for (int k = 0; k < MQ_ILP; ++k) {
                                const uint32_t jj = j0 + (uint32_t)(k >> 1);
                                const bool second = k & 1;
                                const uint32_t tq = second ? t1 : lane;
                                const uint32_t l = jj * cw + tq;
                                valid[k] = (second ? tok1 : true) && jj <= jhi && l >= lo && l < hi;
                                heavy[k] = hw;
                                arc[k] = sw + jj;
                                qs[k] = second ? q1 : q0;
                                labs[k] = second ? lab1 : lab0;
                            }
                            mq_relax(a, st, t, valid, arc, qs, labs, heavy, attempts, improved, narrow_miss);
                        }
                    }
                }
                p = stop;
                i0 += 32;
            }
        }
        if (P) {
            mq_pull_sweep(a, st, P, t.qn, t.qn_count, t.farq, t.far_count, t.tag_next, attempts,
                          improved, narrow_miss);
            ++pull_sweeps;
        }
        unsigned long long tm3 = first ? gtimer() : 0;
        seg_flush(st, t, ctl, a.n);
        if (first)
            ctl->stop_req[it & 1] = (a.yield && a.doorbell) ? *(volatile const uint32_t *)a.doorbell : 0u;
        if (!grid_sync(&ctl->bar, &ctl->err)) { reason = 5; break; }
        if (first) {
            unsigned long long tm4 = gtimer();
            ctl->t_part[0] += tm1 - tm0;
            ctl->t_part[1] += tm2 - tm1;
            ctl->t_part[2] += tm3 - tm2;
            ctl->t_part[3] += tm4 - tm3;
            ctl->items_total += n_all;
            ctl->pairs_total += st.W;
        }
        ++it;
        ++iters;
        if (H) bc = (bc + 1) % 3;

        // per-slot decisions (every block computes the same from global
        // state): a slot with near work queued continues its band; an idle
        // one first runs its band's heavy-arc pass (next iteration), then is
        // converged if nothing is parked far, else its far pile is split
        unsigned long long act_next = __ldcg(&ctl->act[it % 3]);
        hp_done &= ~act_next;
        unsigned long long idle = infl & ~act_next, S = 0, conv = 0;
        H = a.defer ? (idle & ~hp_done) : 0ull;
        hp_done |= H;
        for (unsigned long long m = idle & ~H; m; m &= m - 1) {
            uint32_t q = __ffsll((long long)m) - 1;
            if (__ldcg(&ctl->far_pending[q]) <= 0) conv |= 1ull << q;
            else S |= 1ull << q;
        }
        hp_done &= ~S;                      // a split opens a new band
        band0 &= ~S;
        infl &= ~conv;
        conv_total |= conv;
        if (!infl) { reason = 1; break; }
        if (a.yield && (uint32_t)popc64(conv_total) >= a.yield) { reason = 2; break; }
        if (a.yield && ldcg_u32(&ctl->stop_req[(it - 1) & 1])) { reason = 3; break; }
        if (iters >= a.max_iters) { reason = 4; break; }
        if (!S) continue;

        unsigned long long tm5 = first ? gtimer() : 0;
        // Split the far pile for the slots in S.  A barrier first: every
        // block has read the decision inputs before the split appends to
        // them.  Near pushes go to this iteration's queue (slot it % 3).
        if (!grid_sync(&ctl->bar, &ctl->err)) { reason = 5; break; }
        if (threadIdx.x < MQ_SLOTS) {
            uint32_t q = threadIdx.x;
            unsigned long long Tq = st.T[q];
            if ((S >> q) & 1) {
                uint32_t fm = __ldcg(&ctl->fmin[fc][q]);
                unsigned long long base = (fm != INF32 && (unsigned long long)fm > Tq) ? fm : Tq;
                st.Tnew[q] = base + a.delta;
            } else {
                st.Tnew[q] = Tq;
            }
        }
        seg_reset(st);
        const bool odd2 = it & 1;
        MqTargets u;
        u.qn = odd2 ? a.q1 : a.q0;
        u.qn_count = &ctl->near_count[it % 3];
        u.act = &ctl->act[it % 3];
        u.farq = fc ? a.far0 : a.far1;
        u.far_count = &ctl->far_count[fc ^ 1];
        u.fmin = ctl->fmin[fc ^ 1];
        u.tag_next = a.base_near + it;
        const uint32_t *fs = fc ? a.far1 : a.far0;
        const uint32_t nf = min(ldcg_u32(&ctl->far_count[fc]), a.n);
        for (uint32_t b = warp * 32; b < nf; b += nwarps * 32) {
            uint32_t i = b + lane;
            bool valid = i < nf;
            uint32_t v = valid ? ldcg_u32(&fs[i]) : 0;
            unsigned long long M = valid ? __ldcg(&a.fmask[v]) : 0ull;
            unsigned long long MS = M & S, moved = 0, dropped = 0;
            for (unsigned long long m = MS; m; m &= m - 1) {
                uint32_t q = __ffsll((long long)m) - 1;
                uint64_t d = mq_label(a.label, v, q, st.lshift[q]) >> 32;
                if (d < st.T[q]) {
                    dropped |= 1ull << q;                  // settled while parked
                } else if (d < st.Tnew[q]) {
                    moved |= 1ull << q;
                } else {
                    atomicMin(&st.fmin[q], (uint32_t)d);
                }
            }
            unsigned long long cleared = moved | dropped;
            if (cleared) {
                atomicAnd(&a.fmask[v], ~cleared);
                for (unsigned long long m = cleared; m; m &= m - 1)
                    atomicSub(&st.fpend[__ffsll((long long)m) - 1], 1);
            }
            bool to_near = false;
            if (moved) {
                atomicOr(&a.nmask[v], moved);
                to_near = atomicExch(&a.stamp_near[v], u.tag_next) != u.tag_next;
            }
            unsigned long long act = warp_or64(moved);
            if (lane == 0 && act) atomicOr(&st.act, act);
            bool keep = valid && (M & ~cleared) != 0;
            if (valid && !keep) a.in_far[v] = 0;
            mq_push_near(a, st, u, to_near, v);
            stage_append(keep, v, st.far_buf, &st.far_n, MQ_FAR_STAGE, u.farq, u.far_count, a.n,
                         &ctl->err);
        }
        seg_flush(st, u, ctl, a.n);
        if (!grid_sync(&ctl->bar, &ctl->err)) { reason = 5; break; }
        if (first) {
            for (uint32_t q = 0; q < MQ_SLOTS; ++q) {
                if (!((S >> q) & 1)) {
                    uint32_t fm = ctl->fmin[fc][q];
                    if (fm != INF32) atomicMin(&ctl->fmin[fc ^ 1][q], fm);
                }
                ctl->fmin[fc][q] = INF32;
            }
            ctl->far_count[fc] = 0;
        }
        if (threadIdx.x < MQ_SLOTS) st.T[threadIdx.x] = st.Tnew[threadIdx.x];
        __syncthreads();
        fc ^= 1;
        if (first) ctl->t_part[4] += gtimer() - tm5;
    }
    if (!infl && reason == 0) reason = 1;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        attempts += __shfl_xor_sync(FULL, attempts, o);
        improved += __shfl_xor_sync(FULL, improved, o);
    }
    if (lane == 0) {
        atomicAdd(&ctl->relax_attempts, attempts);
        atomicAdd(&ctl->relax_improved, improved);
    }
    narrow_miss = warp_or64(narrow_miss);
    if (lane == 0 && narrow_miss) atomicOr(&ctl->slot_narrow, narrow_miss);
    if (first) {
        ctl->it = it;
        ctl->fc = fc;
        ctl->hpass = H & infl;
        ctl->hp_done = hp_done;
        ctl->band0 = band0;
        ctl->pull_sweeps += pull_sweeps;
        ctl->blist = bc;
        ctl->converged |= conv_total;
        ctl->iterations = iters;
        ctl->exit_reason = reason;
        for (uint32_t q = 0; q < MQ_SLOTS; ++q) ctl->T[q] = st.T[q];
        if (reason == 4 && infl) atomicOr(&ctl->err, 0u);   // a capped launch resumes later
    }
}

// ---------------------------------------------------------------------------
// admission of one slot: clear its label/pred column, seed it
// ---------------------------------------------------------------------------

__global__ void mq_clear_column_kernel(uint32_t n, uint32_t *label, uint32_t *pred, uint32_t q) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        label[(uint64_t)v * MQ_SLOTS + q] = INF32;
        pred[(uint64_t)v * MQ_SLOTS + q] = INF32;
    }
}

// Clears the label/pred columns of every slot in `mask` with row-wide,
// coalesced stores (one thread per (vertex, slot) element).
__global__ void mq_clear_rows_kernel(uint32_t n, uint32_t *label, uint32_t *pred,
                                     unsigned long long mask) {
    uint64_t total = (uint64_t)n * MQ_SLOTS;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        if ((mask >> (i & (MQ_SLOTS - 1))) & 1ull) {
            label[i] = INF32;
            pred[i] = INF32;
        }
    }
}

__global__ void mq_seed_kernel(const uint32_t *__restrict__ row_ptr, uint32_t n, const int32_t *seeds,
                               const uint32_t *__restrict__ new_of, uint32_t k, uint32_t q,
                               uint32_t delta, MqState m) {
    MqControl *ctl = m.ctl;
    uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t it = ctl->it;
    const unsigned long long bit = 1ull << q;
    if (r == 0) {
        uint32_t b = 1;
        while (b < 31 && (1u << b) < k) ++b;
        ctl->lshift[q] = b;
        ctl->slot_narrow &= ~bit;
        ctl->T[q] = delta;
        ctl->fmin[0][q] = INF32;
        ctl->fmin[1][q] = INF32;
        ctl->far_pending[q] = 0;
        atomicOr(&ctl->act[it % 3], bit);
        ctl->slot_overflow &= ~bit;
        ctl->hp_done &= ~bit;
        ctl->hpass &= ~bit;
        ctl->band0 |= bit;
    }
    if (r >= k) return;
    uint32_t s = internal_id(new_of, (uint32_t)seeds[r]);
    m.label[(uint64_t)s * MQ_SLOTS + q] = r;          // distance 0, rank r
    m.pred[(uint64_t)s * MQ_SLOTS + q] = SEED_ARC;
    atomicOr(&m.nmask[s], bit);
    uint32_t tag = m.base_near + it;
    if (atomicExch(&m.stamp_near[s], tag) == tag) return;   // already queued for iteration it
    uint32_t slot = atomicAdd(&ctl->near_count[it % 3], 1u);
    if (slot >= n) {
        atomicOr(&ctl->err, ERR_CAPACITY);
        return;
    }
    ((it & 1) ? m.q[1] : m.q[0])[slot] = s;
}

// ---------------------------------------------------------------------------
// batched pred + bridge scan for a set of converged slots
// ---------------------------------------------------------------------------

struct MqScanArgs {
    const uint32_t *__restrict__ row_ptr;
    const uint2 *__restrict__ adj;
    const uint64_t *__restrict__ heavy_chunks;
    uint32_t n_heavy_chunks;
    uint32_t n;
    const uint32_t *label;
    const uint32_t *lshift;          // rank bits of each slot's labels
    uint32_t *pred;
    uint64_t *const *pairtab;
    const uint32_t *k;
    unsigned long long slots;
    MqControl *ctl;
    const uint32_t *orig_of;         // internal -> caller ids (null: identity)
    const uint32_t *orig_row_ptr;
};

// One slot's view of the row being scanned, held by the lane that serves
// the slot: v's label, and the slot's pair table from the first entry of
// v's cell's row of the upper triangle (pair_slot(cv, cv + 1, k)), so that
// the entry of pair (cv, cu) is tab[cu - cv - 1].
struct ScanSlot {
    uint64_t lv;
    uint64_t *tab;
    uint32_t pmin;      // running minimum of v's pred arc
    uint32_t q;
};

__device__ __forceinline__ ScanSlot mq_row_slot(const MqScanArgs &a, uint32_t v, uint32_t q,
                                                uint64_t *tab, uint32_t k, uint64_t lv) {
    ScanSlot r;
    r.lv = lv;
    r.q = q;
    r.pmin = INF32;
    const uint32_t cv = (uint32_t)lv;
    r.tab = lv == INF64 ? tab : tab + pair_slot(cv, cv + 1, k);
    return r;
}

// Arc `arc` = (v, e.x, e.y) for one slot, with lu the slot's label of e.x
// and cbase + arc the caller's index of the arc (bridge keys carry it, as in
// the single-query scan).  A tight same-cell arc lowers r.pmin.
__device__ __forceinline__ void mq_scan_eval(ScanSlot &r, uint32_t arc, uint2 e, uint64_t lu,
                                             uint32_t cbase, unsigned long long &overflow) {
    if (r.lv == INF64 || lu == INF64) {
        if (r.lv != lu) overflow |= 1ull << r.q;
        return;
    }
    const uint32_t cv = (uint32_t)r.lv, cu = (uint32_t)lu;
    const uint64_t dv = r.lv >> 32, du = lu >> 32;
    if (cu == cv) {
        if (du + e.y == dv) r.pmin = min(r.pmin, arc);
    } else if (cv < cu) {
        uint64_t b = dv + e.y + du;
        if (b >= INF32) {
            overflow |= 1ull << r.q;
            return;
        }
        uint64_t key = (b << 32) | (uint32_t)(cbase + arc);
        uint64_t *slot = r.tab + (cu - cv - 1);
        if (key < ldcg_u64(slot))
            atomicMin(reinterpret_cast<unsigned long long *>(slot), (unsigned long long)key);
    }
}

__device__ __forceinline__ void mq_store_pred(const MqScanArgs &a, uint32_t v, const ScanSlot &r,
                                              bool whole_row) {
    if (r.pmin == INF32) return;
    uint32_t *pp = &a.pred[(uint64_t)v * MQ_SLOTS + r.q];
    if (whole_row) *pp = r.pmin;
    else atomicMin(pp, r.pmin);
}

constexpr int SCAN_PAIR_ILP = 2;   // arcs in flight per lane in the slot-pair mode

// The slots a lane serves for the whole launch, with their pair tables and
// sizes loaded once.
struct LaneSlots {
    uint32_t q0, k0, k1;
    uint32_t sh0, sh1;      // rank bits of the slots' labels
    bool h0, h1;
    uint64_t *t0, *t1;
};

// One vertex's arcs [s0, s1) for every slot of the launch.  Each lane keeps
// its slots' row state in registers and stores v's pred once per slot
// (atomically when the row is split into chunks over several warps).
// Over 32 slots: lane l takes slots 2l and 2l + 1 (one 16-byte load of the
// pair's labels per arc), and every lane walks every arc.
// Otherwise lanes are grouped as in the SSSP kernel: a group of g lanes
// takes one arc, lane t of the group the t-th slot; the groups' minima meet
// by shuffles.
__device__ __forceinline__ void mq_scan_row(const MqScanArgs &a, const LaneSlots &ls, uint32_t v,
                                            uint32_t rs, uint32_t s0, uint32_t s1, bool whole_row,
                                            uint32_t cnt, uint32_t gsh,
                                            unsigned long long &overflow) {
    const uint32_t lane = lane_id();
    const uint32_t cbase = caller_arc_base(a.orig_of, a.orig_row_ptr, v, rs);
    const uint32_t *lrow = &a.label[(uint64_t)v * MQ_SLOTS];
    if (cnt > 32) {
        if (!ls.h0 && !ls.h1) return;
        const uint2 lv = __ldg(reinterpret_cast<const uint2 *>(&lrow[ls.q0]));
        ScanSlot r0 = mq_row_slot(a, v, ls.q0, ls.t0, ls.k0, widen_label(lv.x, ls.sh0));
        ScanSlot r1 = mq_row_slot(a, v, ls.q0 + 1, ls.t1, ls.k1, widen_label(lv.y, ls.sh1));
        for (uint32_t j0 = s0; j0 < s1; j0 += SCAN_PAIR_ILP) {
            uint2 e[SCAN_PAIR_ILP];
            uint2 lu[SCAN_PAIR_ILP];
#pragma unroll
            for (int k = 0; k < SCAN_PAIR_ILP; ++k)
                if (j0 + k < s1) e[k] = __ldg(&a.adj[j0 + k]);
#pragma unroll
            for (int k = 0; k < SCAN_PAIR_ILP; ++k)
                if (j0 + k < s1)
                    lu[k] = __ldg(reinterpret_cast<const uint2 *>(&a.label[(uint64_t)e[k].x * MQ_SLOTS + ls.q0]));
#pragma unroll
            for (int k = 0; k < SCAN_PAIR_ILP; ++k) {
                if (j0 + k >= s1) break;
                if (ls.h0) mq_scan_eval(r0, j0 + k, e[k], widen_label(lu[k].x, ls.sh0), cbase, overflow);
                if (ls.h1) mq_scan_eval(r1, j0 + k, e[k], widen_label(lu[k].y, ls.sh1), cbase, overflow);
            }
        }
        if (ls.h0) mq_store_pred(a, v, r0, whole_row);
        if (ls.h1) mq_store_pred(a, v, r1, whole_row);
        return;
    }
    const uint32_t g = 1u << gsh, apr = 32 >> gsh, grp = lane >> gsh;
    const bool has_slot = ls.h0;
    ScanSlot r = mq_row_slot(a, v, ls.q0, ls.t0, ls.k0,
                             has_slot ? widen_label(__ldg(&lrow[ls.q0]), ls.sh0) : INF64);
    for (uint32_t j0 = s0; j0 < s1; j0 += apr * 4) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t arc = j0 + k * apr + grp;
            if (has_slot && arc < s1) {
                uint2 e = __ldg(&a.adj[arc]);
                uint64_t lu = widen_label(__ldg(&a.label[(uint64_t)e.x * MQ_SLOTS + ls.q0]), ls.sh0);
                mq_scan_eval(r, arc, e, lu, cbase, overflow);
            }
        }
    }
    for (uint32_t off = g; off < 32; off <<= 1)
        r.pmin = min(r.pmin, __shfl_xor_sync(FULL, r.pmin, off));
    if (grp == 0 && has_slot) mq_store_pred(a, v, r, whole_row);
}

__global__ void __launch_bounds__(256, 5) mq_scan_kernel(MqScanArgs a) {
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t cnt = (uint32_t)popc64(a.slots);
    const uint32_t gsh = cnt > 16 ? 5 : cnt > 8 ? 4 : cnt > 4 ? 3 : cnt > 2 ? 2 : cnt > 1 ? 1 : 0;
    LaneSlots ls;
    if (cnt > 32) {
        ls.q0 = 2 * lane;
        ls.h0 = (a.slots >> ls.q0) & 1;
        ls.h1 = (a.slots >> (ls.q0 + 1)) & 1;
    } else {
        const uint32_t tl = lane & ((1u << gsh) - 1);
        ls.h0 = tl < cnt;
        ls.h1 = false;
        ls.q0 = ls.h0 ? nth_bit64(a.slots, tl) : 0;
    }
    ls.t0 = ls.h0 ? a.pairtab[ls.q0] : nullptr;
    ls.k0 = ls.h0 ? a.k[ls.q0] : 0;
    ls.t1 = ls.h1 ? a.pairtab[ls.q0 + 1] : nullptr;
    ls.k1 = ls.h1 ? a.k[ls.q0 + 1] : 0;
    ls.sh0 = ls.h0 ? a.lshift[ls.q0] : 1;
    ls.sh1 = ls.h1 ? a.lshift[ls.q0 + 1] : 1;
    const uint32_t n_batches = (a.n + 31) / 32;
    const uint32_t n_work = a.n_heavy_chunks + n_batches;
    unsigned long long overflow = 0;
    for (uint32_t wi = warp; wi < n_work; wi += nwarps) {
        if (wi < a.n_heavy_chunks) {
            uint64_t item = a.heavy_chunks[wi];
            uint32_t v = (uint32_t)(item >> 32), c = (uint32_t)item;
            uint32_t rs = a.row_ptr[v];
            uint32_t s = rs + c * CHUNK;
            uint32_t e = min(a.row_ptr[v + 1], s + CHUNK);
            mq_scan_row(a, ls, v, rs, s, e, false, cnt, gsh, overflow);
        } else {
            uint32_t v0 = (wi - a.n_heavy_chunks) * 32;
            uint32_t vl = v0 + lane;
            uint32_t rs = vl < a.n ? a.row_ptr[vl] : 0;
            uint32_t re = vl < a.n ? a.row_ptr[vl + 1] : 0;
            for (uint32_t l = 0; l < 32 && v0 + l < a.n; ++l) {
                uint32_t s = __shfl_sync(FULL, rs, l), e = __shfl_sync(FULL, re, l);
                if (e - s >= HEAVY_DEG) continue;          // covered by the chunk list
                mq_scan_row(a, ls, v0 + l, s, s, e, true, cnt, gsh, overflow);
            }
        }
    }
    overflow = warp_or64(overflow);
    if (lane == 0 && overflow) atomicOr(&a.ctl->slot_overflow, overflow);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

template <class T>
static cudaError_t mq_dalloc(T *&p, uint64_t count) {
    if (count == 0) count = 1;
    return cudaMalloc((void **)&p, count * sizeof(T));
}

cudaError_t mq_alloc(const DevGraph &g, MqState &m, cudaStream_t s) {
    uint32_t n = g.n;
    m.n = n;
    cudaError_t e;
#define MA(ptr, cnt) if ((e = mq_dalloc(ptr, cnt)) != cudaSuccess) return e
    MA(m.label, (uint64_t)n * MQ_SLOTS);      // 32-bit labels
    MA(m.pred, (uint64_t)n * MQ_SLOTS);
    MA(m.nmask, n);
    MA(m.fmask, n);
    MA(m.stamp_near, n);
    MA(m.in_far, n);
    for (int i = 0; i < 2; ++i) {
        MA(m.q[i], n);
        MA(m.far[i], n);
    }
    MA(m.item_mask, 2 * (uint64_t)n);
    MA(m.item_pre, 2 * (uint64_t)n);
    MA(m.bmask, n);
    for (int i = 0; i < 3; ++i) MA(m.bl[i], n);
    MA(m.bsum, MQ_MAX_BLOCKS);
    MA(m.ctl, 1);
    MA(m.d_pairtab, MQ_SLOTS);
    MA(m.d_k, MQ_SLOTS);
#undef MA
    if ((e = mq_reset(m, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(m.d_pairtab, 0, MQ_SLOTS * sizeof(uint64_t *), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(m.d_k, 0, MQ_SLOTS * 4, s)) != cudaSuccess) return e;
    m.base_near = 1;
    return cudaSuccess;
}

cudaError_t mq_reset(MqState &m, cudaStream_t s) {
    const size_t n = m.n;
    cudaError_t e = cudaMemsetAsync(m.nmask, 0, n * 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(m.fmask, 0, n * 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(m.bmask, 0, n * 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(m.stamp_near, 0, n * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(m.in_far, 0, n * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(m.ctl, 0, sizeof(MqControl), s);
    return e;
}

void mq_free(MqState &m) {
    void *bufs[] = {m.label, m.pred, m.nmask, m.fmask, m.stamp_near, m.in_far, m.q[0], m.q[1],
                    m.item_mask, m.item_pre, m.bsum, m.far[0], m.far[1], m.ctl, m.d_pairtab,
                    m.d_k, m.bmask, m.bl[0], m.bl[1], m.bl[2]};
    for (void *p : bufs)
        if (p) cudaFree(p);
    for (int q = 0; q < MQ_SLOTS; ++q) {
        if (m.pairtab[q]) cudaFree(m.pairtab[q]);
        if (m.seeds[q]) cudaFree(m.seeds[q]);
    }
    m = MqState();
}

int mq_occupancy(int threads) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, mq_sssp_kernel, threads, 0) != cudaSuccess)
        return 0;
    return nb;
}

cudaError_t mq_launch_clear(const DevGraph &g, MqState &m, unsigned long long mask,
                            cudaStream_t s) {
    if (!mask) return cudaSuccess;
    if (__builtin_popcountll(mask) >= 8) {
        mq_clear_rows_kernel<<<current_sm_count() * 16, 256, 0, s>>>(g.n, m.label, m.pred, mask);
    } else {
        unsigned grid = (unsigned)std::min<uint64_t>((g.n + 255) / 256, (uint64_t)current_sm_count() * 16);
        for (unsigned long long mm = mask; mm; mm &= mm - 1)
            mq_clear_column_kernel<<<grid, 256, 0, s>>>(g.n, m.label, m.pred,
                                                        (uint32_t)__builtin_ctzll(mm));
    }
    return cudaGetLastError();
}

cudaError_t mq_launch_seed(const DevGraph &g, MqState &m, int q, uint32_t k, uint32_t delta,
                           cudaStream_t s) {
    mq_seed_kernel<<<(k + 255) / 256, 256, 0, s>>>(g.row_ptr, g.n, m.seeds[q], g.new_of, k, (uint32_t)q,
                                                    delta, m);
    return cudaGetLastError();
}

cudaError_t mq_launch_sssp(const DevGraph &g, MqState &m, int blocks, uint32_t delta, uint32_t pull,
                           uint32_t max_iters, uint32_t yield, const uint32_t *doorbell,
                           cudaStream_t s) {
    MqArgs a;
    a.row_ptr = g.row_ptr;
    a.adj = g.adj;
    a.n = g.n;
    a.label = m.label;
    a.nmask = m.nmask;
    a.fmask = m.fmask;
    a.stamp_near = m.stamp_near;
    a.in_far = m.in_far;
    a.q0 = m.q[0];
    a.q1 = m.q[1];
    a.item_mask = m.item_mask;
    a.item_pre = m.item_pre;
    a.bsum = m.bsum;
    a.far0 = m.far[0];
    a.far1 = m.far[1];
    a.bmask = m.bmask;
    a.bl0 = m.bl[0];
    a.bl1 = m.bl[1];
    a.bl2 = m.bl[2];
    a.defer = delta <= g.max_w ? 1u : 0u;
    a.lend = active_lend(g, delta);
    if (a.lend) a.adj = g.adj_w;        // rows partitioned by weight class
    a.pull = a.defer ? pull : 0u;
    a.ctl = m.ctl;
    a.doorbell = doorbell;
    a.delta = delta;
    a.base_near = m.base_near;
    a.max_iters = max_iters;
    a.yield = yield;
    cudaError_t e = cudaMemsetAsync(&m.ctl->bar, 0, sizeof(GridBarrier), s);
    if (e != cudaSuccess) return e;
    if (blocks > MQ_MAX_BLOCKS) blocks = MQ_MAX_BLOCKS;
    void *args[] = {&a};
    return cudaLaunchCooperativeKernel((const void *)mq_sssp_kernel, dim3(blocks), dim3(256), args,
                                       0, s);
}

cudaError_t mq_launch_scan(const DevGraph &g, MqState &m, unsigned long long slots,
                           cudaStream_t s) {
    if (!slots) return cudaSuccess;
    MqScanArgs a;
    a.row_ptr = g.row_ptr;
    a.adj = g.adj;
    a.heavy_chunks = g.heavy_chunks;
    a.n_heavy_chunks = g.n_heavy_chunks;
    a.n = g.n;
    a.label = m.label;
    a.lshift = m.ctl->lshift;
    a.pred = m.pred;
    a.pairtab = m.d_pairtab;
    a.k = m.d_k;
    a.slots = slots;
    a.ctl = m.ctl;
    a.orig_of = g.orig_of;
    a.orig_row_ptr = g.orig_row_ptr;
    uint64_t work = (uint64_t)g.n_heavy_chunks + (g.n + 31) / 32;
    uint64_t blocks = std::max<uint64_t>(1, std::min<uint64_t>((work + 7) / 8, (uint64_t)current_sm_count() * 32));
    mq_scan_kernel<<<(unsigned)blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace stn
