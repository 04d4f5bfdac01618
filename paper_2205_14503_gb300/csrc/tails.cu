// Tails of the multi-query engine for all retiring slots at once: Steps 3-7
// of Algorithm 2 (MST of each slot's distance graph G'_1, expansion of the
// MST bridges along the predecessor chains, D(G_S)) with one launch per step
// over every retiring slot instead of the single-query kernels slot by slot.
//
//  * compaction: every slot's pair table is cut into tiles numbered across
//    all retiring slots; the non-empty entries of each table land, in slot
//    order, in that slot's segment of one concatenated pair list;
//  * MST: one block per slot runs Boruvka on its segment under the strict
//    order (b, rank a, rank b) (block barriers only), so each slot's MST is
//    the unique one Kruskal finds on the same order;
//  * expansion: two walkers per MST pair, as in the single-query path, on
//    the slot's predecessor column; the walkers of all slots share one mark
//    array with a tag per slot, so a walker stops only where its own slot
//    already walked (a vertex in several slots' trees can make a walker
//    repeat a suffix: a duplicate edge, never a missing one);
//  * one radix sort over (slot, u, v) keys of every emitted edge puts each
//    slot's edges in ascending (u, v) order with duplicates adjacent; a
//    pass drops the duplicates and sums each slot's D(G_S).
#include <algorithm>
#include <cstring>
#include <vector>

#include "engine.h"
#include "multi.h"

namespace stn {

constexpr uint32_t BT_THREADS = 256;
constexpr uint32_t BT_PER_THREAD = 8;
constexpr uint32_t BT_TILE = BT_THREADS * BT_PER_THREAD;

// Slot index of global tile `tile`: the last slot whose first tile is at or
// before it (r <= 64 slots, tile0 ascending).
__device__ __forceinline__ uint32_t bt_slot_of_tile(const TailSlot *slots, uint32_t r,
                                                    uint64_t tile) {
    uint32_t lo = 0, hi = r;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) / 2;
        if (slots[mid].tile0 <= tile) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(BT_THREADS) bt_count_kernel(const TailSlot *__restrict__ slots,
                                                              uint32_t r,
                                                              uint32_t *__restrict__ tile_cnt) {
    __shared__ uint32_t wsum[BT_THREADS / 32];
    const uint32_t i = bt_slot_of_tile(slots, r, blockIdx.x);
    const TailSlot sl = slots[i];
    const uint64_t base = (blockIdx.x - sl.tile0) * (uint64_t)BT_TILE +
                          (uint64_t)threadIdx.x * BT_PER_THREAD;
    uint32_t c = 0;
#pragma unroll
    for (uint32_t j = 0; j < BT_PER_THREAD; ++j)
        if (base + j < sl.n_slots && sl.pairtab[base + j] != INF64) ++c;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
    if (lane_id() == 0) wsum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (uint32_t w = 0; w < BT_THREADS / 32; ++w) t += wsum[w];
        tile_cnt[blockIdx.x] = t;
    }
}

// One block: exclusive scan of the tile counts; each slot's segment
// (pair0, n_pairs) and the total in ctl->n_pairs.
__global__ void __launch_bounds__(1024) bt_scan_kernel(uint32_t *tile_cnt, uint32_t n_tiles,
                                                       const TailSlot *__restrict__ slots,
                                                       uint32_t r, TailOut *out, Control *ctl) {
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < n_tiles; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t x = i < n_tiles ? tile_cnt[i] : 0;
        const uint32_t incl = warp_inclusive_scan(x);
        if (lane_id() == 31) wsum[threadIdx.x >> 5] = incl;
        __syncthreads();
        if (threadIdx.x < 32) {
            const uint32_t ws = wsum[threadIdx.x];
            wsum[threadIdx.x] = warp_inclusive_scan(ws) - ws;
        }
        __syncthreads();
        const uint32_t excl = carry + wsum[threadIdx.x >> 5] + incl - x;
        if (i < n_tiles) tile_cnt[i] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + x;
        __syncthreads();
    }
    if (threadIdx.x < r) {
        const uint32_t i = threadIdx.x;
        const uint32_t p0 = tile_cnt[slots[i].tile0];
        const uint32_t p1 = i + 1 < r ? tile_cnt[slots[i + 1].tile0] : carry;
        out[i].pair0 = p0;
        out[i].n_pairs = p1 - p0;
    }
    if (threadIdx.x == 0) ctl->n_pairs = carry;
}

struct BtPairs {
    uint64_t *key;       // (b << 32) | table slot: ordered by (b, rank a, rank b)
    uint32_t *ra, *rb, *arc, *mst, *owner;
};

__global__ void __launch_bounds__(BT_THREADS) bt_write_kernel(const TailSlot *__restrict__ slots,
                                                              uint32_t r,
                                                              const uint32_t *__restrict__ tile_off,
                                                              BtPairs p, uint32_t cap,
                                                              Control *ctl) {
    __shared__ uint32_t wsum[BT_THREADS / 32];
    const uint32_t i = bt_slot_of_tile(slots, r, blockIdx.x);
    const TailSlot sl = slots[i];
    const uint64_t base = (blockIdx.x - sl.tile0) * (uint64_t)BT_TILE +
                          (uint64_t)threadIdx.x * BT_PER_THREAD;
    uint64_t vals[BT_PER_THREAD];
    uint32_t c = 0;
#pragma unroll
    for (uint32_t j = 0; j < BT_PER_THREAD; ++j) {
        vals[j] = base + j < sl.n_slots ? sl.pairtab[base + j] : INF64;
        if (vals[j] != INF64) ++c;
    }
    const uint32_t incl = warp_inclusive_scan(c);
    if (lane_id() == 31) wsum[threadIdx.x >> 5] = incl;
    __syncthreads();
    if (threadIdx.x < 32) {
        const uint32_t ws = threadIdx.x < BT_THREADS / 32 ? wsum[threadIdx.x] : 0;
        const uint32_t wi = warp_inclusive_scan(ws);
        if (threadIdx.x < BT_THREADS / 32) wsum[threadIdx.x] = wi - ws;
    }
    __syncthreads();
    uint32_t o = tile_off[blockIdx.x] + wsum[threadIdx.x >> 5] + incl - c;
#pragma unroll
    for (uint32_t j = 0; j < BT_PER_THREAD; ++j) {
        if (vals[j] == INF64) continue;
        if (o >= cap) {
            atomicOr(&ctl->err, ERR_CAPACITY);
            break;
        }
        const uint64_t slot = base + j;
        uint32_t ra, rb;
        slot_to_pair(slot, sl.k, ra, rb);
        p.key[o] = (vals[j] & 0xFFFFFFFF00000000ull) | slot;
        p.ra[o] = ra;
        p.rb[o] = rb;
        p.arc[o] = (uint32_t)vals[j];
        p.mst[o] = 0;
        p.owner[o] = i;
        ++o;
    }
}

// One block per slot: Boruvka on the slot's segment with block barriers.
// comp / hook / best hold the slot's k entries at comp0.
__global__ void __launch_bounds__(512) bt_mst_kernel(const TailSlot *__restrict__ slots,
                                                     BtPairs p, TailOut *out, uint32_t *comp_all,
                                                     uint32_t *hook_all,
                                                     unsigned long long *best_all,
                                                     Control *ctl) {
    __shared__ int any_s;
    const TailSlot sl = slots[blockIdx.x];
    const uint32_t k = sl.k;
    const uint32_t e0 = out[blockIdx.x].pair0, E = out[blockIdx.x].n_pairs;
    uint32_t *comp = comp_all + sl.comp0, *hook = hook_all + sl.comp0;
    unsigned long long *best = best_all + sl.comp0;
    for (uint32_t c = threadIdx.x; c < k; c += blockDim.x) comp[c] = c;
    __syncthreads();
    for (int round = 0;; ++round) {
        if (round >= 64) {
            if (threadIdx.x == 0) atomicOr(&ctl->err, ERR_TIMEOUT);
            return;
        }
        for (uint32_t c = threadIdx.x; c < k; c += blockDim.x) {
            best[c] = INF64;
            hook[c] = c;
        }
        if (threadIdx.x == 0) any_s = 0;
        __syncthreads();
        // lightest edge leaving every component
        bool any = false;
        for (uint32_t j = e0 + threadIdx.x; j < e0 + E; j += blockDim.x) {
            const uint32_t ca = comp[p.ra[j]], cb = comp[p.rb[j]];
            if (ca == cb) continue;
            const unsigned long long key = p.key[j];
            atomicMin(&best[ca], key);
            atomicMin(&best[cb], key);
            any = true;
        }
        if (any) any_s = 1;
        __syncthreads();
        if (!any_s) break;
        // hook each component along its lightest edge; mark the edge
        for (uint32_t j = e0 + threadIdx.x; j < e0 + E; j += blockDim.x) {
            const uint32_t ca = comp[p.ra[j]], cb = comp[p.rb[j]];
            if (ca == cb) continue;
            const unsigned long long key = p.key[j];
            if (best[ca] == key) {
                hook[ca] = cb;
                p.mst[j] = 1;
            }
            if (best[cb] == key) {
                hook[cb] = ca;
                p.mst[j] = 1;
            }
        }
        __syncthreads();
        // two components that chose each other: the smaller id becomes root
        for (uint32_t c = threadIdx.x; c < k; c += blockDim.x) {
            const uint32_t h = hook[c];
            if (h != c && hook[h] == c && c < h) hook[c] = c;
        }
        __syncthreads();
        for (uint32_t x = threadIdx.x; x < k; x += blockDim.x) {
            uint32_t c = comp[x];
            for (uint32_t steps = 0; steps < k; ++steps) {
                const uint32_t h = hook[c];
                if (h == c) break;
                c = h;
            }
            comp[x] = c;
        }
        __syncthreads();
    }
    uint32_t cnt = 0;
    for (uint32_t j = e0 + threadIdx.x; j < e0 + E; j += blockDim.x) cnt += p.mst[j];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) cnt += __shfl_xor_sync(FULL, cnt, o);
    if (lane_id() == 0 && cnt) atomicAdd(&out[blockIdx.x].n_mst, cnt);
}

__device__ __forceinline__ uint32_t bt_arc_owner(const uint32_t *row_ptr, uint32_t n,
                                                 uint32_t arc) {
    uint32_t lo = 0, hi = n;        // largest v with row_ptr[v] <= arc
    while (hi - lo > 1) {
        const uint32_t mid = lo + (hi - lo) / 2;
        if (row_ptr[mid] <= arc) lo = mid; else hi = mid;
    }
    return lo;
}

struct BtExpandArgs {
    const uint32_t *__restrict__ row_ptr;
    const uint2 *__restrict__ adj;
    const uint32_t *__restrict__ orig_of;
    const uint32_t *__restrict__ new_of;
    const uint32_t *__restrict__ orig_row_ptr;
    uint32_t n;
    const TailSlot *slots;
    BtPairs p;
    const uint32_t *pred;       // the engine's pred columns, MQ_SLOTS per vertex
    uint32_t *mark;
    uint32_t tag0;              // slot i marks with tag0 + i
    uint32_t nbits;
    uint32_t shift;             // 2 * nbits: the slot field of a key
    uint64_t *key;
    uint32_t *w;
    uint32_t cap;
    Control *ctl;
};

// Two walkers per MST pair (one warp-uniform loop; edges are appended with
// one atomic per warp step): walker 0 emits the bridge, then both walk
// pred() to their seeds.
__global__ void __launch_bounds__(256) bt_expand_kernel(BtExpandArgs a) {
    const uint32_t E = ldcg_u32(&a.ctl->n_pairs);
    const uint64_t total = 2ull * E;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < total;
         base += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t t = base + threadIdx.x;
        const uint32_t j = (uint32_t)(t >> 1), side = (uint32_t)(t & 1);
        bool active = t < total && a.p.mst[j];
        uint32_t x = 0, q = 0, tag = 0, owner = 0;
        uint32_t eu = 0, ev = 0, ew = 0;
        bool have = false;
        if (active) {
            owner = a.p.owner[j];
            q = a.slots[owner].q;
            tag = a.tag0 + owner;
            const uint32_t carc = a.p.arc[j];
            uint32_t tail, arc;
            if (a.orig_of) {
                const uint32_t ct = bt_arc_owner(a.orig_row_ptr, a.n, carc);
                tail = a.new_of[ct];
                arc = a.row_ptr[tail] + (carc - a.orig_row_ptr[ct]);
            } else {
                tail = bt_arc_owner(a.row_ptr, a.n, carc);
                arc = carc;
            }
            const uint2 e = a.adj[arc];
            x = e.x;
            if (side == 0) {
                x = tail;
                eu = caller_id(a.orig_of, tail);
                ev = caller_id(a.orig_of, e.x);
                ew = e.y;
                have = true;
            }
        }
        for (uint32_t steps = 0;; ++steps) {
            const uint32_t slot = warp_append(have, &a.ctl->n_tree, a.cap, &a.ctl->err);
            if (slot != INF32) {
                const uint32_t lo = min(eu, ev), hi = max(eu, ev);
                a.key[slot] = ((uint64_t)owner << a.shift) | ((uint64_t)lo << a.nbits) | hi;
                a.w[slot] = ew;
            }
            have = false;
            if (active) {
                const uint32_t pa = a.pred[(uint64_t)x * MQ_SLOTS + q];
                if (pa == SEED_ARC || pa == INF32 || steps >= a.n) {
                    active = false;
                } else {
                    const uint32_t old = atomicExch(&a.mark[x], tag);
                    const uint2 pe = a.adj[pa];
                    if (old == tag) {
                        active = false;        // this slot walked on from here already
                    } else {
                        eu = caller_id(a.orig_of, x);
                        ev = caller_id(a.orig_of, pe.x);
                        ew = pe.y;
                        have = true;
                        x = pe.x;
                    }
                }
            }
            if (!__any_sync(FULL, active || have)) break;
        }
    }
}

// Over the sorted keys: each slot's edge count and D(G_S), duplicates skipped.
__global__ void __launch_bounds__(256) bt_totals_kernel(const uint64_t *__restrict__ key,
                                                        const uint32_t *__restrict__ w,
                                                        uint32_t shift, TailOut *out,
                                                        Control *ctl, uint32_t cap) {
    __shared__ uint32_t s_cnt[MQ_SLOTS];
    __shared__ unsigned long long s_tot[MQ_SLOTS];
    if (threadIdx.x < MQ_SLOTS) {
        s_cnt[threadIdx.x] = 0;
        s_tot[threadIdx.x] = 0;
    }
    __syncthreads();
    const uint32_t N = min(ldcg_u32(&ctl->n_tree), cap);
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
        const uint64_t kj = key[j];
        if (j > 0 && key[j - 1] == kj) continue;
        const uint32_t i = (uint32_t)(kj >> shift);
        if (i >= MQ_SLOTS) continue;
        atomicAdd(&s_cnt[i], 1u);
        atomicAdd(&s_tot[i], (unsigned long long)w[j]);
    }
    __syncthreads();
    if (threadIdx.x < MQ_SLOTS && s_cnt[threadIdx.x]) {
        atomicAdd(&out[threadIdx.x].n_edges, s_cnt[threadIdx.x]);
        atomicAdd(&out[threadIdx.x].total, s_tot[threadIdx.x]);
    }
}

// Grows a group of arrays that share one capacity (in elements) to at
// least `need`, with some headroom; a failed allocation leaves capacity 0.
template <class... T>
static cudaError_t bt_grow(uint64_t &cap, uint64_t need, T *&...ptrs) {
    if (need <= cap) return cudaSuccess;
    const uint64_t c = std::max<uint64_t>(need + need / 4, 1024);
    cudaError_t e = cudaSuccess;
    auto one = [&](auto *&p) {
        if (p) cudaFree(p);
        p = nullptr;
        if (e == cudaSuccess) e = cudaMalloc((void **)&p, c * sizeof(*p));
    };
    (one(ptrs), ...);
    cap = e == cudaSuccess ? c : 0;
    return e;
}

void tail_ws_free(TailWs &t) {
    void *d[] = {t.d_slots, t.d_out, t.tile_cnt, t.e_key, t.e_ra, t.e_rb, t.e_arc, t.e_mst,
                 t.e_owner, t.comp, t.hook, t.best, t.key0, t.key1, t.w0, t.w1, t.hist, t.ctl};
    for (void *p : d)
        if (p) cudaFree(p);
    if (t.h_slots) cudaFreeHost(t.h_slots);
    if (t.h_out) cudaFreeHost(t.h_out);
    if (t.h_ctl) cudaFreeHost(t.h_ctl);
    t = TailWs();
}

static cudaError_t bt_setup(TailWs &t) {
    if (t.ctl) return cudaSuccess;
    cudaError_t e = cudaMalloc((void **)&t.d_slots, MQ_SLOTS * sizeof(TailSlot));
    if (e == cudaSuccess) e = cudaMalloc((void **)&t.d_out, MQ_SLOTS * sizeof(TailOut));
    if (e == cudaSuccess) e = cudaMalloc((void **)&t.hist, 64 * 256 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc((void **)&t.ctl, sizeof(Control));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&t.h_slots, MQ_SLOTS * sizeof(TailSlot));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&t.h_out, MQ_SLOTS * sizeof(TailOut));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&t.h_ctl, sizeof(Control));
    return e;
}

#define BT_CK(call)                                                           \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) {                                              \
            cudaGetLastError();                                               \
            api_set_error(std::string("batched tails: ") + cudaGetErrorString(e_)); \
            return e_ == cudaErrorMemoryAllocation ? STEINER_ENOMEM : STEINER_ECUDA; \
        }                                                                     \
    } while (0)

int run_batched_tails(steiner_graph *G, MqState &m, TailWs &t, const int *qs,
                      const uint32_t *ks, int r, steiner_result_t *res) {
    if (r <= 0) return STEINER_OK;
    if (r > MQ_SLOTS) return STEINER_EINVAL;
    const DevGraph &g = api_graph(G);
    cudaStream_t s = api_stream(G);
    BT_CK(bt_setup(t));
    uint64_t tiles = 0, comps = 0;
    for (int i = 0; i < r; ++i) {
        TailSlot &sl = t.h_slots[i];
        sl.pairtab = m.pairtab[qs[i]];
        sl.n_slots = (uint64_t)ks[i] * (ks[i] - 1) / 2;
        sl.tile0 = tiles;
        sl.k = ks[i];
        sl.q = (uint32_t)qs[i];
        sl.comp0 = (uint32_t)comps;
        sl.pad = 0;
        tiles += std::max<uint64_t>(1, (sl.n_slots + BT_TILE - 1) / BT_TILE);
        comps += ks[i];
    }
    if (tiles > 0x7FFFFFFFull || comps > 0xFFFFFFFFull) return STEINER_ENOMEM;
    BT_CK(bt_grow(t.tile_cap, tiles, t.tile_cnt));
    BT_CK(bt_grow(t.comp_cap, comps, t.comp, t.hook, t.best));
    BT_CK(cudaMemcpyAsync(t.d_slots, t.h_slots, r * sizeof(TailSlot), cudaMemcpyHostToDevice, s));
    BT_CK(cudaMemsetAsync(t.d_out, 0, MQ_SLOTS * sizeof(TailOut), s));
    BT_CK(cudaMemsetAsync(t.ctl, 0, sizeof(Control), s));
    bt_count_kernel<<<(unsigned)tiles, BT_THREADS, 0, s>>>(t.d_slots, r, t.tile_cnt);
    bt_scan_kernel<<<1, 1024, 0, s>>>(t.tile_cnt, (uint32_t)tiles, t.d_slots, r, t.d_out, t.ctl);
    BT_CK(cudaGetLastError());
    BT_CK(cudaMemcpyAsync(t.h_ctl, t.ctl, sizeof(Control), cudaMemcpyDeviceToHost, s));
    BT_CK(cudaStreamSynchronize(s));
    const uint32_t n_pairs = t.h_ctl->n_pairs;
    BT_CK(bt_grow(t.e_cap, n_pairs, t.e_key, t.e_ra, t.e_rb, t.e_arc, t.e_mst, t.e_owner));
    // edge capacity: every slot's tree has at most n - 1 edges, and the
    // walkers of a typical batch emit a few edges per seed; start at 4M and
    // grow after a capacity miss
    if (!t.tree_cap) t.tree_cap = std::min<uint64_t>(1ull << 22, (uint64_t)g.n * r + 64);
    BT_CK(bt_grow(t.key_cap, t.tree_cap, t.key0, t.key1, t.w0, t.w1));
    const uint32_t cap = (uint32_t)std::min<uint64_t>(t.key_cap, 0xFFFFFFF0ull);
    BtPairs p{t.e_key, t.e_ra, t.e_rb, t.e_arc, t.e_mst, t.e_owner};
    bt_write_kernel<<<(unsigned)tiles, BT_THREADS, 0, s>>>(t.d_slots, r, t.tile_cnt, p,
                                                            (uint32_t)t.e_cap, t.ctl);
    bt_mst_kernel<<<r, 512, 0, s>>>(t.d_slots, p, t.d_out, t.comp, t.hook, t.best, t.ctl);
    BT_CK(cudaGetLastError());
    uint32_t *mark = nullptr;
    const uint32_t tag0 = api_reserve_mark_tags(G, (uint32_t)r, &mark);
    if (!mark) return STEINER_ENOMEM;
    const uint32_t nbits = api_nbits(G);
    uint32_t rbits = 1;
    while ((1u << rbits) < (uint32_t)r) ++rbits;
    if (2 * nbits + rbits > 64) return STEINER_ENOMEM;    // keys do not fit: one slot at a time
    BtExpandArgs xa{g.row_ptr, g.adj, g.orig_of, g.new_of, g.orig_row_ptr, g.n, t.d_slots, p,
                    m.pred, mark, tag0, nbits, 2 * nbits, t.key0, t.w0, cap, t.ctl};
    const uint64_t walkers = 2ull * n_pairs;
    const unsigned xb = (unsigned)std::max<uint64_t>(
        1, std::min<uint64_t>((walkers + 255) / 256, (uint64_t)current_sm_count() * 8));
    bt_expand_kernel<<<xb, 256, 0, s>>>(xa);
    BT_CK(cudaGetLastError());
    BT_CK(launch_sort_keys(t.key0, t.key1, t.w0, t.w1, t.hist, cap, 2 * nbits + rbits, t.ctl, s));
    bt_totals_kernel<<<current_sm_count() * 2, 256, 0, s>>>(t.key0, t.w0, 2 * nbits, t.d_out,
                                                            t.ctl, cap);
    BT_CK(cudaGetLastError());
    BT_CK(cudaMemcpyAsync(t.h_ctl, t.ctl, sizeof(Control), cudaMemcpyDeviceToHost, s));
    BT_CK(cudaMemcpyAsync(t.h_out, t.d_out, r * sizeof(TailOut), cudaMemcpyDeviceToHost, s));
    BT_CK(cudaStreamSynchronize(s));
    const Control &c = *t.h_ctl;
    if (c.err & ERR_CAPACITY) {
        // more edges than the buffer holds: grow it for next time, and let
        // the caller run these slots one at a time
        t.tree_cap = std::min<uint64_t>(t.tree_cap * 4, 0xFFFFFFF0ull);
        return STEINER_ENOMEM;
    }
    if (c.err & (ERR_TIMEOUT | ERR_BARRIER)) {
        api_set_error("batched tails: a device loop or barrier hit its cap");
        return STEINER_ETIMEOUT;
    }
    const uint32_t N = std::min(c.n_tree, cap);
    std::vector<uint64_t> keys(N);
    std::vector<uint32_t> ws(N);
    if (N) {
        BT_CK(cudaMemcpyAsync(keys.data(), t.key0, (size_t)N * 8, cudaMemcpyDeviceToHost, s));
        BT_CK(cudaMemcpyAsync(ws.data(), t.w0, (size_t)N * 4, cudaMemcpyDeviceToHost, s));
        BT_CK(cudaStreamSynchronize(s));
    }
    for (int i = 0; i < r; ++i) {
        res[i].edges = nullptr;
        res[i].n_edges = 0;
        res[i].total = 0;
        res[i].status = STEINER_OK;
        const uint32_t ne = t.h_out[i].n_edges;
        if (ne) {
            res[i].edges = (steiner_edge_t *)malloc((size_t)ne * sizeof(steiner_edge_t));
            if (!res[i].edges) {
                for (int j = 0; j <= i; ++j) {
                    free(res[j].edges);
                    res[j].edges = nullptr;
                }
                api_set_error("host allocation of a result failed");
                return STEINER_ENOMEM;
            }
        }
    }
    const uint64_t vmask = (1ull << nbits) - 1;
    for (uint32_t j = 0; j < N; ++j) {
        if (j && keys[j] == keys[j - 1]) continue;
        const uint32_t i = (uint32_t)(keys[j] >> (2 * nbits));
        if (i >= (uint32_t)r || res[i].n_edges >= t.h_out[i].n_edges) continue;
        steiner_edge_t &e = res[i].edges[res[i].n_edges++];
        e.u = (uint32_t)((keys[j] >> nbits) & vmask);
        e.v = (uint32_t)(keys[j] & vmask);
        e.w = ws[j];
    }
    for (int i = 0; i < r; ++i) {
        res[i].total = t.h_out[i].total;
        if (ks[i] > 1 && t.h_out[i].n_mst + 1 < ks[i]) {
            res[i].status = STEINER_EDISCONNECTED;
            api_set_error("seeds lie in more than one component");
        }
    }
    return STEINER_OK;
}

}  // namespace stn
