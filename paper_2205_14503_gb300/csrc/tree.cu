// The tail of Algorithm 2 on the device.
//
//  * Step 3, MST of the distance graph G'_1: Boruvka rounds on the compacted
//    pair list.  Each edge's key is (b << 32) | slot; the slot increases with
//    (rank a, rank b), so keys are distinct and ordered by (b, rank a,
//    rank b).  Under a strict total order the MST is unique, hence equal to
//    the tree Kruskal would build on the same order (the paper runs Prim;
//    its ties are unspecified).
//  * Steps 4-6 (Algorithm 6): the bridge of every MST pair joins the tree
//    and both of its ends walk pred() to their seeds, adding (pred(x), x);
//    a per-vertex stamp stops a walk where another has already been, which
//    also keeps each edge once (the paper's EDGE_PRUNING_COLL keeps one
//    bridge per pair; here the pair table already holds exactly one).
//  * Step 7: the edges are sorted by (u, v) with a cooperative LSD radix
//    sort and their weights summed into D(G_S).
#include "internal.h"

namespace stn {

// ---------------------------------------------------------------------------
// Boruvka MST (cooperative, bounded barriers)
// ---------------------------------------------------------------------------

struct MstArgs {
    const uint64_t *e_key;
    const uint32_t *e_ra;
    const uint32_t *e_rb;
    uint32_t *e_mst;
    uint32_t *comp;
    uint32_t *hook;
    unsigned long long *best;
    uint32_t k;
    Control *ctl;
};

__global__ void __launch_bounds__(512) mst_kernel(MstArgs a) {
    Control *ctl = a.ctl;
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t nth = gridDim.x * blockDim.x;
    const uint32_t E = ldcg_u32(&ctl->n_pairs);
    const bool first = tid == 0;
    for (uint32_t r = tid; r < a.k; r += nth) a.comp[r] = r;
    if (!grid_sync(&ctl->bar2, &ctl->err)) return;
    for (int round = 0;; ++round) {
        if (round >= 64) {
            if (first) atomicOr(&ctl->err, ERR_TIMEOUT);
            return;
        }
        for (uint32_t c = tid; c < a.k; c += nth) {
            a.best[c] = INF64;
            a.hook[c] = c;
        }
        if (first) ctl->mst_any = 0;
        if (!grid_sync(&ctl->bar2, &ctl->err)) return;
        // lightest edge leaving every component
        bool any = false;
        for (uint32_t j = tid; j < E; j += nth) {
            uint32_t ca = ldcg_u32(&a.comp[a.e_ra[j]]), cb = ldcg_u32(&a.comp[a.e_rb[j]]);
            if (ca == cb) continue;
            unsigned long long key = a.e_key[j];
            atomicMin(&a.best[ca], key);
            atomicMin(&a.best[cb], key);
            any = true;
        }
        if (__any_sync(FULL, any) && lane_id() == 0) atomicExch(&ctl->mst_any, 1u);
        if (!grid_sync(&ctl->bar2, &ctl->err)) return;
        if (ldcg_u32(&ctl->mst_any) == 0) break;
        // hook each component along its lightest edge; mark the edge
        for (uint32_t j = tid; j < E; j += nth) {
            uint32_t ca = ldcg_u32(&a.comp[a.e_ra[j]]), cb = ldcg_u32(&a.comp[a.e_rb[j]]);
            if (ca == cb) continue;
            unsigned long long key = a.e_key[j];
            if (__ldcg(&a.best[ca]) == key) {
                a.hook[ca] = cb;
                a.e_mst[j] = 1;
            }
            if (__ldcg(&a.best[cb]) == key) {
                a.hook[cb] = ca;
                a.e_mst[j] = 1;
            }
        }
        if (!grid_sync(&ctl->bar2, &ctl->err)) return;
        // two components that chose each other: the smaller id becomes root
        for (uint32_t c = tid; c < a.k; c += nth) {
            uint32_t p = ldcg_u32(&a.hook[c]);
            if (p != c && ldcg_u32(&a.hook[p]) == c && c < p) a.hook[c] = c;
        }
        if (!grid_sync(&ctl->bar2, &ctl->err)) return;
        // relabel every rank with its new root
        for (uint32_t r = tid; r < a.k; r += nth) {
            uint32_t c = ldcg_u32(&a.comp[r]);
            for (uint32_t steps = 0; steps < a.k; ++steps) {
                uint32_t p = ldcg_u32(&a.hook[c]);
                if (p == c) break;
                c = p;
            }
            a.comp[r] = c;
        }
        if (!grid_sync(&ctl->bar2, &ctl->err)) return;
    }
}

// ---------------------------------------------------------------------------
// expansion: bridges of MST pairs + predecessor walks
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t arc_owner(const uint32_t *row_ptr, uint32_t n, uint32_t arc) {
    uint32_t lo = 0, hi = n;        // largest v with row_ptr[v] <= arc
    while (hi - lo > 1) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (row_ptr[mid] <= arc) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void emit_edge(uint32_t a, uint32_t b, uint32_t w, uint32_t nbits,
                                          uint64_t *key, uint32_t *wout, uint32_t cap,
                                          Control *ctl) {
    uint32_t lo = min(a, b), hi = max(a, b);
    uint32_t slot = atomicAdd(&ctl->n_tree, 1u);
    if (slot >= cap) {
        atomicOr(&ctl->err, ERR_CAPACITY);
        return;
    }
    key[slot] = ((uint64_t)lo << nbits) | hi;
    wout[slot] = w;
}

// Two threads per MST pair: thread 0 emits the bridge and walks pred() from
// the bridge's tail, thread 1 walks from its head.  Per hop the mark exchange
// and the pred load are issued together, so a hop costs two dependent loads
// (pred arc, then the arc's record) instead of three.
__global__ void expand_kernel(const uint32_t *__restrict__ row_ptr, const uint2 *__restrict__ adj,
                              const uint32_t *__restrict__ orig_of,
                              const uint32_t *__restrict__ new_of,
                              const uint32_t *__restrict__ orig_row_ptr,
                              uint32_t n, const uint32_t *__restrict__ e_arc,
                              const uint32_t *__restrict__ e_mst,
                              const uint32_t *__restrict__ pred_arc, uint32_t pred_stride,
                              uint32_t *mark, uint32_t tag, uint32_t nbits, uint64_t *key,
                              uint32_t *wout, uint32_t cap, Control *ctl) {
    const uint32_t E = ldcg_u32(&ctl->n_pairs);
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < 2 * E; t += gridDim.x * blockDim.x) {
        const uint32_t j = t >> 1, side = t & 1;
        if (!e_mst[j]) continue;
        // the pair table holds the caller's arc index: its tail in the
        // caller's CSR, then the same arc in the internal order
        const uint32_t carc = e_arc[j];
        uint32_t tail, arc;
        if (orig_of) {
            const uint32_t ct = arc_owner(orig_row_ptr, n, carc);
            tail = new_of[ct];
            arc = row_ptr[tail] + (carc - orig_row_ptr[ct]);
        } else {
            tail = arc_owner(row_ptr, n, carc);
            arc = carc;
        }
        uint2 e = adj[arc];
        uint32_t x = e.x;
        if (side == 0) {
            atomicAdd(&ctl->n_mst, 1u);
            x = tail;
            emit_edge(caller_id(orig_of, x), caller_id(orig_of, e.x), e.y, nbits, key, wout, cap,
                      ctl);
        }
        for (uint32_t steps = 0; steps < n; ++steps) {
            uint32_t pa = pred_arc[(uint64_t)x * pred_stride];
            if (pa == SEED_ARC || pa == INF32) break;
            uint32_t old = atomicExch(&mark[x], tag);
            uint2 pe = adj[pa];              // independent of the exchange's result
            if (old == tag) break;           // the rest of the chain is another walker's
            emit_edge(caller_id(orig_of, x), caller_id(orig_of, pe.x), pe.y, nbits, key, wout, cap,
                      ctl);
            x = pe.x;
        }
    }
}

// ---------------------------------------------------------------------------
// cooperative LSD radix sort of (key, weight) pairs, 8-bit digits; the
// weights are also summed into ctl->total
// ---------------------------------------------------------------------------

constexpr int RS_THREADS = 512;
constexpr int RS_WARPS = RS_THREADS / 32;

struct SortArgs {
    uint64_t *key0, *key1;
    uint32_t *w0, *w1;
    uint32_t *blk_hist;     // [gridDim.x][256]
    uint32_t passes;
    uint32_t cap;
    Control *ctl;
};

__global__ void __launch_bounds__(RS_THREADS) radix_sort_kernel(SortArgs a) {
    __shared__ uint32_t hist[256];
    __shared__ uint32_t base[256];
    __shared__ uint32_t wcnt[RS_WARPS][256];
    __shared__ uint32_t tile_tot[256];
    __shared__ unsigned long long wsum[RS_WARPS];
    Control *ctl = a.ctl;
    const uint32_t N = min(ldcg_u32(&ctl->n_tree), a.cap);
    const uint32_t per = (N + gridDim.x - 1) / gridDim.x;
    const uint32_t lo = min(N, blockIdx.x * per), hi = min(N, lo + per);
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();

    // total distance
    unsigned long long tot = 0;
    for (uint32_t i = lo + threadIdx.x; i < hi; i += RS_THREADS) tot += a.w0[i];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) tot += __shfl_xor_sync(FULL, tot, o);
    if (lane == 0) wsum[warp] = tot;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int i = 0; i < RS_WARPS; ++i) t += wsum[i];
        if (t) atomicAdd(&ctl->total, t);
    }

    for (uint32_t p = 0; p < a.passes; ++p) {
        const bool odd = p & 1;
        const uint64_t *src = odd ? a.key1 : a.key0;
        const uint32_t *srcw = odd ? a.w1 : a.w0;
        uint64_t *dst = odd ? a.key0 : a.key1;
        uint32_t *dstw = odd ? a.w0 : a.w1;
        const uint32_t sh = 8 * p;
        for (uint32_t d = threadIdx.x; d < 256; d += RS_THREADS) hist[d] = 0;
        __syncthreads();
        for (uint32_t i = lo + threadIdx.x; i < hi; i += RS_THREADS)
            atomicAdd(&hist[(src[i] >> sh) & 255u], 1u);
        __syncthreads();
        for (uint32_t d = threadIdx.x; d < 256; d += RS_THREADS)
            a.blk_hist[blockIdx.x * 256 + d] = hist[d];
        if (!grid_sync(&ctl->bar2, &ctl->err)) return;
        // this block's first output position per digit
        if (threadIdx.x < 256) {
            uint32_t d = threadIdx.x, before = 0, total = 0;
            for (uint32_t b = 0; b < gridDim.x; ++b) {
                uint32_t c = __ldcg(&a.blk_hist[b * 256 + d]);
                if (b < blockIdx.x) before += c;
                total += c;
            }
            base[d] = before;
            hist[d] = total;
        }
        __syncthreads();
        if (threadIdx.x < 32) {       // exclusive scan of the digit totals
            uint32_t carry = 0;
            for (uint32_t c0 = 0; c0 < 256; c0 += 32) {
                uint32_t x = hist[c0 + threadIdx.x];
                uint32_t incl = warp_inclusive_scan(x);
                base[c0 + threadIdx.x] += carry + incl - x;
                carry += __shfl_sync(FULL, incl, 31);
            }
        }
        __syncthreads();
        // stable scatter, one RS_THREADS-key tile at a time
        for (uint32_t t0 = lo; t0 < hi; t0 += RS_THREADS) {
            uint32_t i = t0 + threadIdx.x;
            bool valid = i < hi;
            uint64_t key = valid ? src[i] : 0;
            uint32_t wv = valid ? srcw[i] : 0;
            uint32_t d = valid ? (uint32_t)((key >> sh) & 255u) : 256u + lane;
            for (uint32_t x = threadIdx.x; x < RS_WARPS * 256; x += RS_THREADS)
                (&wcnt[0][0])[x] = 0;
            __syncthreads();
            uint32_t peers = __match_any_sync(FULL, d);
            uint32_t rank = __popc(peers & lanemask_lt());
            if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
            __syncthreads();
            if (threadIdx.x < 256) {
                uint32_t run = 0;
                for (int w2 = 0; w2 < RS_WARPS; ++w2) {
                    uint32_t c = wcnt[w2][threadIdx.x];
                    wcnt[w2][threadIdx.x] = run;
                    run += c;
                }
                tile_tot[threadIdx.x] = run;
            }
            __syncthreads();
            if (valid) {
                uint32_t pos = base[d] + wcnt[warp][d] + rank;
                if (pos < N) {
                    dst[pos] = key;
                    dstw[pos] = wv;
                } else {
                    atomicOr(&ctl->err, ERR_CAPACITY);
                }
            }
            __syncthreads();
            if (threadIdx.x < 256) base[threadIdx.x] += tile_tot[threadIdx.x];
            __syncthreads();
        }
        if (!grid_sync(&ctl->bar2, &ctl->err)) return;
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

int mst_occupancy(int threads) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, mst_kernel, threads, 0) != cudaSuccess)
        return 0;
    return nb;
}

static int sort_blocks_cache = -1;

cudaError_t launch_mst(Workspace &ws, uint32_t k, const Geometry &geo, cudaStream_t s) {
    if (k < 2) return cudaSuccess;
    MstArgs a;
    a.e_key = ws.e_key;
    a.e_ra = ws.e_ra;
    a.e_rb = ws.e_rb;
    a.e_mst = ws.e_mst;
    a.comp = ws.comp;
    a.hook = ws.hook;
    a.best = ws.best;
    a.k = k;
    a.ctl = ws.ctl;
    uint64_t slots = (uint64_t)k * (k - 1) / 2;
    int blocks = slots <= 65536 ? 1 : geo.mst_blocks;
    cudaError_t e = cudaMemsetAsync(&ws.ctl->bar2, 0, sizeof(GridBarrier), s);
    if (e != cudaSuccess) return e;
    void *args[] = {&a};
    return cudaLaunchCooperativeKernel((const void *)mst_kernel, dim3(blocks), dim3(512), args, 0, s);
}

cudaError_t launch_tree(const DevGraph &g, Workspace &ws, uint32_t k, uint32_t tag,
                        uint32_t n_bits, cudaStream_t s) {
    if (k < 2) return cudaSuccess;
    uint64_t slots = (uint64_t)k * (k - 1) / 2;
    uint32_t blocks = (uint32_t)std::min<uint64_t>((2 * slots + 255) / 256, (uint64_t)current_sm_count() * 8);
    expand_kernel<<<blocks, 256, 0, s>>>(g.row_ptr, g.adj, g.orig_of, g.new_of, g.orig_row_ptr,
                                         g.n, ws.e_arc, ws.e_mst, ws.pred_arc,
                                         ws.pred_stride, ws.mark, tag, n_bits, ws.tree_key,
                                         ws.tree_w, ws.tree_cap, ws.ctl);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (sort_blocks_cache < 0) {
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, radix_sort_kernel, RS_THREADS, 0);
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        sort_blocks_cache = std::max(1, std::min(nb * sms, 64));
    }
    SortArgs a;
    a.key0 = ws.tree_key;
    a.key1 = ws.tree_key2;
    a.w0 = ws.tree_w;
    a.w1 = ws.tree_w2;
    a.blk_hist = ws.tile_off;       // reused: >= 64 * 256 entries
    uint32_t bits = 2 * n_bits;
    a.passes = (bits + 7) / 8;
    if (a.passes & 1) a.passes += 1;    // even: the result lands back in key[0]
    a.cap = ws.tree_cap;
    a.ctl = ws.ctl;
    e = cudaMemsetAsync(&ws.ctl->bar2, 0, sizeof(GridBarrier), s);
    if (e != cudaSuccess) return e;
    void *args[] = {&a};
    return cudaLaunchCooperativeKernel((const void *)radix_sort_kernel, dim3(sort_blocks_cache),
                                       dim3(RS_THREADS), args, 0, s);
}

}  // namespace stn

namespace stn {

// Sorts N = min(ctl->n_tree, cap) (key, weight) pairs by the low key_bits
// bits of the key (the result lands back in key0 / w0); blk_hist needs
// 64 * 256 entries.  Also adds the weights into ctl->total.
cudaError_t launch_sort_keys(uint64_t *key0, uint64_t *key1, uint32_t *w0, uint32_t *w1,
                             uint32_t *blk_hist, uint32_t cap, uint32_t key_bits, Control *ctl,
                             cudaStream_t s) {
    if (sort_blocks_cache < 0) {
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, radix_sort_kernel, RS_THREADS, 0);
        sort_blocks_cache = std::max(1, std::min(nb * current_sm_count(), 64));
    }
    SortArgs a;
    a.key0 = key0;
    a.key1 = key1;
    a.w0 = w0;
    a.w1 = w1;
    a.blk_hist = blk_hist;
    a.passes = (key_bits + 7) / 8;
    if (a.passes & 1) a.passes += 1;
    a.cap = cap;
    a.ctl = ctl;
    cudaError_t e = cudaMemsetAsync(&ctl->bar2, 0, sizeof(GridBarrier), s);
    if (e != cudaSuccess) return e;
    void *args[] = {&a};
    return cudaLaunchCooperativeKernel((const void *)radix_sort_kernel, dim3(sort_blocks_cache),
                                       dim3(RS_THREADS), args, 0, s);
}

}  // namespace stn
