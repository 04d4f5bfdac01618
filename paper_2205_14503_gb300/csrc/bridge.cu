// One pass over every arc after the Voronoi fixed point, fusing two steps:
//
//  * pred (Algorithm 2 Step 1's predecessor state; Algorithm 4 line 8):
//    pred(v) = the smallest-id neighbour u with cell(u) = cell(v) and
//    d1(u) + d(u,v) = d1(v).  Rows are sorted by neighbour id, so the
//    smallest arc index in v's row is the smallest id: atomicMin on the
//    arc index.
//  * bridges (Algorithm 2 Step 2; Algorithm 5): for an arc u -> v with
//    rank(cell u) < rank(cell v), b = d1(u) + d(u,v) + d1(v); the pair's
//    table slot keeps min((b << 32) | arc) by 64-bit atomicMin, which is
//    the minimum bridge with the smallest arc id among ties.  This single
//    table stands in for the paper's per-partition maps plus its
//    MPI_Allreduce(MIN) (GLOBAL_MIN_DIST_EDGE_COLL).
//
// The pair table is a direct-address table over the k(k-1)/2 seed pairs
// (an upper-triangle index, i.e. a collision-free hash of the pair).
//
// Load balance: vertices with degree < HEAVY_DEG are processed 32 per warp
// with their arcs flattened over the lanes (labels of 32 consecutive
// vertices are one coalesced load); higher-degree rows are split into
// CHUNK-arc pieces listed once at graph load.
#include "internal.h"

namespace stn {

struct ScanArgs {
    const uint32_t *__restrict__ row_ptr;
    const uint2 *__restrict__ adj;
    const uint64_t *__restrict__ heavy_chunks;
    uint32_t n_heavy_chunks;
    uint32_t n;
    const uint64_t *label;
    const uint32_t *label32;         // narrow labels (the narrow kernel)
    uint32_t lshift;
    uint32_t *pred_arc;
    uint64_t *pairtab;
    uint32_t k;
    bool pairs;
    uint32_t *err;
    const uint32_t *orig_of;         // internal -> caller ids (null: identity)
    const uint32_t *orig_row_ptr;
};

// Label of v in the 64-bit form.
template <bool NARROW>
__device__ __forceinline__ uint64_t scan_label(const ScanArgs &a, uint32_t v) {
    if (NARROW) return widen_label(__ldg(&a.label32[v]), a.lshift);
    return __ldg(reinterpret_cast<const unsigned long long *>(&a.label[v]));
}

// Arc `arc` of row v.  The bridge key carries the caller's arc index,
// cbase + arc (cbase: the caller's row start of v minus v's internal row
// start, taken once per row), so ties between equal bridges break on the
// caller's CSR order whatever the internal vertex order.
template <bool NARROW>
__device__ __forceinline__ void scan_arc(const ScanArgs &a, bool valid, uint32_t v, uint64_t lv,
                                         uint32_t cbase, uint32_t arc, uint2 e, bool &overflow) {
    if (!valid) return;
    uint64_t lu = scan_label<NARROW>(a, e.x);
    if (lv == INF64 || lu == INF64) {
        // a reached vertex next to an unreached one: its true distance is
        // finite but did not fit below 2^32 - 1
        if (lv != lu) overflow = true;
        return;
    }
    uint32_t cv = (uint32_t)lv, cu = (uint32_t)lu;
    uint64_t dv = lv >> 32, du = lu >> 32;
    if (cu == cv) {
        if (du + e.y == dv) atomicMin(&a.pred_arc[v], arc);
    } else if (a.pairs && cv < cu) {
        uint64_t b = dv + e.y + du;
        if (b >= INF32) {
            overflow = true;
            return;
        }
        uint64_t key = (b << 32) | (uint32_t)(cbase + arc);
        uint64_t *slot = &a.pairtab[pair_slot(cv, cu, a.k)];
        // a cached read may be stale, i.e. larger: at worst one atomic more
        if (key < __ldg(reinterpret_cast<const unsigned long long *>(slot)))
            atomicMin(reinterpret_cast<unsigned long long *>(slot), (unsigned long long)key);
    }
}

template <bool NARROW>
__global__ void __launch_bounds__(256) scan_kernel(ScanArgs a) {
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t n_batches = (a.n + 31) / 32;
    const uint32_t n_work = a.n_heavy_chunks + n_batches;
    bool overflow = false;
    for (uint32_t wi = warp; wi < n_work; wi += nwarps) {
        if (wi < a.n_heavy_chunks) {
            uint64_t item = a.heavy_chunks[wi];
            uint32_t v = (uint32_t)(item >> 32), c = (uint32_t)item;
            uint32_t rs = a.row_ptr[v];
            uint32_t s = rs + c * CHUNK;
            uint32_t e = min(a.row_ptr[v + 1], s + CHUNK);
            uint64_t lv = scan_label<NARROW>(a, v);
            uint32_t cbase = caller_arc_base(a.orig_of, a.orig_row_ptr, v, rs);
            // the next 32 arcs' records are loaded while these are scanned
            uint2 en = make_uint2(0, 0);
            if (s + lane < e) en = __ldcs(&a.adj[s + lane]);    // streamed once: evict first
            for (uint32_t b = s; b < e; b += 32) {
                const uint2 ec = en;
                if (b + 32 + lane < e) en = __ldcs(&a.adj[b + 32 + lane]);
                scan_arc<NARROW>(a, b + lane < e, v, lv, cbase, b + lane, ec, overflow);
            }
        } else {
            uint32_t v = (wi - a.n_heavy_chunks) * 32 + lane;
            uint32_t s = 0, deg = 0, cbase = 0;
            uint64_t lv = INF64;
            if (v < a.n) {
                s = a.row_ptr[v];
                deg = a.row_ptr[v + 1] - s;
                if (deg >= HEAVY_DEG) deg = 0;          // covered by the chunk list
                lv = scan_label<NARROW>(a, v);
                if (deg) cbase = caller_arc_base(a.orig_of, a.orig_row_ptr, v, s);
            }
            uint32_t incl = warp_inclusive_scan(deg);
            uint32_t excl = incl - deg;
            uint32_t total = __shfl_sync(FULL, incl, 31);
            // arc j of the batch belongs to the lane whose prefix covers it;
            // the next 32 arcs' records are loaded while these are scanned
            uint32_t own = warp_owner_search(excl, lane < total ? lane : 0);
            const uint32_t s0 = __shfl_sync(FULL, s, own), x0 = __shfl_sync(FULL, excl, own);
            uint2 en = make_uint2(0, 0);
            if (lane < total) en = __ldcs(&a.adj[s0 + (lane - x0)]);
            for (uint32_t b = 0; b < total; b += 32) {
                const uint32_t j = b + lane;
                const bool valid = j < total;
                const uint32_t owner = own;
                const uint32_t arc = __shfl_sync(FULL, s, owner) + (j - __shfl_sync(FULL, excl, owner));
                const uint2 ec = en;
                const uint32_t jn = j + 32;
                own = warp_owner_search(excl, jn < total ? jn : 0);
                const uint32_t sn = __shfl_sync(FULL, s, own), xn = __shfl_sync(FULL, excl, own);
                if (jn < total) en = __ldcs(&a.adj[sn + (jn - xn)]);
                const uint64_t lo = __shfl_sync(FULL, lv, owner);
                const uint32_t co = __shfl_sync(FULL, cbase, owner);
                const uint32_t vo = (wi - a.n_heavy_chunks) * 32 + owner;
                scan_arc<NARROW>(a, valid, vo, lo, co, arc, ec, overflow);
            }
        }
    }
    if (__any_sync(FULL, overflow) && lane == 0) atomicOr(a.err, ERR_OVERFLOW);
}

// ---------------------------------------------------------------------------
// ordered compaction of the pair table: entries != INF in slot order,
// i.e. ascending (rank a, rank b)
// ---------------------------------------------------------------------------

constexpr uint32_t CT_THREADS = 256;
constexpr uint32_t CT_PER_THREAD = 8;
constexpr uint32_t CT_TILE = CT_THREADS * CT_PER_THREAD;

__global__ void __launch_bounds__(CT_THREADS) pair_count_kernel(const uint64_t *__restrict__ tab,
                                                                uint64_t slots,
                                                                uint32_t *__restrict__ tile_cnt) {
    __shared__ uint32_t wsum[CT_THREADS / 32];
    uint64_t base = (uint64_t)blockIdx.x * CT_TILE + (uint64_t)threadIdx.x * CT_PER_THREAD;
    uint32_t c = 0;
#pragma unroll
    for (uint32_t i = 0; i < CT_PER_THREAD; ++i)
        if (base + i < slots && tab[base + i] != INF64) ++c;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
    if (lane_id() == 0) wsum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (uint32_t w = 0; w < CT_THREADS / 32; ++w) t += wsum[w];
        tile_cnt[blockIdx.x] = t;
    }
}

// single block: exclusive scan of the tile counts, total into *n_pairs
__global__ void __launch_bounds__(1024) tile_scan_kernel(uint32_t *tile_cnt, uint32_t n_tiles,
                                                         uint32_t *n_pairs) {
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < n_tiles; base += blockDim.x) {
        uint32_t i = base + threadIdx.x;
        uint32_t x = i < n_tiles ? tile_cnt[i] : 0;
        uint32_t incl = warp_inclusive_scan(x);
        if (lane_id() == 31) wsum[threadIdx.x >> 5] = incl;
        __syncthreads();
        if (threadIdx.x < 32) {
            uint32_t ws = wsum[threadIdx.x];
            uint32_t wi = warp_inclusive_scan(ws);
            wsum[threadIdx.x] = wi - ws;
        }
        __syncthreads();
        uint32_t excl = carry + wsum[threadIdx.x >> 5] + incl - x;
        if (i < n_tiles) tile_cnt[i] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_pairs = carry;
}

__global__ void __launch_bounds__(CT_THREADS) pair_write_kernel(
    const uint64_t *__restrict__ tab, uint64_t slots, uint32_t k,
    const uint32_t *__restrict__ tile_off, uint64_t *e_key, uint32_t *e_ra, uint32_t *e_rb,
    uint32_t *e_arc, uint32_t *e_mst) {
    __shared__ uint32_t wsum[CT_THREADS / 32];
    uint64_t base = (uint64_t)blockIdx.x * CT_TILE + (uint64_t)threadIdx.x * CT_PER_THREAD;
    uint64_t vals[CT_PER_THREAD];
    uint32_t c = 0;
#pragma unroll
    for (uint32_t i = 0; i < CT_PER_THREAD; ++i) {
        vals[i] = base + i < slots ? tab[base + i] : INF64;
        if (vals[i] != INF64) ++c;
    }
    uint32_t incl = warp_inclusive_scan(c);
    if (lane_id() == 31) wsum[threadIdx.x >> 5] = incl;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t ws = threadIdx.x < CT_THREADS / 32 ? wsum[threadIdx.x] : 0;
        uint32_t wi = warp_inclusive_scan(ws);
        if (threadIdx.x < CT_THREADS / 32) wsum[threadIdx.x] = wi - ws;
    }
    __syncthreads();
    uint32_t out = tile_off[blockIdx.x] + wsum[threadIdx.x >> 5] + incl - c;
#pragma unroll
    for (uint32_t i = 0; i < CT_PER_THREAD; ++i) {
        if (vals[i] == INF64) continue;
        uint64_t slot = base + i;
        uint32_t ra, rb;
        slot_to_pair(slot, k, ra, rb);
        e_key[out] = (vals[i] & 0xFFFFFFFF00000000ull) | slot;    // (b << 32) | slot
        e_ra[out] = ra;
        e_rb[out] = rb;
        e_arc[out] = (uint32_t)vals[i];
        e_mst[out] = 0;
        ++out;
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

cudaError_t launch_scan(const DevGraph &g, Workspace &ws, uint32_t k, bool pairs,
                        cudaStream_t s) {
    ScanArgs a;
    a.row_ptr = g.row_ptr;
    a.adj = g.adj;
    a.heavy_chunks = g.heavy_chunks;
    a.n_heavy_chunks = g.n_heavy_chunks;
    a.n = g.n;
    a.label = ws.label;
    a.label32 = ws.label32;
    a.lshift = ws.lshift;
    a.pred_arc = ws.pred_arc;
    a.pairtab = ws.pairtab;
    a.k = k;
    a.pairs = pairs && k > 1;
    a.err = &ws.ctl->err;
    a.orig_of = g.orig_of;
    a.orig_row_ptr = g.orig_row_ptr;
    if (a.pairs) {
        uint64_t slots = (uint64_t)k * (k - 1) / 2;
        cudaError_t e = cudaMemsetAsync(ws.pairtab, 0xFF, slots * sizeof(uint64_t), s);
        if (e != cudaSuccess) return e;
    }
    uint64_t work = (uint64_t)g.n_heavy_chunks + (g.n + 31) / 32;
    uint64_t blocks = (work + 7) / 8;          // 8 warps per block
    const uint64_t cap = (uint64_t)current_sm_count() * 32;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (ws.narrow) scan_kernel<true><<<(unsigned)blocks, 256, 0, s>>>(a);
    else scan_kernel<false><<<(unsigned)blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_compact_pairs(Workspace &ws, uint32_t k, cudaStream_t s) {
    uint64_t slots = k > 1 ? (uint64_t)k * (k - 1) / 2 : 0;
    if (slots == 0) return cudaMemsetAsync(&ws.ctl->n_pairs, 0, sizeof(uint32_t), s);
    uint32_t tiles = (uint32_t)((slots + CT_TILE - 1) / CT_TILE);
    pair_count_kernel<<<tiles, CT_THREADS, 0, s>>>(ws.pairtab, slots, ws.tile_off);
    tile_scan_kernel<<<1, 1024, 0, s>>>(ws.tile_off, tiles, &ws.ctl->n_pairs);
    pair_write_kernel<<<tiles, CT_THREADS, 0, s>>>(ws.pairtab, slots, k, ws.tile_off, ws.e_key,
                                                   ws.e_ra, ws.e_rb, ws.e_arc, ws.e_mst);
    return cudaGetLastError();
}

}  // namespace stn
