// Graph upload: device-side validation of the CSR (the paper's graphs are
// symmetric with positive integer weights: Table "preliminaries_notation",
// Section "Evaluation") and interleaving of (neighbour, weight) into one
// 8-byte record per arc, so a relaxation reads one sector-aligned pair.
#include <atomic>

#include "internal.h"

namespace stn {

int current_sm_count() {
    constexpr int MAX_DEVICES = 64;
    static std::atomic<int> cache[MAX_DEVICES];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        dev = -1;
    }
    int sms = dev >= 0 ? cache[dev].load(std::memory_order_relaxed) : 0;
    if (sms > 0) return sms;
    if (dev < 0 || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms < 1) {
        cudaGetLastError();
        return 1;
    }
    cache[dev].store(sms, std::memory_order_relaxed);
    return sms;
}

enum : uint32_t {
    BAD_RANGE = 1u,      // neighbour id out of range
    BAD_SELF = 2u,       // self-loop
    BAD_WEIGHT = 4u,     // weight 0
    BAD_ORDER = 8u,      // row not strictly ascending (unsorted or duplicate)
    BAD_SYMMETRY = 16u,  // reverse arc missing or with another weight
};

__device__ __forceinline__ bool find_reverse(const uint32_t *row_ptr, const int32_t *col,
                                             const uint32_t *w, uint32_t v, uint32_t u,
                                             uint32_t wt) {
    uint32_t lo = row_ptr[v], hi = row_ptr[v + 1];
    while (lo < hi) {
        uint32_t mid = lo + (hi - lo) / 2;
        uint32_t c = (uint32_t)col[mid];
        if (c == u) return w[mid] == wt;
        if (c < u) lo = mid + 1; else hi = mid;
    }
    return false;
}

__global__ void __launch_bounds__(256) validate_kernel(const uint32_t *__restrict__ row_ptr,
                                                       const int32_t *__restrict__ col,
                                                       const uint32_t *__restrict__ w,
                                                       uint32_t n, uint2 *__restrict__ adj,
                                                       const uint32_t *__restrict__ new_of,
                                                       const uint32_t *__restrict__ new_row_ptr,
                                                       uint32_t *bad, uint32_t *max_w) {
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    uint32_t flags = 0, wmax = 0;
    for (uint32_t b0 = warp * 32; b0 < n; b0 += nwarps * 32) {
        uint32_t u = b0 + lane;
        uint32_t s = 0, deg = 0;
        if (u < n) {
            s = row_ptr[u];
            deg = row_ptr[u + 1] - s;
        }
        uint32_t incl = warp_inclusive_scan(deg);
        uint32_t excl = incl - deg;
        uint32_t total = __shfl_sync(FULL, incl, 31);
        for (uint32_t b = 0; b < total; b += 32) {
            uint32_t j = b + lane;
            bool valid = j < total;
            uint32_t owner = warp_owner_search(excl, valid ? j : 0);
            uint32_t so = __shfl_sync(FULL, s, owner);
            uint32_t eo = __shfl_sync(FULL, excl, owner);
            if (!valid) continue;
            uint32_t src = b0 + owner;
            uint32_t e = so + (j - eo);
            int32_t c = col[e];
            uint32_t wt = w[e];
            wmax = max(wmax, wt);
            if (c < 0 || (uint32_t)c >= n) {
                flags |= BAD_RANGE;
                continue;
            }
            if (new_of)
                adj[new_row_ptr[new_of[src]] + (e - so)] = make_uint2(new_of[c], wt);
            else
                adj[e] = make_uint2((uint32_t)c, wt);
            if ((uint32_t)c == src) flags |= BAD_SELF;
            if (wt == 0) flags |= BAD_WEIGHT;
            if (e > so && col[e - 1] >= c) flags |= BAD_ORDER;
            if (!find_reverse(row_ptr, col, w, (uint32_t)c, src, wt)) flags |= BAD_SYMMETRY;
        }
    }
    if (flags) atomicOr(bad, flags);
    wmax = __reduce_max_sync(FULL, wmax);
    if (lane == 0 && wmax) atomicMax(max_w, wmax);
}

// One warp per row: arcs lighter than delta first, then the rest, each part
// in the row's order.
__global__ void __launch_bounds__(256) partition_kernel(const uint32_t *__restrict__ row_ptr,
                                                        const uint2 *__restrict__ adj, uint32_t n,
                                                        uint32_t delta, uint2 *__restrict__ adj_w,
                                                        uint32_t *__restrict__ lend) {
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t v = warp; v < n; v += nwarps) {
        const uint32_t s = row_ptr[v], e = row_ptr[v + 1];
        uint32_t nl = 0;
        for (uint32_t b = s; b < e; b += 32) {
            const uint32_t j = b + lane;
            nl += __popc(__ballot_sync(FULL, j < e && __ldg(&adj[j].y) < delta));
        }
        if (lane == 0) lend[v] = s + nl;
        uint32_t lo = s, hi = s + nl;
        for (uint32_t b = s; b < e; b += 32) {
            const uint32_t j = b + lane;
            const bool valid = j < e;
            const uint2 x = valid ? __ldg(&adj[j]) : make_uint2(0, 0);
            const bool light = valid && x.y < delta;
            const uint32_t ml = __ballot_sync(FULL, light), mv = __ballot_sync(FULL, valid);
            const uint32_t mh = mv & ~ml, lt = lanemask_lt();
            if (light) adj_w[lo + __popc(ml & lt)] = x;
            else if (valid) adj_w[hi + __popc(mh & lt)] = x;
            lo += __popc(ml);
            hi += __popc(mh);
        }
    }
}

cudaError_t launch_partition(const DevGraph &g, uint32_t delta, cudaStream_t s) {
    uint64_t blocks = ((uint64_t)g.n + 7) / 8;
    const uint64_t cap = (uint64_t)current_sm_count() * 32;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    partition_kernel<<<(unsigned)blocks, 256, 0, s>>>(g.row_ptr, g.adj, g.n, delta, g.adj_w, g.lend);
    return cudaGetLastError();
}

cudaError_t ensure_partition_dev(DevGraph &g, uint32_t delta, cudaStream_t s) {
    if (delta > g.max_w || g.m == 0 || g.part_delta == delta) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (!g.adj_w) e = cudaMalloc((void **)&g.adj_w, (size_t)g.m * sizeof(uint2));
    if (e == cudaSuccess && !g.lend) e = cudaMalloc((void **)&g.lend, (size_t)g.n * 4);
    if (e == cudaSuccess) e = launch_partition(g, delta, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        g.part_delta = 0;
        return e;
    }
    g.part_delta = delta;
    return cudaSuccess;
}

cudaError_t launch_validate_graph(const uint32_t *row_ptr, const int32_t *col, const uint32_t *w,
                                  uint32_t n, uint64_t m, uint2 *adj, const uint32_t *new_of,
                                  const uint32_t *new_row_ptr, uint32_t *bad, uint32_t *max_w,
                                  cudaStream_t s) {
    (void)m;
    uint64_t blocks = ((uint64_t)n + 255) / 256;
    const uint64_t cap = (uint64_t)current_sm_count() * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    validate_kernel<<<(unsigned)blocks, 256, 0, s>>>(row_ptr, col, w, n, adj, new_of, new_row_ptr,
                                                      bad, max_w);
    return cudaGetLastError();
}

}  // namespace stn
