// Device-side helpers shared by the library's kernels: constants, the
// bounded grid-wide barrier used by the persistent kernels, cache-global
// loads for data other blocks write, and warp-level scans.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace stn {

constexpr uint32_t INF32 = 0xFFFFFFFFu;
constexpr uint64_t INF64 = ~0ull;
constexpr uint32_t SEED_ARC = 0xFFFFFFFEu;   // pred_arc marker of a seed (pred = self)
constexpr uint32_t FULL = 0xFFFFFFFFu;

// Device status bits, collected in Control::err and mapped to STEINER_E* on
// the host.
enum : uint32_t {
    ERR_OVERFLOW = 1u,      // a distance or bridge sum reached 2^32 - 1
    ERR_TIMEOUT = 2u,       // iteration cap hit
    ERR_CAPACITY = 4u,      // an append would have overrun its buffer (skipped)
    ERR_BARRIER = 8u,       // a grid barrier wait gave up
    ERR_NARROW = 16u,       // a distance did not fit a 32-bit label (rerun with 64 bits)
};

// Labels.  The 64-bit form is (dist << 32) | rank.  The narrow 32-bit form
// is (dist << shift) | rank with shift = the bits of the largest rank, for
// distances up to (2^(32 - shift)) - 2; both order lexicographically by
// (dist, rank), so an atomicMin on either finds the same fixed point.  The
// all-ones word is "unreached" in both.  widen_label maps the narrow form
// to the 64-bit one.
__host__ __device__ __forceinline__ uint64_t widen_label(uint32_t l, uint32_t shift) {
    if (l == 0xFFFFFFFFu) return ~0ull;
    return ((uint64_t)(l >> shift) << 32) | (l & ((1u << shift) - 1u));
}

// Spin limit of a grid barrier wait (each spin sleeps ~64 ns): ~4 s.
constexpr long long BARRIER_SPIN_LIMIT = 1ll << 26;

struct GridBarrier {
    unsigned int count;
    unsigned int gen;
};

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add_u32(unsigned int *p, unsigned int v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// Loads that bypass L1: for values written by other blocks of a persistent
// kernel (labels, queues, counters).
__device__ __forceinline__ uint64_t ldcg_u64(const uint64_t *p) {
    return __ldcg(reinterpret_cast<const unsigned long long *>(p));
}
__device__ __forceinline__ uint32_t ldcg_u32(const uint32_t *p) { return __ldcg(p); }

// Grid-wide barrier for cooperatively launched kernels.  Every wait is
// bounded: a block that waits longer than BARRIER_SPIN_LIMIT spins sets
// ERR_BARRIER in *err and returns false; callers then leave their loop.
// Once ERR_BARRIER is set every later barrier returns false too, so all
// blocks leave within one more bounded wait.  Returns true on a normal
// release.  Single-block grids use __syncthreads.
__device__ __forceinline__ bool grid_sync(GridBarrier *bar, uint32_t *err) {
    __shared__ int ok_s;
    if (gridDim.x == 1) {
        __syncthreads();
        return true;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned int g = ld_acquire_u32(&bar->gen);
        __threadfence();
        unsigned int arrived = atomicAdd(&bar->count, 1u) + 1u;
        if (arrived == gridDim.x) {
            bar->count = 0;
            __threadfence();
            red_release_add_u32(&bar->gen, 1u);
        } else {
            long long spins = 0;
            while (ld_acquire_u32(&bar->gen) == g) {
                if (++spins > BARRIER_SPIN_LIMIT) {
                    atomicOr(err, ERR_BARRIER);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        // a block that gave up earlier poisons every later barrier
        if (ld_acquire_u32(err) & ERR_BARRIER) ok = 0;
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

// The GPU's global nanosecond timer (for the iteration trace).
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Inclusive warp scan (all 32 lanes participate).
__device__ __forceinline__ uint32_t warp_inclusive_scan(uint32_t x) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane_id() >= (uint32_t)o) x += y;
    }
    return x;
}

// Largest lane L whose value excl[L] <= j (excl non-decreasing across lanes).
__device__ __forceinline__ uint32_t warp_owner_search(uint32_t excl, uint32_t j) {
    uint32_t lo = 0;
#pragma unroll
    for (uint32_t step = 16; step >= 1; step >>= 1) {
        uint32_t cand = lo + step;
        uint32_t ev = __shfl_sync(FULL, excl, cand & 31u);
        if (cand < 32 && ev <= j) lo = cand;
    }
    return lo;
}

// Warp-aggregated append: lanes with `want` get consecutive slots of a
// queue whose fill counter is *count and capacity cap.  Returns the slot or
// INF32 if the lane did not append or the queue was full (ERR_CAPACITY).
__device__ __forceinline__ uint32_t warp_append(bool want, uint32_t *count, uint32_t cap,
                                                uint32_t *err) {
    uint32_t mask = __ballot_sync(FULL, want);
    if (mask == 0) return INF32;
    uint32_t leader = __ffs(mask) - 1;
    uint32_t base = 0;
    if (lane_id() == leader) base = atomicAdd(count, (uint32_t)__popc(mask));
    base = __shfl_sync(FULL, base, leader);
    if (!want) return INF32;
    uint32_t slot = base + (uint32_t)__popc(mask & lanemask_lt());
    if (slot >= cap) {
        atomicOr(err, ERR_CAPACITY);
        return INF32;
    }
    return slot;
}

// Warp-aggregated append of v into a staging buffer, spilling to the
// global queue (gq, gcount, gcap) when the buffer is full.  All lanes call.
__device__ __forceinline__ void stage_append(bool want, uint32_t v, uint32_t *buf, uint32_t *cnt,
                                             uint32_t cap, uint32_t *gq, uint32_t *gcount,
                                             uint32_t gcap, uint32_t *err) {
    uint32_t mask = __ballot_sync(FULL, want);
    if (mask == 0) return;
    uint32_t leader = __ffs(mask) - 1;
    uint32_t base = 0;
    if (lane_id() == leader) base = atomicAdd(cnt, (uint32_t)__popc(mask));
    base = __shfl_sync(FULL, base, leader);
    uint32_t slot = base + (uint32_t)__popc(mask & lanemask_lt());
    bool local = want && slot < cap;
    if (local) buf[slot] = v;
    uint32_t g = warp_append(want && !local, gcount, gcap, err);
    if (g != INF32) gq[g] = v;
}

// Warp-aggregated append of v (lanes with `want`) to a global queue; with
// a stamp array, only lanes whose exchange of stamp[v] to `tag` finds
// another value append (the vertex joins the queue once per tag).  All
// lanes call.
__device__ __forceinline__ void queue_append(bool want, uint32_t v, uint32_t *gq, uint32_t *gcount,
                                             uint32_t gcap, uint32_t *err, uint32_t *stamp,
                                             uint32_t tag) {
    if (want && stamp) want = atomicExch(&stamp[v], tag) != tag;
    const uint32_t g = warp_append(want, gcount, gcap, err);
    if (g != INF32) gq[g] = v;
}

// Warp-synchronous append of v (lanes with `want`) to this warp's own
// region (region[0, *cnt), capacity cap; *cnt is written by this warp
// only).  If the appends do not fit and `flush` allows it, the warp first
// moves the region to the global queue (gq, *gcount, capacity gcap) and
// starts the region over; otherwise the lanes that do not fit go to the
// global queue directly.  Without a stamp array the move is one atomicAdd
// for the whole region; with one (a region that may hold a vertex more than
// once) every item is deduplicated against stamp[v] == tag on its way to
// the queue.  All lanes call.
__device__ __forceinline__ void region_append(bool want, uint32_t v, uint32_t *region,
                                              uint32_t *cnt, uint32_t cap, bool flush,
                                              uint32_t *gq, uint32_t *gcount, uint32_t gcap,
                                              uint32_t *err, uint32_t *stamp = nullptr,
                                              uint32_t tag = 0) {
    const uint32_t mask = __ballot_sync(FULL, want);
    if (mask == 0) return;
    const uint32_t lane = lane_id();
    uint32_t n = *(volatile uint32_t *)cnt;
    const uint32_t k = (uint32_t)__popc(mask);
    if (flush && n + k > cap) {
        n = min(n, cap);
        if (stamp) {
            for (uint32_t i0 = 0; i0 < n; i0 += 32)
                queue_append(i0 + lane < n, i0 + lane < n ? region[i0 + lane] : 0u, gq, gcount,
                             gcap, err, stamp, tag);
        } else {
            uint32_t base = 0;
            if (lane == 0 && n) base = atomicAdd(gcount, n);
            base = __shfl_sync(FULL, base, 0);
            for (uint32_t i = lane; i < n; i += 32) {
                const uint32_t slot = base + i;
                if (slot < gcap) gq[slot] = region[i];
                else atomicOr(err, ERR_CAPACITY);
            }
        }
        __syncwarp();       // the region is read out before it is refilled
        n = 0;
    }
    const uint32_t slot = n + (uint32_t)__popc(mask & lanemask_lt());
    const bool local = want && slot < cap;
    if (local) region[slot] = v;
    queue_append(want && !local, v, gq, gcount, gcap, err, stamp, tag);
    __syncwarp();
    if (lane == 0) *(volatile uint32_t *)cnt = n + k;
    __syncwarp();
}

// Slot of the seed pair (a, b), a < b < k, in the upper-triangle table:
// ascending slot order is ascending (a, b) order.
__host__ __device__ __forceinline__ uint64_t pair_slot(uint64_t a, uint64_t b, uint64_t k) {
    return a * k - a * (a + 1) / 2 + (b - a - 1);
}

// rank pair (a, b) of a table slot: largest a with row start R(a) <= slot
__device__ __forceinline__ void slot_to_pair(uint64_t slot, uint32_t k, uint32_t &ra,
                                             uint32_t &rb) {
    double kk = 2.0 * k - 1.0;
    double disc = kk * kk - 8.0 * (double)slot;
    int64_t a = (int64_t)floor((kk - sqrt(disc > 0 ? disc : 0)) * 0.5);
    if (a < 0) a = 0;
    if (a > (int64_t)k - 2) a = (int64_t)k - 2;
    auto row_start = [k](int64_t x) { return (uint64_t)(x * (2 * (int64_t)k - x - 1) / 2); };
    while (a > 0 && row_start(a) > slot) --a;
    while (a + 1 <= (int64_t)k - 2 && row_start(a + 1) <= slot) ++a;
    ra = (uint32_t)a;
    rb = (uint32_t)(slot - row_start(a) + (uint64_t)a + 1);
}

}  // namespace stn
