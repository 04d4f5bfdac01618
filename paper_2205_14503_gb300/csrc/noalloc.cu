// steiner_voronoi_noalloc: Voronoi cells for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside a
// framework that owns every device allocation through its own pool, code
// that must not grow its memory footprint after start-up, or code that has
// to run while the allocator is unavailable.  They already hold the graph
// and the output arrays in device memory of their own.  This entry point
// computes the same per-vertex cell / distance / predecessor as
// steiner_voronoi on such caller-owned arrays, and keeps all of its working
// memory in one fixed file-scope device array (g_scratch below), so it
// allocates nothing: no cudaMalloc, no cudaFree, no allocating library call.
//
// The scratch array exists on every GPU that loads the library, for the
// lifetime of the process, and bounds the graph size (NA_MAX_VERTICES).
// Every call reuses it: a call clears what must start empty and overwrites
// the rest, so calls that overlap on the GPU (other streams, other host
// threads) race with each other and must be serialised by the caller.
//
// The kernels here are a simpler variant of the library's Voronoi path:
// the same packed (distance << 32 | seed rank) 64-bit atomicMin fixed point,
// run as a plain frontier Bellman-Ford in one cooperative kernel, followed
// by one pass that derives predecessors and writes the outputs.
#include <algorithm>
#include <cstddef>
#include <mutex>
#include <string>

#include "../../include/steiner.h"
#include "common.cuh"

namespace stn {
namespace na {

constexpr uint32_t NA_MAX_VERTICES = STEINER_NOALLOC_MAX_VERTICES;

struct NaControl {
    GridBarrier bar;
    uint32_t err;            // ERR_* bits, plus NA_BAD_INPUT
    uint32_t count[3];       // frontier sizes, rotating by iteration
    uint32_t iterations;
};

constexpr uint32_t NA_BAD_INPUT = 1u << 8;   // seed list, row offsets or arc out of range

// Layout of the scratch array: control block, then per-vertex arrays.
constexpr size_t CTL_BYTES = 256;
constexpr size_t LABEL_OFF = CTL_BYTES;                                   // uint64 [max]
constexpr size_t STAMP_OFF = LABEL_OFF + 8ull * NA_MAX_VERTICES;          // uint32 [max]
constexpr size_t Q0_OFF = STAMP_OFF + 4ull * NA_MAX_VERTICES;             // uint32 [max]
constexpr size_t Q1_OFF = Q0_OFF + 4ull * NA_MAX_VERTICES;                // uint32 [max]
constexpr size_t SCRATCH_BYTES = Q1_OFF + 4ull * NA_MAX_VERTICES;
static_assert(sizeof(NaControl) <= CTL_BYTES, "control block does not fit");

// The only working memory of steiner_voronoi_noalloc (24 MiB + 256 B).
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

struct NaArgs {
    const uint32_t *row_ptr;
    const int32_t *col;
    const uint32_t *w;
    uint32_t n;
    uint64_t n_arcs;
    const int32_t *seeds;
    uint32_t k;
    unsigned char *scratch;     // device address of g_scratch
    uint32_t max_iters;
    int32_t *cell;
    uint32_t *dist;
    int32_t *pred;
};

__device__ __forceinline__ NaControl *ctl_of(const NaArgs &a) {
    return reinterpret_cast<NaControl *>(a.scratch);
}
__device__ __forceinline__ uint64_t *label_of(const NaArgs &a) {
    return reinterpret_cast<uint64_t *>(a.scratch + LABEL_OFF);
}
__device__ __forceinline__ uint32_t *stamp_of(const NaArgs &a) {
    return reinterpret_cast<uint32_t *>(a.scratch + STAMP_OFF);
}
__device__ __forceinline__ uint32_t *queue_of(const NaArgs &a, uint32_t it) {
    return reinterpret_cast<uint32_t *>(a.scratch + ((it & 1) ? Q1_OFF : Q0_OFF));
}

// Clears the control block of the previous call (one thread).
__global__ void na_ctl_reset_kernel(NaArgs a) {
    NaControl *c = ctl_of(a);
    c->bar.count = 0;
    c->bar.gen = 0;
    c->err = 0;
    c->count[0] = c->count[1] = c->count[2] = 0;
    c->iterations = 0;
}

// Clears the per-vertex state of the previous call and checks the row
// offsets (row_ptr[0] = 0, non-decreasing, row_ptr[n] = n_arcs), so that no
// later kernel reads an arc outside [0, n_arcs).
__global__ void na_reset_kernel(NaArgs a) {
    uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    NaControl *c = ctl_of(a);
    if (tid == 0 && (a.row_ptr[0] != 0 || (uint64_t)a.row_ptr[a.n] != a.n_arcs))
        atomicOr(&c->err, NA_BAD_INPUT);
    uint64_t *label = label_of(a);
    uint32_t *stamp = stamp_of(a);
    bool bad = false;
    for (uint32_t v = tid; v < a.n; v += gridDim.x * blockDim.x) {
        label[v] = INF64;
        stamp[v] = 0;
        bad |= a.row_ptr[v] > a.row_ptr[v + 1];
    }
    if (bad) atomicOr(&c->err, NA_BAD_INPUT);
}

// Seeds (ascending, distinct, in range) at distance 0 on the first frontier.
__global__ void na_seed_kernel(NaArgs a) {
    uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.k) return;
    NaControl *c = ctl_of(a);
    int32_t s = a.seeds[r];
    bool ok = s >= 0 && (uint32_t)s < a.n && (r == 0 || a.seeds[r - 1] < s);
    if (!ok) {
        atomicOr(&c->err, NA_BAD_INPUT);
        return;
    }
    label_of(a)[s] = (uint64_t)r;
    stamp_of(a)[s] = 1;
    queue_of(a, 0)[r] = (uint32_t)s;
    if (r == 0) c->count[0] = a.k;
}

// Frontier Bellman-Ford: iteration `it` relaxes the arcs of its frontier,
// pushing every vertex whose label drops (once per iteration, by stamp).
__global__ void __launch_bounds__(256) na_sssp_kernel(NaArgs a) {
    NaControl *c = ctl_of(a);
    uint64_t *label = label_of(a);
    uint32_t *stamp = stamp_of(a);
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const bool first = blockIdx.x == 0 && threadIdx.x == 0;
    if (ldcg_u32(&c->err) & NA_BAD_INPUT) return;   // set by the reset or seed kernel: all blocks agree
    for (uint32_t it = 0;; ++it) {
        uint32_t nf = min(ldcg_u32(&c->count[it % 3]), a.n);
        if (first) c->count[(it + 2) % 3] = 0;
        const uint32_t *qc = queue_of(a, it);
        uint32_t *qn = queue_of(a, it + 1);
        uint32_t *cn = &c->count[(it + 1) % 3];
        const uint32_t tag = it + 2;
        for (uint32_t b0 = warp * 32; b0 < nf; b0 += nwarps * 32) {
            uint32_t i = b0 + lane;
            uint32_t s = 0, deg = 0;
            uint64_t lab = INF64;
            if (i < nf) {
                uint32_t u = ldcg_u32(&qc[i]);
                s = a.row_ptr[u];
                deg = a.row_ptr[u + 1] - s;
                lab = ldcg_u64(&label[u]);
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
                uint64_t lo = __shfl_sync(FULL, lab, owner);
                bool push = false;
                uint32_t v = 0;
                if (valid) {
                    uint32_t arc = so + (j - eo);
                    int32_t cv = a.col[arc];
                    if (cv < 0 || (uint32_t)cv >= a.n) {
                        atomicOr(&c->err, NA_BAD_INPUT);
                    } else {
                        v = (uint32_t)cv;
                        uint64_t nd = (lo >> 32) + (uint64_t)a.w[arc];
                        if (nd < INF32) {
                            uint64_t nl = (nd << 32) | (lo & 0xFFFFFFFFull);
                            uint64_t old = atomicMin(reinterpret_cast<unsigned long long *>(&label[v]),
                                                     (unsigned long long)nl);
                            if (nl < old) push = atomicExch(&stamp[v], tag) != tag;
                        }
                    }
                }
                uint32_t slot = warp_append(push, cn, a.n, &c->err);
                if (slot != INF32) qn[slot] = v;
            }
        }
        if (!grid_sync(&c->bar, &c->err)) return;
        if (it + 1 >= a.max_iters) {
            if (first) atomicOr(&c->err, ERR_TIMEOUT);
            return;
        }
        if (ldcg_u32(&c->count[(it + 1) % 3]) == 0) {
            if (first) c->iterations = it + 1;
            return;
        }
    }
}

// pred(v) = smallest-id tight neighbour in v's cell; outputs in the
// steiner_voronoi format.  A reached vertex next to an unreached one means
// a distance did not fit below 2^32 - 1 (ERR_OVERFLOW).
// A rejected input (NA_BAD_INPUT) leaves the caller's outputs untouched.
__global__ void na_export_kernel(NaArgs a) {
    NaControl *c = ctl_of(a);
    if (ldcg_u32(&c->err) & NA_BAD_INPUT) return;
    const uint64_t *label = label_of(a);
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < a.n; v += gridDim.x * blockDim.x) {
        uint64_t lv = label[v];
        int32_t p = -1;
        bool overflow = false;
        if (lv != INF64) {
            uint64_t dv = lv >> 32;
            if (dv == 0) p = (int32_t)v;
            for (uint32_t e = a.row_ptr[v]; e < a.row_ptr[v + 1]; ++e) {
                int32_t cu = a.col[e];
                if (cu < 0 || (uint32_t)cu >= a.n) continue;
                uint64_t lu = label[cu];
                if (lu == INF64) {
                    overflow = true;
                    continue;
                }
                if (p < 0 && (uint32_t)lu == (uint32_t)lv && (lu >> 32) + a.w[e] == dv) p = cu;
            }
        }
        if (overflow) atomicOr(&c->err, ERR_OVERFLOW);
        if (a.cell) a.cell[v] = lv == INF64 ? -1 : a.seeds[(uint32_t)lv];
        if (a.dist) a.dist[v] = lv == INF64 ? INF32 : (uint32_t)(lv >> 32);
        if (a.pred) a.pred[v] = p;
    }
}

// Per-device set-up: the device address of g_scratch (host code cannot use
// the symbol itself) and the cooperative grid size.
struct DeviceSetup {
    bool ready = false;
    unsigned char *scratch = nullptr;
    int blocks = 0;
    int sms = 0;
};
constexpr int NA_MAX_DEVICES = 64;
static DeviceSetup g_setup[NA_MAX_DEVICES];
static std::mutex g_setup_mu;

static int setup_device(int dev, DeviceSetup &out, const char **why) {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    DeviceSetup &s = g_setup[dev];
    if (!s.ready) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess) {
            *why = cudaGetErrorString(e);
            return STEINER_ECUDA;
        }
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, na_sssp_kernel, 256, 0);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess || per_sm < 1) {
            *why = e != cudaSuccess ? cudaGetErrorString(e) : "kernel does not fit on an SM";
            return STEINER_ECUDA;
        }
        s.scratch = static_cast<unsigned char *>(ptr);
        s.blocks = per_sm * sms;
        s.sms = sms;
        s.ready = true;
    }
    out = s;
    return STEINER_OK;
}

}  // namespace na

void api_set_error(const std::string &msg);

}  // namespace stn

using namespace stn;
using namespace stn::na;

extern "C" int steiner_voronoi_noalloc(const uint32_t *row_ptr, const int32_t *col,
                                       const uint32_t *w, uint32_t n, uint64_t n_arcs,
                                       const int32_t *seeds, uint32_t k, int32_t *cell,
                                       uint32_t *dist, int32_t *pred, void *stream) {
    if (n > NA_MAX_VERTICES) {
        api_set_error("steiner_voronoi_noalloc: n exceeds its fixed scratch limit of "
                      "STEINER_NOALLOC_MAX_VERTICES (1048576) vertices");
        return STEINER_ENOMEM;
    }
    if (n == 0 || k == 0 || k > n || !row_ptr || !seeds || (n_arcs && (!col || !w)) ||
        n_arcs >= 0xFFFFFFFFull) {
        api_set_error("steiner_voronoi_noalloc: invalid arguments");
        return STEINER_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        api_set_error("steiner_voronoi_noalloc: no usable current device");
        return STEINER_ECUDA;
    }
    DeviceSetup su;
    const char *why = "";
    int rc = setup_device(dev, su, &why);
    if (rc) {
        api_set_error(std::string("steiner_voronoi_noalloc set-up: ") + why);
        return rc;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    NaArgs a{row_ptr, col, w, n, n_arcs, seeds, k, su.scratch, 1u << 22, cell, dist, pred};
    unsigned grid = (unsigned)std::min<uint64_t>((n + 255) / 256, (uint64_t)su.sms * 16);
    na_ctl_reset_kernel<<<1, 1, 0, s>>>(a);
    na_reset_kernel<<<grid, 256, 0, s>>>(a);
    na_seed_kernel<<<(k + 255) / 256, 256, 0, s>>>(a);
    void *args[] = {&a};
    e = cudaLaunchCooperativeKernel((const void *)na_sssp_kernel, dim3(su.blocks), dim3(256), args,
                                    0, s);
    if (e == cudaSuccess) {
        na_export_kernel<<<grid, 256, 0, s>>>(a);
        e = cudaGetLastError();
    }
    uint32_t err = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&err, su.scratch + offsetof(NaControl, err), sizeof(err),
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        api_set_error(std::string("steiner_voronoi_noalloc: ") + cudaGetErrorString(e));
        return STEINER_ECUDA;
    }
    if (err & NA_BAD_INPUT) {
        api_set_error("steiner_voronoi_noalloc: seeds must be distinct, ascending and below n, "
                      "row_ptr must run from 0 to n_arcs without decreasing, and every "
                      "neighbour id must be below n");
        return STEINER_EINVAL;
    }
    if (err & (ERR_BARRIER | ERR_TIMEOUT)) {
        api_set_error("steiner_voronoi_noalloc: device loop or barrier hit its cap");
        return STEINER_ETIMEOUT;
    }
    if (err & ERR_OVERFLOW) {
        api_set_error("steiner_voronoi_noalloc: a distance reached 2^32 - 1");
        return STEINER_EOVERFLOW;
    }
    if (err & ERR_CAPACITY) {
        api_set_error("steiner_voronoi_noalloc: frontier capacity exceeded");
        return STEINER_ENOMEM;
    }
    return STEINER_OK;
}
