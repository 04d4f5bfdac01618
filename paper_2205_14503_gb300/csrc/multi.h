// Multi-query engine state shared by the batch and serving entry points.
//
// Up to MQ_SLOTS queries ("slots") run in one persistent kernel over the
// resident graph.  Per-vertex state is vertex-major: the labels of vertex v
// for all slots are label[v * MQ_SLOTS + q], so relaxing one arc for every
// pending slot touches one contiguous 256-byte run (32-bit labels), and each CSR row is
// read once per frontier visit for all the slots that need it (a 64-bit
// mask per vertex says which).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/steiner.h"
#include "internal.h"

struct steiner_graph;

namespace stn {

constexpr int MQ_SLOTS = 64;

struct MqControl {
    GridBarrier bar;
    uint32_t err;                 // ERR_* (global)
    uint32_t it;                  // next iteration (persists across launches)
    uint32_t fc;                  // far pile being filled
    // doorbell as seen by block 0 before the barrier that ends iteration i,
    // at stop_req[i & 1] (two copies: a slow block still reading one copy
    // never sees block 0 overwrite it with the next iteration's)
    uint32_t stop_req[2];
    uint32_t near_count[3];
    uint32_t far_count[2];
    unsigned long long act[3];    // slots with near work queued, per iteration slot
    unsigned long long inflight;  // admitted, not yet converged (host-written)
    unsigned long long converged; // converged slots (kernel-written, host clears)
    unsigned long long slot_overflow;   // per-slot overflow seen by the scan
    unsigned long long T[MQ_SLOTS];     // near/far threshold per slot
    uint32_t fmin[2][MQ_SLOTS];         // lower bound of far distances per slot
    int32_t far_pending[MQ_SLOTS];      // set far bits per slot
    uint32_t exit_reason;               // 1 all converged, 2 slot converged, 3 yield, 4 cap, 5 barrier
    uint32_t iterations;                // iterations run by the last launch
    unsigned long long relax_attempts;
    unsigned long long relax_improved;
    // block 0's time in each part of an iteration (ns, accumulated): masks +
    // prefix sums, barrier after them, relaxation, flush + barrier, split
    unsigned long long t_part[5];
    unsigned long long items_total;     // frontier items visited
    unsigned long long pairs_total;     // (arc, slot) pairs relaxed
    // light/heavy arc split, per slot (as in the single-query kernel)
    unsigned long long hp_done;         // slots whose current band had its heavy-arc pass
    unsigned long long hpass;           // slots whose heavy-arc pass runs in the next iteration
    uint32_t blist;                     // band list receiving appends (rotates over 3)
    uint32_t bcount[3];
    uint32_t lshift[MQ_SLOTS];          // rank bits of each slot's 32-bit labels
    unsigned long long slot_narrow;     // slots with a distance too large for their labels
    // slots still in their first band (set at admission, cleared by the
    // slot's first split): their heavy-arc pass may run in the pull form
    unsigned long long band0;
    uint32_t pull_sweeps;               // pull-form passes run (accumulated)
};

struct MqState {
    uint32_t n = 0;
    uint32_t *label = nullptr;              // n * MQ_SLOTS: (dist << lshift[q]) | rank
    uint32_t *pred = nullptr;               // n * MQ_SLOTS (pred arc per slot)
    unsigned long long *nmask = nullptr;    // n
    unsigned long long *fmask = nullptr;    // n
    uint32_t *stamp_near = nullptr;         // n
    uint32_t *in_far = nullptr;             // n
    uint32_t *q[2] = {nullptr, nullptr};    // frontier, n
    unsigned long long *item_mask = nullptr;    // 2n: slot mask taken by each work item
    uint64_t *item_pre = nullptr;           // 2n: pair prefix within its block segment
    unsigned long long *bmask = nullptr;    // n: slots that relaxed v in their current band
    uint32_t *bl[3] = {nullptr, nullptr, nullptr};  // band lists, n each
    uint64_t *bsum = nullptr;               // pairs per block segment
    uint32_t *far[2] = {nullptr, nullptr};  // n
    MqControl *ctl = nullptr;
    uint64_t *pairtab[MQ_SLOTS] = {};       // per-slot pair table
    uint64_t pairtab_cap[MQ_SLOTS] = {};
    uint64_t **d_pairtab = nullptr;         // device copy of the pointers
    uint32_t *d_k = nullptr;                // device copy of the slot sizes
    int32_t *seeds[MQ_SLOTS] = {};          // per-slot sorted seeds
    uint32_t seeds_cap[MQ_SLOTS] = {};
    uint32_t base_near = 1;                 // stamp tags are base_near + it
};

// Batched tails (tails.cu): one retiring slot, and its results.
struct TailSlot {
    const uint64_t *pairtab;     // its pair table, k (k - 1) / 2 entries
    uint64_t n_slots;
    uint64_t tile0;              // first tile of its table in the global tile numbering
    uint32_t k;
    uint32_t q;                  // engine slot: its pred column
    uint32_t comp0;              // first of its k MST scratch entries
    uint32_t pad;
};

struct TailOut {
    uint32_t pair0, n_pairs;     // its segment of the concatenated pair list
    uint32_t n_mst;              // MST pairs
    uint32_t n_edges;            // distinct tree edges
    unsigned long long total;    // D(G_S)
};

// Device workspace of the batched tails, grown on demand.
struct TailWs {
    TailSlot *d_slots = nullptr, *h_slots = nullptr;
    TailOut *d_out = nullptr, *h_out = nullptr;
    Control *ctl = nullptr, *h_ctl = nullptr;
    uint32_t *tile_cnt = nullptr;
    uint64_t tile_cap = 0;
    uint64_t *e_key = nullptr;
    uint32_t *e_ra = nullptr, *e_rb = nullptr, *e_arc = nullptr, *e_mst = nullptr,
             *e_owner = nullptr;
    uint64_t e_cap = 0;
    uint32_t *comp = nullptr, *hook = nullptr;
    unsigned long long *best = nullptr;
    uint64_t comp_cap = 0;
    uint64_t *key0 = nullptr, *key1 = nullptr;
    uint32_t *w0 = nullptr, *w1 = nullptr;
    uint64_t key_cap = 0;
    uint64_t tree_cap = 0;       // edges the walkers may emit before a fallback
    uint32_t *hist = nullptr;
};

void tail_ws_free(TailWs &t);
// Steps 3-7 of Algorithm 2 for r retiring slots (engine slots qs[i], seed
// counts ks[i] >= 2, pred columns and pair tables in m) with one launch per
// step.  Fills res[i] (edges allocated with malloc) and returns STEINER_OK;
// on a buffer shortfall returns STEINER_ENOMEM with no results, and the
// caller runs those slots one at a time.
int run_batched_tails(steiner_graph *G, MqState &m, TailWs &t, const int *qs, const uint32_t *ks,
                      int r, steiner_result_t *res);

cudaError_t mq_alloc(const DevGraph &g, MqState &m, cudaStream_t s);
void mq_free(MqState &m);
int mq_occupancy(int threads);

// Admission: clear the label/pred columns of the slots in `mask`, then
// seed slot q from the k sorted seeds already copied to m.seeds[q].
cudaError_t mq_launch_clear(const DevGraph &g, MqState &m, unsigned long long mask,
                            cudaStream_t s);
cudaError_t mq_launch_seed(const DevGraph &g, MqState &m, int q, uint32_t k, uint32_t delta,
                           cudaStream_t s);
// Runs the persistent multi-query SSSP.  yield > 0: return once `yield`
// slots converged or *doorbell (host-mapped) is set; yield = 0: run until
// every in-flight slot converged.  max_iters caps this launch.
cudaError_t mq_launch_sssp(const DevGraph &g, MqState &m, int blocks, uint32_t delta, uint32_t pull,
                           uint32_t max_iters, uint32_t yield, const uint32_t *doorbell,
                           cudaStream_t s);
// Clears the shared frontier state (after an error).
cudaError_t mq_reset(MqState &m, cudaStream_t s);
// Predecessors and per-slot bridge tables for the slots in `slots`.
cudaError_t mq_launch_scan(const DevGraph &g, MqState &m, unsigned long long slots,
                           cudaStream_t s);

}  // namespace stn
