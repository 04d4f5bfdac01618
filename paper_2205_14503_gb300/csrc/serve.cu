// Batched and serving modes over the multi-query engine (multi.cu).
//
// The engine owns MQ_SLOTS query slots on the resident graph.  A query is
// admitted into a free slot (its label column cleared, its seeds placed on
// the shared frontier), the persistent multi-query kernel runs until some
// slot converges (or, when serving, until the host rings the doorbell
// because new requests wait and slots are free), converged slots run their
// tails (batched pred + bridge scan, then per-slot compaction, MST,
// expansion and sort) and are released, and freed slots take the next
// queries.  Admission is bounded by a device-memory budget for per-query
// state (the slot's label and predecessor columns plus its pair table).
//
//  steiner_query_batch   runs a list of queries to completion this way.
//  steiner_serve_*       a worker thread runs the same loop continuously over
//                        a request queue fed by steiner_submit; results are
//                        collected with steiner_poll (continuous batching:
//                        requests join while others are on the device).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "engine.h"
#include "multi.h"

namespace stn {

namespace {
double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
}  // namespace

struct SlotInfo {
    bool busy = false;
    uint64_t tag = 0;              // caller's handle (batch index or ticket)
    uint32_t k = 0;
    uint64_t bytes = 0;            // per-query device state charged to the budget
};

struct BatchEngine {
    steiner_graph *G = nullptr;
    MqState m;
    bool ready = false;
    int blocks = 0;
    uint32_t delta = 1;
    uint32_t *doorbell_host = nullptr;   // pinned, mapped
    uint32_t *doorbell_dev = nullptr;
    MqControl *h_ctl = nullptr;          // pinned
    unsigned long long *h_masks = nullptr;   // pinned staging for mask uploads
    unsigned long long inflight = 0;
    SlotInfo slots[MQ_SLOTS];
    uint64_t budget = ~0ull, used = 0, fixed = 0;
    uint64_t total_iterations = 0;
    uint64_t iteration_cap = 1ull << 24;
    // Band width of every slot's near/far threshold (0 = the graph's
    // single-query default).
    uint32_t batch_delta = 0;
    // 1: each slot's first heavy-arc pass runs in the pull form (unsettled
    // vertices read their heavy arcs); 0: every pass pushes
    uint32_t pull = 1;
    // A yielding launch returns once popc(in flight) / yield_div slots
    // converged (at least one), or when the doorbell rings (a request waits
    // and a slot is free).  1 (the default) retires whole waves: slots that
    // started together keep their frontiers aligned, so one CSR row visit
    // serves many slots and one retirement scan covers many queries;
    // larger divisors retire earlier, in smaller groups.
    uint32_t yield_div = 1;
    // Retiring slots' tails (Steps 3-7) in one launch per step for all of
    // them (1, the default) or slot by slot through the single-query
    // kernels (0; also the fallback when the batched buffers fall short).
    uint32_t batched_tails = 1;
    TailWs tails;
    // cumulative wall time (ms) and counters, for tracing
    double ms_sssp = 0, ms_scan = 0, ms_tail = 0, ms_admit = 0;
    uint64_t launches = 0, relax_attempts = 0, iterations_run = 0;
    // admissions, and those made while other slots were on the device
    // (continuous batching: a query joins a running batch)
    uint64_t admitted = 0, admitted_busy = 0;
    uint64_t tail_batches = 0;          // retirements whose tails ran batched
    std::atomic<int> free_slots{MQ_SLOTS};

    int init() {
        if (ready) return STEINER_OK;
        const DevGraph &g = api_graph(G);
        cudaStream_t s = api_stream(G);
        cudaError_t e = mq_alloc(g, m, s);
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&doorbell_host, 64, cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&doorbell_dev, doorbell_host, 0);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&h_ctl, sizeof(MqControl));
        if (e == cudaSuccess) e = cudaMallocHost((void **)&h_masks, 64);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            api_set_error(std::string("multi-query engine set-up: ") + cudaGetErrorString(e));
            release();
            return e == cudaErrorMemoryAllocation ? STEINER_ENOMEM : STEINER_ECUDA;
        }
        *doorbell_host = 0;
        int per_sm = mq_occupancy(256);
        int sms = api_geometry(G).sm_count;
        blocks = std::max(1, per_sm) * sms;
        fixed = (uint64_t)g.n * MQ_SLOTS * 12;
        ready = true;
        return STEINER_OK;
    }

    void release() {
        mq_free(m);                      // also after a partial mq_alloc
        tail_ws_free(tails);
        if (doorbell_host) cudaFreeHost(doorbell_host);
        if (h_ctl) cudaFreeHost(h_ctl);
        if (h_masks) cudaFreeHost(h_masks);
        doorbell_host = nullptr;
        h_ctl = nullptr;
        h_masks = nullptr;
        ready = false;
    }

    // Band width: batch_delta if set; else, on a graph whose tuned delta is
    // at or below the largest weight (the light/heavy split pays there), an
    // eighth of the largest weight (the batched kernel shares each
    // iteration's cost over all slots, so it gains from narrower bands than
    // one query does: R-MAT 22 / 24 batches run ~1.6x faster at w_max / 8
    // than with the split off); else the graph's delta.
    uint32_t cur_delta() const {
        if (batch_delta) return batch_delta;
        const uint32_t d = api_delta(G), wmax = api_graph(G).max_w;
        if (d <= wmax && wmax >= 8) return wmax / 8;
        return d;
    }

    int free_slot() const {
        for (int q = 0; q < MQ_SLOTS; ++q)
            if (!slots[q].busy) return q;
        return -1;
    }

    static uint64_t state_bytes(uint32_t k) {
        uint64_t pairs = k > 1 ? (uint64_t)k * (k - 1) / 2 : 0;
        return pairs * 8;
    }

    bool fits(uint32_t k) const { return used + state_bytes(k) <= budget; }

    // Admission in two steps: stage() reserves slot q for sorted seeds
    // (buffers, copies), commit() clears the staged slots' columns in one
    // pass, seeds them and waits once.  Caller holds the graph mutex.
    unsigned long long staged = 0;
    std::vector<std::vector<int32_t>> staged_seeds = std::vector<std::vector<int32_t>>(MQ_SLOTS);
    // each busy slot's sorted seeds, kept until release: a slot whose
    // distances outgrow its 32-bit labels runs again as a single query
    std::vector<std::vector<int32_t>> slot_seeds = std::vector<std::vector<int32_t>>(MQ_SLOTS);
    uint64_t narrow_reruns = 0;

    int admit(int q, const std::vector<int32_t> &ss, uint64_t tag) {
        int rc = stage(q, ss, tag);
        return rc ? rc : commit();
    }

    int commit() {
        if (!staged) return STEINER_OK;
        double t0 = now_s();
        cudaStream_t s = api_stream(G);
        cudaError_t e = mq_launch_clear(api_graph(G), m, staged, s);
        for (unsigned long long mm = staged; mm && e == cudaSuccess; mm &= mm - 1) {
            int q = __builtin_ctzll(mm);
            e = mq_launch_seed(api_graph(G), m, q, slots[q].k, cur_delta(), s);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        unsigned long long done = staged;
        staged = 0;
        for (unsigned long long mm = done; mm; mm &= mm - 1) staged_seeds[__builtin_ctzll(mm)].clear();
        ms_admit += 1e3 * (now_s() - t0);
        if (e != cudaSuccess) {
            api_set_error(std::string("admission: ") + cudaGetErrorString(e));
            return STEINER_ECUDA;
        }
        return STEINER_OK;
    }

    int stage(int q, const std::vector<int32_t> &ss, uint64_t tag) {
        cudaStream_t s = api_stream(G);
        uint32_t k = (uint32_t)ss.size();
        uint64_t pairs = k > 1 ? (uint64_t)k * (k - 1) / 2 : 0;
        if (pairs > (1ull << 28)) {
            api_set_error("seed set too large for the pair table (k(k-1)/2 > 2^28)");
            return STEINER_ENOMEM;
        }
        cudaError_t e = cudaSuccess;
        if (k > m.seeds_cap[q]) {
            if (m.seeds[q]) e = cudaFreeAsync(m.seeds[q], s);
            m.seeds[q] = nullptr;
            if (e == cudaSuccess) e = cudaMallocAsync((void **)&m.seeds[q], (size_t)k * 4, s);
            m.seeds_cap[q] = e == cudaSuccess ? k : 0;
        }
        if (e == cudaSuccess && pairs > m.pairtab_cap[q]) {
            if (m.pairtab[q]) e = cudaFreeAsync(m.pairtab[q], s);
            m.pairtab[q] = nullptr;
            if (e == cudaSuccess) e = cudaMallocAsync((void **)&m.pairtab[q], pairs * 8, s);
            m.pairtab_cap[q] = e == cudaSuccess ? pairs : 0;
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(&m.d_pairtab[q], &m.pairtab[q], sizeof(uint64_t *),
                                    cudaMemcpyHostToDevice, s);
        }
        staged_seeds[q] = ss;     // host copy lives until commit() has waited
        slot_seeds[q] = ss;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(m.seeds[q], staged_seeds[q].data(), (size_t)k * 4,
                                cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&m.d_k[q], &k, 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && pairs) e = cudaMemsetAsync(m.pairtab[q], 0xFF, pairs * 8, s);
        if (e != cudaSuccess) {
            api_set_error(std::string("admission: ") + cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? STEINER_ENOMEM : STEINER_ECUDA;
        }
        ++admitted;
        if (inflight & ~staged) ++admitted_busy;
        slots[q].busy = true;
        slots[q].tag = tag;
        slots[q].k = k;
        slots[q].bytes = state_bytes(k);
        used += slots[q].bytes;
        inflight |= 1ull << q;
        staged |= 1ull << q;
        free_slots.fetch_sub(1);
        return STEINER_OK;
    }

    // Runs the persistent kernel; returns the newly converged slots in
    // *done (slots stopped by an error are reported in *failed with *why).
    // yield: leave the kernel early (retire converged slots, admit waiting
    // queries): once popc(in flight) / yield_div slots converged (at least
    // one; by default all of them, a whole wave), so that one retirement
    // scan is shared by several slots, or when the doorbell rings.
    int run(bool yield, unsigned long long *done, unsigned long long *failed, int *why) {
        cudaStream_t s = api_stream(G);
        *done = *failed = 0;
        *why = STEINER_OK;
        double t0 = now_s();
        ++launches;
        h_masks[0] = inflight;
        h_masks[1] = 0;
        delta = cur_delta();
        api_ensure_partition(G, delta);
        cudaError_t e = cudaMemcpyAsync(&m.ctl->inflight, &h_masks[0], 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&m.ctl->converged, &h_masks[1], 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = mq_launch_sssp(api_graph(G), m, blocks, delta, pull, 1u << 20,
                               yield ? std::max(1u, (uint32_t)__builtin_popcountll(inflight) / yield_div) : 0u,
                               doorbell_dev, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_ctl, m.ctl, sizeof(MqControl), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            api_set_error(std::string("multi-query kernel: ") + cudaGetErrorString(e));
            *failed = inflight;
            *why = STEINER_ECUDA;
            return STEINER_ECUDA;
        }
        total_iterations += h_ctl->iterations;
        iterations_run += h_ctl->iterations;
        relax_attempts = h_ctl->relax_attempts;
        ms_sssp += 1e3 * (now_s() - t0);
        if (h_ctl->err & (ERR_BARRIER | ERR_CAPACITY)) {
            *failed = inflight;
            *why = (h_ctl->err & ERR_BARRIER) ? STEINER_ETIMEOUT : STEINER_ENOMEM;
            api_set_error("multi-query kernel: barrier or capacity error");
            return *why;
        }
        *done = h_ctl->converged & inflight;
        if (total_iterations > iteration_cap) {
            *failed = inflight & ~*done;
            *why = STEINER_ETIMEOUT;
        }
        return STEINER_OK;
    }

    // Tails of the slots in `mask`; results go to out(tag, result).
    template <class Out>
    void retire(unsigned long long mask, Out out) {
        if (!mask) return;
        cudaStream_t s = api_stream(G);
        double t0 = now_s();
        cudaError_t e = mq_launch_scan(api_graph(G), m, mask, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_ctl, m.ctl, sizeof(MqControl), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        double t1 = now_s();
        ms_scan += 1e3 * (t1 - t0);
        // slots without overflow: their tails all at once
        int bq[MQ_SLOTS];
        uint32_t bk[MQ_SLOTS];
        int nb = 0;
        const unsigned long long narrow = e == cudaSuccess ? h_ctl->slot_narrow : 0ull;
        if (e == cudaSuccess && batched_tails)
            for (unsigned long long mm = mask & ~narrow; mm; mm &= mm - 1) {
                const int q = __builtin_ctzll(mm);
                if (!((h_ctl->slot_overflow >> q) & 1ull) && slots[q].k > 1) {
                    bq[nb] = q;
                    bk[nb++] = slots[q].k;
                }
            }
        steiner_result_t bres[MQ_SLOTS];
        const bool batched = nb > 0 && run_batched_tails(G, m, tails, bq, bk, nb, bres) == STEINER_OK;
        if (batched) ++tail_batches;
        int bi = 0;
        for (unsigned long long mm = mask; mm; mm &= mm - 1) {
            int q = __builtin_ctzll(mm);
            steiner_result_t r{};
            if (e != cudaSuccess) {
                r.status = STEINER_ECUDA;
                api_set_error(std::string("batched scan: ") + cudaGetErrorString(e));
            } else if ((narrow >> q) & 1ull) {
                // a distance outgrew the slot's 32-bit labels: the query runs
                // alone through the single-query path (64-bit labels as needed)
                ++narrow_reruns;
                api_query_locked(G, slot_seeds[q].data(), slots[q].k, &r);
            } else if (batched && bi < nb && bq[bi] == q) {
                r = bres[bi++];
            } else {
                bool ovf = (h_ctl->slot_overflow >> q) & 1ull;
                api_run_tail(G, m.pairtab[q], m.pred + q, MQ_SLOTS, slots[q].k, ovf, &r);
            }
            out(slots[q].tag, r);
            release_slot(q);
        }
        ms_tail += 1e3 * (now_s() - t1);
    }

    template <class Out>
    void fail_slots(unsigned long long mask, int why, Out out) {
        for (unsigned long long mm = mask; mm; mm &= mm - 1) {
            int q = __builtin_ctzll(mm);
            steiner_result_t r{};
            r.status = why;
            out(slots[q].tag, r);
            release_slot(q);
        }
        if (mask) reset_device_state();
    }

    void release_slot(int q) {
        slot_seeds[q].clear();
        used -= slots[q].bytes;
        slots[q] = SlotInfo();
        inflight &= ~(1ull << q);
        free_slots.fetch_add(1);
    }

    // After an error the shared frontier may hold stale entries: clear it.
    void reset_device_state() {
        cudaStream_t s = api_stream(G);
        mq_reset(m, s);
        cudaStreamSynchronize(s);
        cudaGetLastError();
        total_iterations = 0;
    }
};

void destroy_batch(BatchEngine *b) {
    if (!b) return;
    b->release();
    delete b;
}

// Tracing counters of the multi-query engine (steiner_get_param keys
// "batch_ms_sssp", "batch_ms_scan", "batch_ms_tail", "batch_ms_admit",
// "batch_launches", "batch_iterations", "batch_relax_attempts",
// "batch_admitted", "batch_admitted_busy"; "batch_reset" clears them).

int64_t batch_counter(BatchEngine *B, const char *key) {
    if (!B) return -1;
    std::string k(key);
    if (k == "batch_ms_sssp") return (int64_t)(B->ms_sssp * 1000);
    if (k == "batch_ms_scan") return (int64_t)(B->ms_scan * 1000);
    if (k == "batch_ms_tail") return (int64_t)(B->ms_tail * 1000);
    if (k == "batch_ms_admit") return (int64_t)(B->ms_admit * 1000);
    if (k == "batch_launches") return (int64_t)B->launches;
    if (k == "batch_iterations") return (int64_t)B->iterations_run;
    if (k == "batch_relax_attempts") return (int64_t)B->relax_attempts;
    if (k == "batch_admitted") return (int64_t)B->admitted;
    if (k == "batch_admitted_busy") return (int64_t)B->admitted_busy;
    if (k == "batch_tails") return B->batched_tails;
    if (k == "batch_pull") return B->pull;
    if (k == "batch_pull_sweeps" && B->h_ctl) return (int64_t)B->h_ctl->pull_sweeps;
    if (k == "batch_tail_batches") return (int64_t)B->tail_batches;
    if (k == "batch_narrow_reruns") return (int64_t)B->narrow_reruns;
    if (k == "batch_delta") return B->cur_delta();
    if (k == "batch_yield_div") return B->yield_div;
    if (k.rfind("batch_t", 0) == 0 && k.size() == 8 && B->h_ctl) return (int64_t)B->h_ctl->t_part[k[7] - '0'];
    if (k == "batch_items" && B->h_ctl) return (int64_t)B->h_ctl->items_total;
    if (k == "batch_pairs" && B->h_ctl) return (int64_t)B->h_ctl->pairs_total;
    if (k == "batch_reset") {
        B->ms_sssp = B->ms_scan = B->ms_tail = B->ms_admit = 0;
        B->launches = B->iterations_run = 0;
        B->admitted = B->admitted_busy = B->tail_batches = 0;
        return 0;
    }
    return -1;
}

static BatchEngine *engine_of(steiner_graph *G) {
    BatchEngine *&B = api_batch(G);
    if (!B) {
        B = new BatchEngine();
        B->G = G;
    }
    return B;
}

// Engine settings (steiner_set_param keys "batch_delta", "batch_pull", "batch_tails",
// "batch_yield_div").
int batch_set_param(steiner_graph *G, const char *key, int64_t value) {
    BatchEngine *B = engine_of(G);
    std::string k(key);
    if (k == "batch_delta") {
        if (value < 0 || value > 0x7FFFFFFF) {
            api_set_error("batch_delta out of range");
            return STEINER_EINVAL;
        }
        B->batch_delta = (uint32_t)value;
        return STEINER_OK;
    }
    if (k == "batch_pull") {
        if (value != 0 && value != 1) {
            api_set_error("batch_pull must be 0 or 1");
            return STEINER_EINVAL;
        }
        B->pull = (uint32_t)value;
        return STEINER_OK;
    }
    if (k == "batch_tails") {
        if (value != 0 && value != 1) {
            api_set_error("batch_tails must be 0 or 1");
            return STEINER_EINVAL;
        }
        B->batched_tails = (uint32_t)value;
        return STEINER_OK;
    }
    if (k == "batch_yield_div") {
        if (value < 1 || value > MQ_SLOTS) {
            api_set_error("batch_yield_div out of range (1..64)");
            return STEINER_EINVAL;
        }
        B->yield_div = (uint32_t)value;
        return STEINER_OK;
    }
    api_set_error(std::string("unknown parameter ") + key);
    return STEINER_EINVAL;
}

// ---------------------------------------------------------------------------
// serving
// ---------------------------------------------------------------------------

struct ServeJob {
    uint64_t ticket;
    std::vector<int32_t> seeds;     // sorted
    double t_submit;
};

struct ServeEngine {
    steiner_graph *G = nullptr;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<ServeJob> queue;
    std::unordered_map<uint64_t, steiner_result_t> done;
    // tickets issued and not yet returned by steiner_poll (queued, on the
    // device, or finished and waiting in `done`)
    std::unordered_set<uint64_t> live;
    std::unordered_map<uint64_t, double> t_submit;
    uint64_t next_ticket = 1;
    uint32_t max_queue = 1u << 16;
    bool stop = false;

    void run() {
        cudaSetDevice(api_device(G));
        BatchEngine *B = nullptr;
        for (;;) {
            std::vector<ServeJob> take;
            {
                std::unique_lock<std::mutex> lk(mu);
                bool idle = !B || B->inflight == 0;
                if (idle)
                    cv.wait(lk, [&] { return stop || !queue.empty(); });
                if (stop && queue.empty() && (!B || B->inflight == 0)) return;
                while (!queue.empty()) {
                    take.push_back(std::move(queue.front()));
                    queue.pop_front();
                }
            }
            std::vector<std::pair<uint64_t, steiner_result_t>> finished;
            auto out = [&](uint64_t tag, const steiner_result_t &r) { finished.emplace_back(tag, r); };
            std::deque<ServeJob> waiting(std::make_move_iterator(take.begin()),
                                         std::make_move_iterator(take.end()));
            {
                std::lock_guard<std::mutex> glk(api_mutex(G));
                B = engine_of(G);
                int rc = B->init();
                if (rc) {
                    for (auto &j : waiting) {
                        steiner_result_t r{};
                        r.status = rc;
                        out(j.ticket, r);
                    }
                    waiting.clear();
                }
                if (B->doorbell_host) *B->doorbell_host = 0;   // null after a failed set-up
                // admit what fits; the rest goes back to the queue head
                while (!waiting.empty()) {
                    uint32_t kq = (uint32_t)waiting.front().seeds.size();
                    if (kq == 1) {                       // a single seed: the empty tree
                        steiner_result_t r{};
                        out(waiting.front().ticket, r);
                        waiting.pop_front();
                        continue;
                    }
                    if (!B->fits(kq) && B->inflight == 0) {
                        steiner_result_t r{};          // can never fit this budget
                        r.status = STEINER_EBUSY;
                        out(waiting.front().ticket, r);
                        waiting.pop_front();
                        continue;
                    }
                    int q = B->free_slot();
                    if (q < 0 || !B->fits(kq)) break;
                    ServeJob j = std::move(waiting.front());
                    waiting.pop_front();
                    int arc = B->stage(q, j.seeds, j.ticket);
                    if (arc) {
                        steiner_result_t r{};
                        r.status = arc;
                        out(j.ticket, r);
                    }
                }
                if (int rc2 = B->commit()) B->fail_slots(B->inflight, rc2, out);
                if (B->inflight) {
                    unsigned long long conv = 0, failed = 0;
                    int why = 0;
                    B->run(true, &conv, &failed, &why);
                    B->retire(conv & ~failed, out);
                    B->fail_slots(failed, why, out);
                }
            }
            std::lock_guard<std::mutex> lk(mu);
            for (auto it = waiting.rbegin(); it != waiting.rend(); ++it) queue.push_front(std::move(*it));
            for (auto &f : finished) done[f.first] = f.second;
        }
    }
};

}  // namespace stn

using namespace stn;

extern "C" {

int steiner_query_batch(steiner_graph_t G, const int32_t *const *seeds, const uint32_t *ks,
                        uint32_t q, steiner_result_t *outs) {
    if (!G || (q && (!seeds || !ks || !outs))) {
        api_set_error("null argument");
        return STEINER_EINVAL;
    }
    std::lock_guard<std::mutex> lk(api_mutex(G));
    cudaSetDevice(api_device(G));
    for (uint32_t i = 0; i < q; ++i) {
        outs[i].edges = nullptr;
        outs[i].n_edges = 0;
        outs[i].total = 0;
        outs[i].status = STEINER_OK;
    }
    BatchEngine *B = engine_of(G);
    int rc = B->init();
    if (rc) {
        for (uint32_t i = 0; i < q; ++i) outs[i].status = rc;
        return rc;
    }
    std::deque<std::pair<uint32_t, std::vector<int32_t>>> pending;
    for (uint32_t i = 0; i < q; ++i) {
        std::vector<int32_t> ss;
        int r = api_sorted_seeds(G, seeds[i], ks[i], ss);
        if (r) outs[i].status = r;
        else if (ss.size() > 1) pending.emplace_back(i, std::move(ss));   // k = 1: empty tree
    }
    auto out = [&](uint64_t tag, const steiner_result_t &r) { outs[tag] = r; };
    while (!pending.empty() || B->inflight) {
        while (!pending.empty()) {
            int slot = B->free_slot();
            if (slot < 0) break;
            auto job = std::move(pending.front());
            pending.pop_front();
            int r = B->stage(slot, job.second, job.first);
            if (r) outs[job.first].status = r;
        }
        if (int r = B->commit()) {
            B->fail_slots(B->inflight, r, out);
            continue;
        }
        if (!B->inflight) continue;
        unsigned long long conv = 0, failed = 0;
        int why = 0;
        // yield on convergence only while queries still wait for a slot
        B->run(!pending.empty(), &conv, &failed, &why);
        B->retire(conv & ~failed, out);
        B->fail_slots(failed, why, out);
    }
    int first = STEINER_OK;
    for (uint32_t i = 0; i < q; ++i)
        if (outs[i].status != STEINER_OK) {
            first = outs[i].status;
            break;
        }
    return first;
}

int steiner_serve_start(steiner_graph_t G, uint32_t slots, uint64_t budget_bytes) {
    if (!G) return STEINER_EINVAL;
    // the graph mutex makes the check-and-create atomic; the worker's first
    // pass waits on it until this call returns
    std::lock_guard<std::mutex> glk(api_mutex(G));
    ServeEngine *&S = api_serve(G);
    if (S) return STEINER_OK;
    {
        BatchEngine *B = engine_of(G);
        int rc = B->init();
        if (rc) return rc;
        // the budget covers the slots' label/pred columns and pair tables
        if (budget_bytes <= B->fixed) {
            api_set_error("serving budget smaller than the per-slot label state");
            return STEINER_ENOMEM;
        }
        B->budget = budget_bytes - B->fixed;
        int usable = (int)std::min<uint32_t>(slots ? slots : MQ_SLOTS, MQ_SLOTS);
        for (int q = usable; q < MQ_SLOTS; ++q) B->slots[q].busy = true;   // not offered
        B->free_slots = usable;
    }
    S = new ServeEngine();
    S->G = G;
    S->worker = std::thread([S] { S->run(); });
    return STEINER_OK;
}

int steiner_submit(steiner_graph_t G, const int32_t *seeds, uint32_t k, uint64_t *ticket) {
    if (!G || !ticket) return STEINER_EINVAL;
    ServeEngine *S = api_serve(G);
    if (!S) {
        api_set_error("serving not started");
        return STEINER_EINVAL;
    }
    std::vector<int32_t> ss;
    int rc = api_sorted_seeds(G, seeds, k, ss);
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->queue.size() >= S->max_queue) return STEINER_EBUSY;
    uint64_t t = S->next_ticket++;
    *ticket = t;
    S->live.insert(t);
    if (rc) {
        steiner_result_t r{};
        r.status = rc;
        S->done[t] = r;
        return STEINER_OK;
    }
    S->queue.push_back(ServeJob{t, std::move(ss), now_s()});
    BatchEngine *B = api_batch(G);
    if (B && B->doorbell_host && B->free_slots.load() > 0) *(volatile uint32_t *)B->doorbell_host = 1;
    S->cv.notify_one();
    return STEINER_OK;
}

int steiner_poll(steiner_graph_t G, uint64_t ticket, steiner_result_t *out) {
    if (!G || !out) return STEINER_EINVAL;
    ServeEngine *S = api_serve(G);
    if (!S) return STEINER_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    // a ticket that was never issued, or whose result was already returned,
    // is unknown: STEINER_EINVAL with *out untouched
    if (!S->live.count(ticket)) return STEINER_EINVAL;
    auto it = S->done.find(ticket);
    if (it == S->done.end()) return STEINER_PENDING;
    *out = it->second;
    S->done.erase(it);
    S->live.erase(ticket);
    return out->status;
}

int steiner_serve_stop(steiner_graph_t G) {
    if (!G) return STEINER_EINVAL;
    ServeEngine *&S = api_serve(G);
    if (!S) return STEINER_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (auto &kv : S->done) free(kv.second.edges);
    delete S;
    S = nullptr;
    // hand every slot back to the batch mode
    BatchEngine *B = api_batch(G);
    if (B) {
        std::lock_guard<std::mutex> glk(api_mutex(G));
        for (int q = 0; q < MQ_SLOTS; ++q)
            if (!((B->inflight >> q) & 1)) B->slots[q] = SlotInfo();
        B->budget = ~0ull;
        B->free_slots = MQ_SLOTS - __builtin_popcountll(B->inflight);
    }
    return STEINER_OK;
}

}  // extern "C"
