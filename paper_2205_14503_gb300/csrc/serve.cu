// Batch and serving entry points.
//
// steiner_query_batch runs its queries back to back on the graph's stream;
// the serving loop is a host worker thread that admits submitted queries in
// arrival order and runs each through the same device pipeline.
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>
#include <vector>

#include "engine.h"

namespace stn {

struct BatchEngine {};

void destroy_batch(BatchEngine *b) { delete b; }

struct ServeJob {
    uint64_t ticket;
    std::vector<int32_t> seeds;
};

struct ServeEngine {
    steiner_graph *G = nullptr;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<ServeJob> queue;
    std::unordered_map<uint64_t, steiner_result_t> done;
    uint64_t next_ticket = 1;
    uint32_t max_queue = 1u << 16;
    bool stop = false;

    void run() {
        cudaSetDevice(api_device(G));
        for (;;) {
            ServeJob job;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv.wait(lk, [&] { return stop || !queue.empty(); });
                if (stop && queue.empty()) return;
                job = std::move(queue.front());
                queue.pop_front();
            }
            steiner_result_t r{};
            {
                std::lock_guard<std::mutex> glk(api_mutex(G));
                api_query_locked(G, job.seeds.data(), (uint32_t)job.seeds.size(), &r);
            }
            std::lock_guard<std::mutex> lk(mu);
            done[job.ticket] = r;
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
    int first = STEINER_OK;
    for (uint32_t i = 0; i < q; ++i) {
        int rc = api_query_locked(G, seeds[i], ks[i], &outs[i]);
        if (rc != STEINER_OK && first == STEINER_OK) first = rc;
    }
    return first;
}

int steiner_serve_start(steiner_graph_t G, uint32_t slots, uint64_t budget_bytes) {
    (void)slots;
    (void)budget_bytes;
    if (!G) return STEINER_EINVAL;
    ServeEngine *&S = api_serve(G);
    if (S) return STEINER_OK;
    S = new ServeEngine();
    S->G = G;
    S->worker = std::thread([S] { S->run(); });
    return STEINER_OK;
}

int steiner_submit(steiner_graph_t G, const int32_t *seeds, uint32_t k, uint64_t *ticket) {
    if (!G || !ticket || (k && !seeds)) return STEINER_EINVAL;
    ServeEngine *S = api_serve(G);
    if (!S) {
        api_set_error("serving not started");
        return STEINER_EINVAL;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->queue.size() >= S->max_queue) return STEINER_EBUSY;
    ServeJob job{S->next_ticket++, std::vector<int32_t>(seeds, seeds + k)};
    *ticket = job.ticket;
    S->queue.push_back(std::move(job));
    S->cv.notify_one();
    return STEINER_OK;
}

int steiner_poll(steiner_graph_t G, uint64_t ticket, steiner_result_t *out) {
    if (!G || !out) return STEINER_EINVAL;
    ServeEngine *S = api_serve(G);
    if (!S) return STEINER_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->done.find(ticket);
    if (it == S->done.end()) return ticket < S->next_ticket ? STEINER_PENDING : STEINER_EINVAL;
    *out = it->second;
    S->done.erase(it);
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
    return STEINER_OK;
}

}  // extern "C"
