// Interfaces between the C ABI and the multi-query engines (batch and
// serving).  The engines reach the graph handle only through these hooks.
#pragma once
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/steiner.h"
#include "internal.h"

struct steiner_graph;

namespace stn {

struct BatchEngine;
struct ServeEngine;

int api_query_locked(steiner_graph *G, const int32_t *seeds, uint32_t k, steiner_result_t *out);
std::mutex &api_mutex(steiner_graph *G);
const DevGraph &api_graph(steiner_graph *G);
int api_device(steiner_graph *G);
BatchEngine *&api_batch(steiner_graph *G);
ServeEngine *&api_serve(steiner_graph *G);
uint32_t api_delta(steiner_graph *G);
// Builds the weight-partitioned rows for band width delta if needed.
void api_ensure_partition(steiner_graph *G, uint32_t delta);
uint32_t api_nbits(steiner_graph *G);
const Geometry &api_geometry(steiner_graph *G);
void api_set_error(const std::string &msg);
void destroy_batch(BatchEngine *b);
int64_t batch_counter(BatchEngine *B, const char *key);
int batch_set_param(steiner_graph *G, const char *key, int64_t value);
int api_run_tail(steiner_graph *G, uint64_t *pairtab, uint32_t *pred_base, uint32_t pred_stride,
                 uint32_t k, bool overflow, steiner_result_t *out);
int api_sorted_seeds(steiner_graph *G, const int32_t *seeds, uint32_t k, std::vector<int32_t> &out);
cudaStream_t api_stream(steiner_graph *G);
// Reserves `count` consecutive tree-walk tags of the graph's mark array
// (clearing it when the tags would run out); returns the first tag and the
// array, or a null array when the workspace cannot be set up.
uint32_t api_reserve_mark_tags(steiner_graph *G, uint32_t count, uint32_t **mark);

}  // namespace stn
