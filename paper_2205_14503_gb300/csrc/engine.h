// Interfaces between the C ABI and the multi-query engines (batch and
// serving).  The engines reach the graph handle only through these hooks.
#pragma once
#include <cstdint>
#include <mutex>
#include <string>

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
uint32_t api_nbits(steiner_graph *G);
const Geometry &api_geometry(steiner_graph *G);
void api_set_error(const std::string &msg);
void destroy_batch(BatchEngine *b);

}  // namespace stn
