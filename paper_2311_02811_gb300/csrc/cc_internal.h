// Internal declarations shared by the translation units of libcontour.so.
#pragma once

#include <cuda_runtime.h>

#include "../../include/contour.h"

namespace cc {

cc_status set_error(cc_status s, const char* fmt, ...);
cc_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);
int device_sms();
int persistent_blocks(const void* fn, int threads, size_t smem);

// Graph accessors for the scheduler (features are computed on the graph's edges).
const void* graph_src(const cc_graph* g);
const void* graph_dst(const cc_graph* g);
int graph_id_bits(const cc_graph* g);
cc_status graph_nm(const cc_graph* g, long long* n, long long* m);

// CC_ORDER_AUTO: pick (order, mode, check interval) for a graph; the plain
// order-2 synchronous schedule with c = 1 when no scheduler weights are loaded.
cc_status resolve_schedule(cc_graph* g, int* order, int* mode, int* c);

}  // namespace cc
