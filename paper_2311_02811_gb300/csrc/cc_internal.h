// Internal declarations shared by the translation units of libcontour.so.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <stdint.h>

#include "../../include/contour.h"

namespace cc {

// NVTX range for profilers (a no-op unless a tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

struct SchedCtx;  // scheduler buffers of a handle or plan (sched.cu)
void sched_ctx_free(SchedCtx* c);

cc_status set_error(cc_status s, const char* fmt, ...);
cc_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);
int device_sms();
// Stream-ordered allocation from the library's per-device memory pool.
cudaError_t dmalloc(void** ptr, size_t bytes, cudaStream_t s);
cudaError_t dfree(void* ptr, cudaStream_t s);
int persistent_blocks(const void* fn, int threads, size_t smem);

// Graph accessors for the scheduler (features are computed on the graph's edges).
const void* graph_src(const cc_graph* g);
const void* graph_dst(const cc_graph* g);
int graph_id_bits(const cc_graph* g);
int graph_layout(const cc_graph* g);            // CC_COO or a native CSR layout
const int64_t* graph_csr_off(const cc_graph* g);  // native CSR row offsets
int graph_hub_count(const cc_graph* g);           // hubs of a CC_REORDER_HUB edge list (0: none)
const int32_t* graph_hubs(const cc_graph* g);
// Hand the hub table (device array of k ids) to the handle, which frees it.
void graph_set_hubs(cc_graph* g, int32_t* hubs, int k);
cc_status graph_nm(const cc_graph* g, long long* n, long long* m);
cudaStream_t graph_stream(const cc_graph* g);
SchedCtx** graph_sched_slot(cc_graph* g);
// Replace the handle's edge arrays by device arrays it then owns (reorder.cu).
cc_status graph_replace_edges(cc_graph* g, void* src, void* dst);
// CC_REORDER_DEGREE: hand the id maps (n int32 each, owned by the handle from
// then on) and the shared-memory prefix length to the handle.
void graph_set_relabel(cc_graph* g, int32_t* perm, int32_t* inv, int k);
bool graph_relabeled(const cc_graph* g);

// CC_ORDER_AUTO: pick (order, mode, check interval) for a graph; the plain
// order-2 synchronous schedule with c = 1 when no scheduler weights are loaded.
// *deferred: the handle has no prediction for the loaded model yet; the
// caller solves with the returned default and then calls
// sched_defer_features, which enqueues the feature pass behind that solve.
cc_status resolve_schedule(cc_graph* g, int* order, int* mode, int* c, bool* deferred);
cc_status sched_defer_features(cc_graph* g, cudaStream_t s);

// Stable radix sort of cnt (key, value) pairs by the low end_bit bits of the
// key, between two buffer pairs (reorder.cu): the input in (k0, v0), the
// other pair as scratch; *in_second says which pair holds the result.  temp ==
// nullptr: only sets *temp_bytes.
cudaError_t sort_pairs_u32(void* temp, size_t* temp_bytes, uint32_t* k0, uint32_t* k1, uint32_t* v0, uint32_t* v1,
                           int64_t cnt, int end_bit, cudaStream_t s, bool* in_second);
int key_bits(int64_t n);

// Batched path (batch.cu) and its schedule resolution (sched.cu).
cc_status batch_solve(cc_batch_plan* b, int32_t max_sweeps, int32_t* labels_out, int32_t* sweeps_out,
                      double* solve_ms);
cc_status batch_resolve_schedule(cc_batch_plan* b, int mode, int c);
cc_status batch_autotune(cc_batch_plan* b, int force);
int32_t batch_graph_count(const cc_batch_plan* b);
const int64_t* batch_off_v(const cc_batch_plan* b);
const int64_t* batch_off_e(const cc_batch_plan* b);
const int32_t* batch_src(const cc_batch_plan* b);
const int32_t* batch_dst(const cc_batch_plan* b);
cudaStream_t batch_stream(const cc_batch_plan* b);
SchedCtx** batch_sched_slot(cc_batch_plan* b);
void batch_set_schedule(cc_batch_plan* b, const int32_t* h, const int32_t* sync, const int32_t* c);

}  // namespace cc
