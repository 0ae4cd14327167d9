// Host engine and C ABI of the single-graph Contour path (include/contour.h).
//
// cc_run enqueues, on the caller's stream:
//   ctl reset -> label init (Alg. 1 initialisation, or a validated snapshot)
//   -> one CUDA graph holding a conditional WHILE node whose body runs one
//      check block (c sweeps, plus L = L_u after each synchronous sweep) and
//      a one-thread check kernel that clears the flag and sets the loop
//      condition (Section III-B2 early convergence check)
//   -> compress -> labels / control block back to the caller.
// The loop never returns to the host between sweeps.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/contour.h"
#include "cc_internal.h"
#include "mm_kernels.cuh"
#include "csr_kernels.cuh"
#include "hub_kernels.cuh"
#include "compact_kernels.cuh"
#include "relabel_kernels.cuh"
#include "stream_kernels.cuh"

using cc::Ctl;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------

static thread_local std::string g_last_error;

namespace cc {

cc_status set_error(cc_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

cc_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
    cudaGetLastError();  // clear a sticky-free error so later calls are not poisoned
    return set_error(e == cudaErrorMemoryAllocation ? CC_ENOMEM : CC_ECUDA, "%s failed at %s:%d: %s",
                     what, file, line, cudaGetErrorString(e));
}

int device_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

// Persistent grid: blocks resident on every SM at once (occupancy-limited).
int persistent_blocks(const void* fn, int threads, size_t smem) {
    static std::mutex mu;
    static std::unordered_map<const void*, int> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(fn);
    if (it != cache.end()) return it->second;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess ||
        per_sm <= 0)
        per_sm = 1;
    const int blocks = per_sm * device_sms();
    cache[fn] = blocks;
    return blocks;
}

// Device memory of handles comes from one stream-ordered pool per device
// (cudaMallocFromPoolAsync / cudaFreeAsync) that keeps released memory for
// reuse, so repeated cc_init / cc_free cycles do not pay for cudaMalloc and
// cudaFree each time; cc_release_memory() returns it to the device.
namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pools[64] = {};
}  // namespace

cudaError_t pool_for_device(cudaMemPool_t* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p;
        e = cudaMemPoolCreate(&p, &props);
        if (e != cudaSuccess) return e;
        unsigned long long keep = ~0ull;
        e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return e;
        }
        g_pools[dev] = p;
    }
    *out = g_pools[dev];
    return cudaSuccess;
}

cudaError_t dmalloc(void** ptr, size_t bytes, cudaStream_t s) {
    cudaMemPool_t pool;
    cudaError_t e = pool_for_device(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(ptr, bytes > 0 ? bytes : 16, pool, s);
}

cudaError_t dfree(void* ptr, cudaStream_t s) {
    if (!ptr) return cudaSuccess;
    return cudaFreeAsync(ptr, s);
}

}  // namespace cc

extern "C" cc_status cc_release_memory(void) {
    for (int d = 0; d < 64; ++d) {
        cudaMemPool_t p = nullptr;
        {
            std::lock_guard<std::mutex> lock(cc::g_pool_mu);
            p = cc::g_pools[d];
        }
        if (!p) continue;
        cudaError_t e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaMemPoolTrimTo(p, 0);
        if (e != cudaSuccess) return cc::cuda_fail(e, "cc_release_memory", __FILE__, __LINE__);
    }
    return CC_OK;
}

using cc::cuda_fail;
using cc::set_error;

#define CC_CUDA(expr)                                                   \
    do {                                                                \
        cudaError_t e_ = (expr);                                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, #expr, __FILE__, __LINE__); \
    } while (0)

#define CC_LAUNCHED()                                                   \
    do {                                                                \
        cudaError_t e_ = cudaGetLastError();                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, "kernel launch", __FILE__, __LINE__); \
    } while (0)

// ---------------------------------------------------------------------------
// handle
// ---------------------------------------------------------------------------

struct LoopGraph {
    int order = 0, mode = 0, c = 0;
    void* L = nullptr;
    void* Lu = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

struct cc_graph {
    int64_t n = 0, m = 0;
    int id_bits = 32;
    int layout = CC_COO;  // CC_COO (also after CSR expansion), CC_CSR_NATIVE or CC_CSR_NATIVE_SYM
    void* src = nullptr;  // COO only
    void* dst = nullptr;  // COO: dst ids; native CSR: columns
    bool own_edges = false;
    int64_t* off = nullptr;   // native CSR: row offsets (n + 1)
    bool own_off = false;
    int32_t* seg = nullptr;   // native CSR: row of every 4th entry
    int32_t* hubs = nullptr;  // CC_REORDER_HUB: dst entry ~s names hubs[s]
    int hub_k = 0;            // hub table entries (CC_REORDER_DEGREE: new ids read from shared memory)
    int32_t* perm = nullptr;  // CC_REORDER_DEGREE: new id of every vertex
    int32_t* inv = nullptr;   //   and its inverse
    int32_t* tree_min = nullptr;  //   work arrays of the label mapping
    int32_t* Lx = nullptr;
    int launch = CC_LAUNCH_GRAPH;  // or CC_LAUNCH_HOST (cc_graph_set_launch)
    cc::CompactLists clists = {};  // CC_ASYNC_COMPACT: two edge lists + counters (allocated on first use)
    void* L = nullptr;   // working labels when the caller's output is on the host
    void* Lu = nullptr;  // update array of synchronous runs
    Ctl* ctl = nullptr;
    Ctl* ctl_h = nullptr;  // pinned mirror
    cudaStream_t stream = nullptr;  // caller's stream (cc_init / cc_graph_set_stream)
    cudaStream_t cap = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, evl0 = nullptr, evl1 = nullptr;
    std::vector<LoopGraph> loops;
    cc::SchedCtx* sched = nullptr;  // CC_ORDER_AUTO buffers
};

static size_t id_size(int id_bits) { return id_bits == 64 ? 8 : 4; }

static void free_loops(cc_graph* g) {
    for (auto& lg : g->loops) {
        if (lg.exec) cudaGraphExecDestroy(lg.exec);
        if (lg.graph) cudaGraphDestroy(lg.graph);
    }
    g->loops.clear();
}

static void destroy(cc_graph* g) {
    if (!g) return;
    free_loops(g);
    cc::sched_ctx_free(g->sched);
    if (g->own_edges) {
        cc::dfree(g->src, g->stream);
        cc::dfree(g->dst, g->stream);
    }
    if (g->own_off) cc::dfree(g->off, g->stream);
    cc::dfree(g->seg, g->stream);
    cc::dfree(g->hubs, g->stream);
    cc::dfree(g->perm, g->stream);
    cc::dfree(g->inv, g->stream);
    cc::dfree(g->tree_min, g->stream);
    cc::dfree(g->Lx, g->stream);
    for (int i = 0; i < 2; ++i) {
        cc::dfree(g->clists.src[i], g->stream);
        cc::dfree(g->clists.dst[i], g->stream);
    }
    cc::dfree(g->clists.cnt, g->stream);
    cc::dfree(g->L, g->stream);
    cc::dfree(g->Lu, g->stream);
    cc::dfree(g->ctl, g->stream);
    if (g->ctl_h) cudaFreeHost(g->ctl_h);
    if (g->cap) cudaStreamDestroy(g->cap);
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    if (g->evl0) cudaEventDestroy(g->evl0);
    if (g->evl1) cudaEventDestroy(g->evl1);
    delete g;
}

static const int kThreads = 256;

template <typename K>
static int grid_for(K kernel, int64_t work_items) {
    const int cap = cc::persistent_blocks(reinterpret_cast<const void*>(kernel), kThreads, 0);
    int64_t need = (work_items + kThreads - 1) / kThreads;
    if (need < 1) need = 1;
    return (int)(need < cap ? need : cap);
}

// ---------------------------------------------------------------------------
// sweep dispatch
// ---------------------------------------------------------------------------

template <int H, bool SYNC, typename IdT>
static cudaError_t launch_sweep_t(const cc_graph* g, IdT* L, IdT* Lu, int h, int32_t* flag,
                                  int first, cudaStream_t s, int gate = 0) {
    if constexpr (sizeof(IdT) == 4) {
        if (g->layout == CC_CSR_NATIVE || g->layout == CC_CSR_NATIVE_SYM) {
            auto kc = cc::csr_sweep_kernel<H, SYNC>;
            const int grid = grid_for(kc, (g->m + cc::kCsrGroup - 1) / cc::kCsrGroup + 1);
            kc<<<grid, kThreads, 0, s>>>(g->off, static_cast<const int32_t*>(g->dst), g->seg, g->m, L, Lu, h,
                                          flag, g->ctl, first, gate, g->layout == CC_CSR_NATIVE_SYM);
            return cudaGetLastError();
        }
    }
    if constexpr (sizeof(IdT) == 4) {
        if (g->perm) {
            auto kp = cc::mm_sweep_prefix_kernel<H, SYNC>;
            // synchronous sweeps hold two tables (labels and L_u minima) in the same space
            const int kt = SYNC ? (g->hub_k < cc::kHubMax / 2 ? g->hub_k : cc::kHubMax / 2) : g->hub_k;
            const size_t smem = (size_t)kt * (SYNC ? 2 : 1) * sizeof(int32_t);
            cudaError_t e = cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 cc::kHubMax * (int)sizeof(int32_t));
            if (e != cudaSuccess) return e;
            kp<<<cc::device_sms(), cc::kHubThreads, smem, s>>>(static_cast<const int32_t*>(g->src),
                                                                static_cast<const int32_t*>(g->dst), g->m, L, Lu,
                                                                h, flag, g->ctl, first, gate, kt);
            return cudaGetLastError();
        }
        if (g->hub_k > 0) {
            auto kh = cc::mm_sweep_hub_kernel<H, SYNC>;
            const size_t smem = (size_t)g->hub_k * sizeof(int32_t);
            // per device and cheap: set before every launch (or capture)
            cudaError_t e = cudaFuncSetAttribute(kh, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 cc::kHubMax * (int)sizeof(int32_t));
            if (e != cudaSuccess) return e;
            kh<<<cc::device_sms(), cc::kHubThreads, smem, s>>>(
                static_cast<const int32_t*>(g->src), static_cast<const int32_t*>(g->dst), g->m, L, Lu, h, flag,
                g->ctl, first, gate, g->hubs, g->hub_k);
            return cudaGetLastError();
        }
    }
    constexpr int G = (H == 1) ? 2 : 1;  // edge groups of 4 per thread per step
    auto k = cc::mm_sweep_kernel<H, SYNC, G, IdT>;
    const int grid = grid_for(k, g->m / (4 * G) + 1);
    k<<<grid, kThreads, 0, s>>>(static_cast<const IdT*>(g->src), static_cast<const IdT*>(g->dst),
                                 g->m, L, Lu, h, flag, g->ctl, first, gate);
    return cudaGetLastError();
}

template <bool SYNC, typename IdT>
static cudaError_t launch_sweep_m(const cc_graph* g, int order, IdT* L, IdT* Lu, int32_t* flag,
                                  int first, cudaStream_t s) {
    switch (order) {
        case 1: return launch_sweep_t<1, SYNC, IdT>(g, L, Lu, 1, flag, first, s);
        case 2: return launch_sweep_t<2, SYNC, IdT>(g, L, Lu, 2, flag, first, s);
        // order 4 runs on the run-time-order kernels: their chains advance
        // in lockstep and stop at roots, and they fit each layout's register
        // budget, where four unrolled order-4 chains per thread spill or
        // halve the resident warps (R-MAT 24, hub layout, asynchronous:
        // 4.03 -> 2.31 ms per solve; grid 4096²: 1.50 -> 1.28 ms)
        case 4: return launch_sweep_t<0, SYNC, IdT>(g, L, Lu, 4, flag, first, s);
        case CC_ORDER_FULL: return launch_sweep_t<0, SYNC, IdT>(g, L, Lu, cc::kFullChainHops, flag, first, s);
        default: return launch_sweep_t<0, SYNC, IdT>(g, L, Lu, order, flag, first, s);
    }
}

template <typename IdT>
static cudaError_t launch_copy(IdT* dst, const IdT* src, int64_t n, cudaStream_t s) {
    auto k = cc::copy_kernel<IdT>;
    const int per = 16 / (int)sizeof(IdT);
    k<<<grid_for(k, n / per + 1), kThreads, 0, s>>>(dst, src, n);
    return cudaGetLastError();
}

// One check block: c sweeps (the flag only from the last), then the check.
// A per-iteration order schedule (C-11mm, C-1m1m) has one sweep per block,
// run by whichever of its two gated kernels the control word selects.
// The end of a check block for host-polled runs: the bookkeeping of
// check_kernel without the graph's loop condition; the host reads ctl.
static __global__ void check_host_kernel(Ctl* ctl, int32_t block_sweeps, int sched) {
    if (threadIdx.x == 0) {
        const int32_t f = ctl->flag;
        ctl->flag = 0;
        ctl->sweeps += block_sweeps;
        if (sched == 1) ctl->sched_h = ctl->sweeps < 2 ? 1 : cc::kFullChainHops;
        if (sched == 2) ctl->sched_h = (ctl->sweeps % 2 == 0) ? 1 : cc::kFullChainHops;
        ctl->converged = (f == 0);
    }
}

// host_polled: end the block with check_host_kernel instead of the graph's
// loop-condition update.
template <typename IdT>
static cudaError_t enqueue_block(cc_graph* g, int order, int mode, int c, IdT* L, IdT* Lu,
                                 cudaGraphConditionalHandle loop, cudaStream_t s, bool host_polled = false) {
    if (order == CC_ORDER_11MM || order == CC_ORDER_1M1M) {
        const int first = mode == CC_SYNC ? 1 : 0;
        int32_t* flag = &g->ctl->flag;
        cudaError_t e = (mode == CC_SYNC)
            ? launch_sweep_t<1, true, IdT>(g, L, Lu, 1, flag, first, s, 1)
            : launch_sweep_t<1, false, IdT>(g, L, nullptr, 1, flag, first, s, 1);
        if (e != cudaSuccess) return e;
        e = (mode == CC_SYNC)
            ? launch_sweep_t<0, true, IdT>(g, L, Lu, cc::kFullChainHops, flag, 0, s, cc::kFullChainHops)
            : launch_sweep_t<0, false, IdT>(g, L, nullptr, cc::kFullChainHops, flag, 0, s, cc::kFullChainHops);
        if (e != cudaSuccess) return e;
        if (mode == CC_SYNC) {
            e = launch_copy<IdT>(L, Lu, g->n, s);
            if (e != cudaSuccess) return e;
        }
        if (host_polled) check_host_kernel<<<1, 32, 0, s>>>(g->ctl, 1, order == CC_ORDER_11MM ? 1 : 2);
        else cc::check_kernel<<<1, 32, 0, s>>>(g->ctl, 1, loop, order == CC_ORDER_11MM ? 1 : 2);
        return cudaGetLastError();
    }
    if (mode == CC_ASYNC_COMPACT) {
        // one sweep per iteration: the compacting kernel or, once a compacting
        // sweep was clean, the ordinary full-chain sweep over all edges
        if constexpr (sizeof(IdT) == 4) {
            int32_t* flag = &g->ctl->flag;
            auto k = cc::mm_sweep_compact_kernel;
            k<<<grid_for(k, g->m / 4 + 1), kThreads, 0, s>>>(static_cast<const int32_t*>(g->src),
                                                            static_cast<const int32_t*>(g->dst), g->m, g->clists,
                                                            (int32_t*)L, flag, g->ctl);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            e = launch_sweep_t<0, false, IdT>(g, L, nullptr, cc::kFullChainHops, flag, 0, s, cc::kFullChainHops);
            if (e != cudaSuccess) return e;
        } else {
            return cudaErrorInvalidValue;  // rejected by run_impl: int32 ids only
        }
        if (host_polled) cc::compact_check_host_kernel<<<1, 32, 0, s>>>(g->ctl);
        else cc::compact_check_kernel<<<1, 32, 0, s>>>(g->ctl, loop);
        return cudaGetLastError();
    }
    for (int j = 0; j < c; ++j) {
        int32_t* flag = (j == c - 1) ? &g->ctl->flag : nullptr;
        // synchronous runs start with the gather-free identity sweep (the
        // first iteration of Alg. 1, exactly); asynchronous runs gain more
        // from reading labels that other edges have already lowered
        const int first = (j == 0 && mode == CC_SYNC) ? 1 : 0;
        cudaError_t e = (mode == CC_SYNC) ? launch_sweep_m<true, IdT>(g, order, L, Lu, flag, first, s)
                                          : launch_sweep_m<false, IdT>(g, order, L, nullptr, flag, first, s);
        if (e != cudaSuccess) return e;
        if (mode == CC_SYNC) {
            e = launch_copy<IdT>(L, Lu, g->n, s);
            if (e != cudaSuccess) return e;
        }
    }
    if (host_polled) check_host_kernel<<<1, 32, 0, s>>>(g->ctl, c, 0);
    else cc::check_kernel<<<1, 32, 0, s>>>(g->ctl, c, loop);
    return cudaGetLastError();
}

static cc_status build_loop(cc_graph* g, int order, int mode, int c, void* L, void* Lu,
                            LoopGraph* out) {
    LoopGraph lg;
    lg.order = order;
    lg.mode = mode;
    lg.c = c;
    lg.L = L;
    lg.Lu = Lu;
    CC_CUDA(cudaGraphCreate(&lg.graph, 0));
    cudaGraphConditionalHandle loop;
    cudaError_t e = cudaGraphConditionalHandleCreate(&loop, lg.graph, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) {
        cudaGraphDestroy(lg.graph);
        return cuda_fail(e, "cudaGraphConditionalHandleCreate", __FILE__, __LINE__);
    }
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = loop;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, lg.graph, nullptr, nullptr, 0, &p);
    if (e != cudaSuccess) {
        cudaGraphDestroy(lg.graph);
        return cuda_fail(e, "cudaGraphAddNode(conditional)", __FILE__, __LINE__);
    }
    cudaGraph_t body = p.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(g->cap, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t ek = (g->id_bits == 64)
                             ? enqueue_block<int64_t>(g, order, mode, c, (int64_t*)L, (int64_t*)Lu, loop, g->cap)
                             : enqueue_block<int32_t>(g, order, mode, c, (int32_t*)L, (int32_t*)Lu, loop, g->cap);
        cudaGraph_t captured = nullptr;
        e = cudaStreamEndCapture(g->cap, &captured);
        if (ek != cudaSuccess) e = ek;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&lg.exec, lg.graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(lg.graph);
        return cuda_fail(e, "building the sweep loop graph", __FILE__, __LINE__);
    }
    *out = lg;
    return CC_OK;
}

static cc_status get_loop(cc_graph* g, int order, int mode, int c, void* L, void* Lu,
                          cudaGraphExec_t* exec) {
    for (auto& lg : g->loops)
        if (lg.order == order && lg.mode == mode && lg.c == c && lg.L == L && lg.Lu == Lu) {
            *exec = lg.exec;
            return CC_OK;
        }
    // keep a few: a loop graph bakes in the label buffer of the run
    if (g->loops.size() >= 8) {
        cudaGraphExecDestroy(g->loops.front().exec);
        cudaGraphDestroy(g->loops.front().graph);
        g->loops.erase(g->loops.begin());
    }
    LoopGraph lg;
    cc_status st = build_loop(g, order, mode, c, L, Lu, &lg);
    if (st != CC_OK) return st;
    g->loops.push_back(lg);
    *exec = lg.exec;
    return CC_OK;
}

// ---------------------------------------------------------------------------
// cc_init
// ---------------------------------------------------------------------------

// Native CSR (int32 ids): keep offsets and columns, validate both, and index
// the row of every 4th entry.
static cc_status init_csr_native(cc_graph* g, int layout, const void* a, const void* b, int64_t cnt,
                                 int on_device, cudaStream_t s) {
    const int64_t n = g->n;
    g->layout = layout;
    g->m = cnt;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (on_device && (reinterpret_cast<uintptr_t>(a) & 7) == 0) {
        g->off = static_cast<int64_t*>(const_cast<void*>(a));
    } else {
        CC_CUDA(cc::dmalloc(reinterpret_cast<void**>(&g->off), (size_t)(n + 1) * sizeof(int64_t), s));
        g->own_off = true;
        CC_CUDA(cudaMemcpyAsync(g->off, a, (size_t)(n + 1) * sizeof(int64_t), kind, s));
    }
    if (cnt > 0) {
        if (on_device && (reinterpret_cast<uintptr_t>(b) & 15) == 0) {
            g->dst = const_cast<void*>(b);
        } else {
            CC_CUDA(cc::dmalloc(&g->dst, (size_t)cnt * sizeof(int32_t), s));
            g->own_edges = true;
            CC_CUDA(cudaMemcpyAsync(g->dst, b, (size_t)cnt * sizeof(int32_t), kind, s));
        }
    }
    auto kv = cc::validate_offsets_kernel;
    kv<<<grid_for(kv, n + 1), kThreads, 0, s>>>(g->off, n, cnt, g->ctl);
    CC_LAUNCHED();
    CC_CUDA(cudaMemcpyAsync(g->ctl_h, g->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CC_CUDA(cudaStreamSynchronize(s));
    if (g->ctl_h->bad_count)
        return set_error(CC_EINVAL, "CSR offsets are not non-decreasing from 0 to nnz=%lld (first bad index %llu)",
                         (long long)cnt, g->ctl_h->first_bad);
    if (cnt > 0) {
        const int32_t* cols = static_cast<const int32_t*>(g->dst);
        auto ki = cc::validate_ids_kernel<int32_t>;
        ki<<<grid_for(ki, cnt / 4 + 1), kThreads, 0, s>>>(cols, cols, cnt, n, g->ctl);
        CC_LAUNCHED();
        const int64_t groups = (cnt + cc::kCsrGroup - 1) / cc::kCsrGroup;
        CC_CUDA(cc::dmalloc(reinterpret_cast<void**>(&g->seg), (size_t)groups * sizeof(int32_t), s));
        auto ks = cc::csr_seg_rows_kernel;
        ks<<<grid_for(ks, groups), kThreads, 0, s>>>(g->off, n, cnt, g->seg);
        CC_LAUNCHED();
    }
    CC_CUDA(cudaMemcpyAsync(g->ctl_h, g->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CC_CUDA(cudaStreamSynchronize(s));
    if (g->ctl_h->bad_count)
        return set_error(CC_EIDRANGE, "%llu column ids outside [0, %lld) (first at entry %llu)",
                         g->ctl_h->bad_count / 2, (long long)n, g->ctl_h->first_bad);
    return CC_OK;
}

template <typename IdT>
static cc_status init_edges(cc_graph* g, int layout, const void* a, const void* b, int64_t cnt,
                            int on_device, cudaStream_t s) {
    const size_t B = sizeof(IdT);
    const int64_t n = g->n;
    g->m = cnt;
    const bool aligned = on_device && ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15) == 0;
    if (layout == CC_COO && aligned) {
        g->src = const_cast<void*>(a);
        g->dst = const_cast<void*>(b);
        g->own_edges = false;
    } else {
        g->own_edges = true;
        const size_t bytes = (size_t)(cnt > 0 ? cnt : 1) * B;
        CC_CUDA(cc::dmalloc(&g->src, bytes, s));
        CC_CUDA(cc::dmalloc(&g->dst, bytes, s));
        const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        if (layout == CC_COO) {
            if (cnt) {
                CC_CUDA(cudaMemcpyAsync(g->src, a, cnt * B, kind, s));
                CC_CUDA(cudaMemcpyAsync(g->dst, b, cnt * B, kind, s));
            }
        } else {
            // CSR: offsets (int64, n+1) and columns; rows are expanded on the device
            int64_t* off = nullptr;
            CC_CUDA(cc::dmalloc(reinterpret_cast<void**>(&off), (size_t)(n + 1) * sizeof(int64_t), s));
            cudaError_t e = cudaMemcpyAsync(off, a, (size_t)(n + 1) * sizeof(int64_t), kind, s);
            if (e == cudaSuccess && cnt) e = cudaMemcpyAsync(g->dst, b, cnt * B, kind, s);
            if (e == cudaSuccess) {
                auto kv = cc::validate_offsets_kernel;
                kv<<<grid_for(kv, n + 1), kThreads, 0, s>>>(off, n, cnt, g->ctl);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) {
                CC_CUDA(cudaMemcpyAsync(g->ctl_h, g->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
                e = cudaStreamSynchronize(s);
            }
            if (e == cudaSuccess && g->ctl_h->bad_count) {
                cc::dfree(off, s);
                return set_error(CC_EINVAL, "CSR offsets are not non-decreasing from 0 to nnz=%lld (first bad index %llu)",
                                 (long long)cnt, g->ctl_h->first_bad);
            }
            if (e == cudaSuccess && cnt) {
                auto kr = cc::csr_rows_kernel<IdT>;
                kr<<<grid_for(kr, cnt), kThreads, 0, s>>>(off, n, cnt, static_cast<IdT*>(g->src));
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            cc::dfree(off, s);
            if (e != cudaSuccess) return cuda_fail(e, "CSR expansion", __FILE__, __LINE__);
        }
    }
    // every endpoint must lie in [0, n)
    if (cnt) {
        auto kv = cc::validate_ids_kernel<IdT>;
        kv<<<grid_for(kv, cnt / 4 + 1), kThreads, 0, s>>>(static_cast<const IdT*>(g->src),
                                                            static_cast<const IdT*>(g->dst), cnt, n, g->ctl);
        CC_LAUNCHED();
    }
    CC_CUDA(cudaMemcpyAsync(g->ctl_h, g->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CC_CUDA(cudaStreamSynchronize(s));
    if (g->ctl_h->bad_count)
        return set_error(CC_EIDRANGE, "%llu edge endpoints outside [0, %lld) (first at edge %llu)",
                         g->ctl_h->bad_count, (long long)n, g->ctl_h->first_bad);
    return CC_OK;
}

// A handle without edges: control block, events, capture stream.
static cc_status new_handle(int64_t n, int id_bits, cudaStream_t s, const char* who, cc_graph** out) {
    cc_graph* g = new (std::nothrow) cc_graph();
    if (!g) return set_error(CC_ENOMEM, "%s: host allocation failed", who);
    g->n = n;
    g->id_bits = id_bits;
    g->stream = s;
    cudaError_t e = cc::dmalloc(reinterpret_cast<void**>(&g->ctl), sizeof(Ctl), s);
    if (e == cudaSuccess) e = cudaMallocHost(&g->ctl_h, sizeof(Ctl));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&g->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&g->ev1);
    if (e == cudaSuccess) e = cudaEventCreate(&g->evl0);
    if (e == cudaSuccess) e = cudaEventCreate(&g->evl1);
    if (e == cudaSuccess) {
        cc::ctl_reset_kernel<<<1, 32, 0, s>>>(g->ctl, 1, 0);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        destroy(g);
        return cuda_fail(e, who, __FILE__, __LINE__);
    }
    *out = g;
    return CC_OK;
}

extern "C" cc_status cc_init(cc_graph** out, int64_t n, int id_bits, int layout, const void* a,
                             const void* b, int64_t cnt, int on_device, void* cuda_stream) {
    cc::NvtxRange range("cc_init");
    g_last_error.clear();
    if (!out) return set_error(CC_EINVAL, "cc_init: g is NULL");
    *out = nullptr;
    if (n < 0 || cnt < 0) return set_error(CC_EINVAL, "cc_init: negative n or m");
    if (id_bits != CC_ID32 && id_bits != CC_ID64) return set_error(CC_EINVAL, "cc_init: id_bits must be 32 or 64");
    if (id_bits == CC_ID32 && n > 0x7fffffffLL) return set_error(CC_EINVAL, "cc_init: n >= 2^31 needs CC_ID64");
    if (layout != CC_COO && layout != CC_CSR && layout != CC_CSR_NATIVE && layout != CC_CSR_NATIVE_SYM)
        return set_error(CC_EINVAL, "cc_init: bad layout");
    const bool native = layout == CC_CSR_NATIVE || layout == CC_CSR_NATIVE_SYM;
    if (layout != CC_COO && !a) return set_error(CC_EINVAL, "cc_init: CSR offsets are NULL");
    if (native && id_bits != CC_ID32) return set_error(CC_EINVAL, "cc_init: the native CSR layouts take int32 ids");
    if (cnt > 0 && (!a || !b)) return set_error(CC_EINVAL, "cc_init: edge arrays are NULL");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

    cc_graph* g = nullptr;
    cc_status st = new_handle(n, id_bits, s, "cc_init", &g);
    if (st != CC_OK) return st;
    auto fail = [&](cc_status x) {
        destroy(g);
        return x;
    };
    st = native ? init_csr_native(g, layout, a, b, cnt, on_device, s)
         : (id_bits == 64) ? init_edges<int64_t>(g, layout, a, b, cnt, on_device, s)
                           : init_edges<int32_t>(g, layout, a, b, cnt, on_device, s);
    if (st != CC_OK) return fail(st);
    *out = g;
    return CC_OK;
}

// ---------------------------------------------------------------------------
// cc_run
// ---------------------------------------------------------------------------

template <typename IdT>
static cudaError_t enqueue_init(cc_graph* g, IdT* L, IdT* Lu, const void* init, cudaStream_t s) {
    if (init) {
        if ((void*)L != init) {
            cudaError_t e = cudaMemcpyAsync(L, init, g->n * sizeof(IdT), cudaMemcpyDefault, s);
            if (e != cudaSuccess) return e;
        }
        auto kv = cc::validate_snapshot_kernel<IdT>;
        kv<<<grid_for(kv, g->n), kThreads, 0, s>>>(L, g->n, g->ctl);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (Lu) return launch_copy<IdT>(Lu, L, g->n, s);
        return cudaSuccess;
    }
    auto k = cc::iota_kernel<IdT>;
    k<<<grid_for(k, g->n), kThreads, 0, s>>>(L, Lu, g->n);
    return cudaGetLastError();
}

// a[i] = v for i < n
static __global__ void fill_i32_kernel(int32_t* a, int64_t n, int32_t v) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) a[i] = v;
}

// Label mapping of a renumbered handle (relabel_kernels.cuh): every tree of
// src gets the smallest key[] of its members, and out[x] = that minimum for
// the tree of map[x].  Export: src = the new-id labels, key = inv, map = perm;
// stars_if_converged: after a converged loop and its compress the trees are
// stars (read from the control block on the device).  Import: src = a
// snapshot in the caller's ids, key = perm, map = inv, chains walked.
static cudaError_t enqueue_map(cc_graph* g, const int32_t* src, const int32_t* key, const int32_t* map,
                               int32_t* out, cudaStream_t s, bool stars_if_converged) {
    const Ctl* ctl = stars_if_converged ? g->ctl : nullptr;
    auto kf = fill_i32_kernel;
    kf<<<grid_for(kf, g->n), kThreads, 0, s>>>(g->tree_min, g->n, 0x7fffffff);  // above every id
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    auto kt = cc::tree_min_kernel;
    kt<<<grid_for(kt, g->n / 64 + 1), kThreads, 0, s>>>(src, key, g->n, g->tree_min, ctl, &g->ctl->bad_count);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    auto km = cc::map_labels_kernel;
    km<<<grid_for(km, g->n), kThreads, 0, s>>>(src, map, g->tree_min, g->n, out, ctl, &g->ctl->bad_count);
    return cudaGetLastError();
}

template <typename IdT>
static cudaError_t enqueue_compress(cc_graph* g, IdT* L, cudaStream_t s) {
    auto k = cc::compress_kernel<IdT>;
    k<<<grid_for(k, g->n), kThreads, 0, s>>>(L, g->n, g->ctl);
    return cudaGetLastError();
}

static cc_status run_impl(cc_graph* g, int order, int mode, int c, int32_t max_sweeps,
                          const void* init_labels, void* labels_out, int out_on_device,
                          cc_stats* stats, cudaStream_t s);

extern "C" cc_status cc_run(cc_graph* g, int order, int mode, int c, int32_t max_sweeps,
                            const void* init_labels, void* labels_out, int out_on_device,
                            cc_stats* stats) {
    return run_impl(g, order, mode, c, max_sweeps, init_labels, labels_out, out_on_device, stats,
                       g ? g->stream : nullptr);
}

extern "C" cc_status cc_graph_set_stream(cc_graph* g, void* cuda_stream) {
    if (!g) return set_error(CC_EINVAL, "cc_graph_set_stream: g is NULL");
    g->stream = static_cast<cudaStream_t>(cuda_stream);
    return CC_OK;
}

static cc_status run_impl(cc_graph* g, int order, int mode, int c, int32_t max_sweeps,
                          const void* init_labels, void* labels_out, int out_on_device,
                          cc_stats* stats, cudaStream_t s) {
    cc::NvtxRange range("cc_run");
    g_last_error.clear();
    if (!g) return set_error(CC_EINVAL, "cc_run: g is NULL");
    if (g->n > 0 && !labels_out) return set_error(CC_EINVAL, "cc_run: labels_out is NULL");
    bool defer_features = false;
    if (order == CC_ORDER_AUTO) {
        cc_status st = cc::resolve_schedule(g, &order, &mode, &c, &defer_features);
        if (st != CC_OK) return st;
    }
    const bool schedule = order == CC_ORDER_11MM || order == CC_ORDER_1M1M;
    if (schedule || mode == CC_ASYNC_COMPACT) c = 1;
    if ((order < 0 || order > CC_MAX_ORDER) && !schedule)
        return set_error(CC_EINVAL, "cc_run: order must be 1..%d, CC_ORDER_FULL, CC_ORDER_AUTO, CC_ORDER_11MM or CC_ORDER_1M1M", CC_MAX_ORDER);
    if (mode != CC_SYNC && mode != CC_ASYNC && mode != CC_ASYNC_COMPACT)
        return set_error(CC_EINVAL, "cc_run: mode must be CC_SYNC, CC_ASYNC or CC_ASYNC_COMPACT");
    if (mode == CC_ASYNC_COMPACT) {
        if (order != CC_ORDER_FULL)
            return set_error(CC_EINVAL, "cc_run: CC_ASYNC_COMPACT needs CC_ORDER_FULL (a finite order can split trees)");
        if (g->id_bits != 32 || g->layout != CC_COO || g->hub_k > 0 || g->perm)
            return set_error(CC_EINVAL, "cc_run: CC_ASYNC_COMPACT takes int32 edge lists (no native CSR, no hub or "
                                        "renumbered layout)");
    }
    if (c < 1 || c > 64) return set_error(CC_EINVAL, "cc_run: check_interval must be 1..64");
    if (max_sweeps < 1) return set_error(CC_EINVAL, "cc_run: max_sweeps must be >= 1");
    const size_t B = id_size(g->id_bits);
    if (stats) {
        std::memset(stats, 0, sizeof *stats);
        stats->order = order;
        stats->mode = mode;
        stats->check_interval = c;
    }
    if (g->n == 0) return CC_OK;

    void* L = labels_out;
    const bool relabeled = g->perm != nullptr;  // sweeps work on the renumbered ids
    if (relabeled || !out_on_device || (reinterpret_cast<uintptr_t>(labels_out) & 15)) {
        if (!g->L) CC_CUDA(cc::dmalloc(&g->L, g->n * B, s));
        L = g->L;
    }
    if (relabeled) {
        if (!g->tree_min) CC_CUDA(cc::dmalloc(reinterpret_cast<void**>(&g->tree_min), g->n * sizeof(int32_t), s));
        if (!g->Lx) CC_CUDA(cc::dmalloc(reinterpret_cast<void**>(&g->Lx), g->n * sizeof(int32_t), s));
    }
    void* Lu = nullptr;
    if (mode == CC_SYNC) {
        if (!g->Lu) CC_CUDA(cc::dmalloc(&g->Lu, g->n * B, s));
        Lu = g->Lu;
    }
    const bool compact = mode == CC_ASYNC_COMPACT;
    if (compact && !g->clists.cnt) {
        // two edge lists of the handle's size (a sweep keeps at most what it
        // reads), then the counters; allocated before any loop graph captures them
        const size_t bytes = (size_t)(g->m > 0 ? g->m : 1) * sizeof(int32_t);
        for (int i = 0; i < 2; ++i) {
            CC_CUDA(cc::dmalloc(reinterpret_cast<void**>(&g->clists.src[i]), bytes, s));
            CC_CUDA(cc::dmalloc(reinterpret_cast<void**>(&g->clists.dst[i]), bytes, s));
        }
        CC_CUDA(cc::dmalloc(reinterpret_cast<void**>(&g->clists.cnt), 5 * sizeof(unsigned long long), s));
    }
    cudaGraphExec_t loop = nullptr;
    const bool host_polled = g->launch == CC_LAUNCH_HOST;
    if (!host_polled) {
        cc_status st = get_loop(g, order, mode, c, L, Lu, &loop);
        if (st != CC_OK) return st;
    }

    CC_CUDA(cudaEventRecord(g->ev0, s));
    cc::ctl_reset_kernel<<<1, 32, 0, s>>>(g->ctl, max_sweeps, init_labels ? 0 : 1,
                                          (schedule || mode == CC_ASYNC_COMPACT) ? 1 : 0);
    CC_LAUNCHED();
    if (relabeled && init_labels) {
        // a snapshot in the caller's ids: validated here, mapped below
        CC_CUDA(cudaMemcpyAsync(g->Lx, init_labels, g->n * sizeof(int32_t), cudaMemcpyDefault, s));
        auto kv = cc::validate_snapshot_kernel<int32_t>;
        kv<<<grid_for(kv, g->n), kThreads, 0, s>>>(g->Lx, g->n, g->ctl);
        CC_LAUNCHED();
    } else {
        CC_CUDA(g->id_bits == 64 ? enqueue_init<int64_t>(g, (int64_t*)L, (int64_t*)Lu, init_labels, s)
                                 : enqueue_init<int32_t>(g, (int32_t*)L, (int32_t*)Lu, init_labels, s));
    }
    if (init_labels) {
        // a bad snapshot could point outside [0, n): check before any gather
        CC_CUDA(cudaMemcpyAsync(g->ctl_h, g->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
        CC_CUDA(cudaStreamSynchronize(s));
        if (g->ctl_h->bad_count)
            return set_error(CC_EINVAL, "cc_run: init_labels violates 0 <= L[x] <= x at %llu entries (first %llu)",
                             g->ctl_h->bad_count, g->ctl_h->first_bad);
    }
    if (relabeled && init_labels) {
        // each tree of the snapshot gets its smallest new id
        CC_CUDA(enqueue_map(g, g->Lx, g->perm, g->inv, (int32_t*)L, s, false));
        if (Lu) CC_CUDA(launch_copy<int32_t>((int32_t*)Lu, (const int32_t*)L, g->n, s));
    }
    if (compact) CC_CUDA(cudaMemsetAsync(g->clists.cnt, 0, 5 * sizeof(unsigned long long), s));
    CC_CUDA(cudaEventRecord(g->evl0, s));
    if (host_polled) {
        // one check block at a time; the host reads the control block after each
        while (true) {
            CC_CUDA(g->id_bits == 64
                        ? enqueue_block<int64_t>(g, order, mode, c, (int64_t*)L, (int64_t*)Lu, 0, s, true)
                        : enqueue_block<int32_t>(g, order, mode, c, (int32_t*)L, (int32_t*)Lu, 0, s, true));
            CC_CUDA(cudaMemcpyAsync(g->ctl_h, g->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
            CC_CUDA(cudaStreamSynchronize(s));
            if (g->ctl_h->converged || g->ctl_h->sweeps >= max_sweeps) break;
        }
    } else {
        CC_CUDA(cudaGraphLaunch(loop, s));
    }
    CC_CUDA(cudaEventRecord(g->evl1, s));
    CC_CUDA(g->id_bits == 64 ? enqueue_compress<int64_t>(g, (int64_t*)L, s)
                             : enqueue_compress<int32_t>(g, (int32_t*)L, s));
    void* result = L;
    if (relabeled) {
        // back to the caller's ids: each tree labelled by its smallest member
        const bool direct = out_on_device && (reinterpret_cast<uintptr_t>(labels_out) & 3) == 0;
        result = direct ? labels_out : g->Lx;
        CC_CUDA(enqueue_map(g, (const int32_t*)L, g->inv, g->perm, (int32_t*)result, s, true));
    }
    CC_CUDA(cudaEventRecord(g->ev1, s));
    if (result != labels_out)
        CC_CUDA(cudaMemcpyAsync(labels_out, result, g->n * B, cudaMemcpyDefault, s));
    CC_CUDA(cudaMemcpyAsync(g->ctl_h, g->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    if (defer_features) {
        // the first CC_ORDER_AUTO call: the scheduler's feature pass goes
        // behind this solve, on the handle's own stream
        cc_status st = cc::sched_defer_features(g, s);
        if (st != CC_OK) return st;
    }
    unsigned long long cwords[2] = {0, 0};  // compacting runs: edges read and sweeps of the compacting phase
    if (compact) CC_CUDA(cudaMemcpyAsync(cwords, g->clists.cnt + 3, sizeof cwords, cudaMemcpyDeviceToHost, s));
    CC_CUDA(cudaStreamSynchronize(s));

    const Ctl& h = *g->ctl_h;
    if (stats) {
        float ms = 0.f, lms = 0.f;
        cudaEventElapsedTime(&ms, g->ev0, g->ev1);
        cudaEventElapsedTime(&lms, g->evl0, g->evl1);
        stats->sweeps = h.sweeps;
        stats->solve_ms = ms;
        stats->loop_ms = lms;
        stats->edges_per_s = ms > 0 ? (double)g->m / (ms * 1e-3) : 0.0;
        // COO: both id arrays and every label once; native CSR: columns,
        // offsets and every label once
        double per = (g->layout == CC_CSR_NATIVE || g->layout == CC_CSR_NATIVE_SYM)
                         ? B * (double)g->m + 8.0 * (double)(g->n + 1) + B * (double)g->n
                         : 2.0 * B * (double)g->m + B * (double)g->n;
        if (mode == CC_SYNC) per += 3.0 * B * (double)g->n;
        // compacting runs: the compacting sweeps' edges (counted on the device)
        // plus one full edge list for each ordinary sweep that followed
        const double ordinary = (double)h.sweeps - (double)cwords[1];
        stats->alg_bytes = compact ? 2.0 * B * ((double)cwords[0] + ordinary * (double)g->m) + B * (double)g->n * h.sweeps
                                   : per * h.sweeps;
    }
    if (relabeled && h.bad_count)
        return set_error(CC_ECUDA, "cc_run: label chain longer than %d hops while mapping ids", cc::kMapChaseCap);
    if (!h.converged)
        return set_error(CC_ENOTCONVERGED, "cc_run: not converged after %d sweeps", h.sweeps);
    if (h.compress_changes)
        return set_error(CC_ECUDA, "cc_run: converged state was not a set of stars (%llu labels moved)",
                         h.compress_changes);
    return CC_OK;
}

// ---------------------------------------------------------------------------
// cc_solve_host: one solve of a host edge list, the upload overlapped with sweeps
// ---------------------------------------------------------------------------

constexpr int64_t kStreamChunk = 1ll << 24;  // edges per chunk (64 MB of each id array)
constexpr int64_t kStreamTail = 1ll << 21;   // the smallest chunk of the geometric tail

// Chunks of the streamed upload: kStreamChunk edges each, then a tail that
// halves down to kStreamTail edges, so that little work is left to do after
// the last copy lands.  Every chunk but the last is a multiple of 4 edges
// (16-byte aligned starts).
static std::vector<std::pair<int64_t, int64_t>> stream_chunks(int64_t m) {
    std::vector<std::pair<int64_t, int64_t>> c;
    int64_t off = 0;
    while (off < m) {
        const int64_t rem = m - off;
        int64_t len = rem;
        if (rem > 2 * kStreamChunk) len = kStreamChunk;
        else if (rem > kStreamTail) len = std::max<int64_t>(kStreamTail, ((rem + 1) / 2 + 3) & ~int64_t(3));
        len = std::min(len, rem);
        c.emplace_back(off, len);
        off += len;
    }
    return c;
}

template <int H>
static cudaError_t launch_chunk(const int32_t* src, const int32_t* dst, int64_t cnt, int32_t* L, int h,
                                cudaStream_t s) {
    auto k = cc::chunk_sweep_kernel<H>;
    k<<<grid_for(k, cnt / 4 + 1), kThreads, 0, s>>>(src, dst, cnt, L, h);
    return cudaGetLastError();
}

extern "C" cc_status cc_solve_host(int64_t n, const int32_t* src, const int32_t* dst, int64_t m, int order,
                                   int mode, int c, int32_t max_sweeps, void* labels_out, int out_on_device,
                                   cc_stats* stats, void* cuda_stream) {
    cc::NvtxRange range("cc_solve_host");
    g_last_error.clear();
    if (n < 0 || m < 0) return set_error(CC_EINVAL, "cc_solve_host: negative n or m");
    if (n > 0x7fffffffLL) return set_error(CC_EINVAL, "cc_solve_host: int32 ids (n < 2^31)");
    if (m > 0 && (!src || !dst)) return set_error(CC_EINVAL, "cc_solve_host: edge arrays are NULL");
    if (n > 0 && !labels_out) return set_error(CC_EINVAL, "cc_solve_host: labels_out is NULL");
    if (mode != CC_SYNC && mode != CC_ASYNC) return set_error(CC_EINVAL, "cc_solve_host: mode must be CC_SYNC or CC_ASYNC");
    if (order < 0 || order > CC_MAX_ORDER)
        return set_error(CC_EINVAL, "cc_solve_host: order must be 1..%d or CC_ORDER_FULL", CC_MAX_ORDER);
    if (c < 1 || c > 64) return set_error(CC_EINVAL, "cc_solve_host: check_interval must be 1..64");
    for (const void* p : {static_cast<const void*>(src), static_cast<const void*>(dst)}) {
        if (m == 0) break;
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
            cudaGetLastError();
            continue;  // not known to CUDA: pageable host memory
        }
        if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)
            return set_error(CC_EINVAL, "cc_solve_host: src and dst must be host memory (device edges: cc_init + cc_run)");
    }
    const bool async = mode == CC_ASYNC;
    // the streamed pass counts as the first sweep of an asynchronous solve
    if (max_sweeps < (async ? 2 : 1))
        return set_error(CC_EINVAL, "cc_solve_host: max_sweeps must be >= %d", async ? 2 : 1);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cc_graph* g = nullptr;
    cc_status st = new_handle(n, CC_ID32, s, "cc_solve_host", &g);
    if (st != CC_OK) return st;
    cudaStream_t cs = nullptr;  // copy stream
    std::vector<cudaEvent_t> evs;
    cudaEvent_t ev_start = nullptr;
    int32_t* stg_s[2] = {nullptr, nullptr};  // staging pairs of the copies
    int32_t* stg_d[2] = {nullptr, nullptr};
    void* sort_tmp = nullptr;
    auto done = [&](cc_status x) {
        if (cs) cudaStreamSynchronize(cs);
        for (int i = 0; i < 2; ++i) {
            cc::dfree(stg_s[i], s);
            cc::dfree(stg_d[i], s);
        }
        cc::dfree(sort_tmp, s);
        for (cudaEvent_t e : evs) cudaEventDestroy(e);
        if (ev_start) cudaEventDestroy(ev_start);
        if (cs) cudaStreamDestroy(cs);
        destroy(g);
        return x;
    };
#define SH_CUDA(expr)                                                              \
    do {                                                                           \
        cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess) return done(cuda_fail(e_, #expr, __FILE__, __LINE__)); \
    } while (0)
    g->m = m;
    g->own_edges = true;
    const auto chunks = stream_chunks(m);
    const int64_t K = (int64_t)chunks.size();
    SH_CUDA(cudaEventCreate(&ev_start));
    SH_CUDA(cudaEventRecord(ev_start, s));
    SH_CUDA(cc::dmalloc(&g->src, (size_t)(m > 0 ? m : 1) * sizeof(int32_t), s));
    SH_CUDA(cc::dmalloc(&g->dst, (size_t)(m > 0 ? m : 1) * sizeof(int32_t), s));
    // the labels the streamed sweeps lower are the ones the loop starts from
    // (the caller's output when it is an aligned device buffer, as in cc_run).
    // Synchronous solves with c = 1 stream Alg. 1's first iteration, which
    // reads no label: its L_u, built in place from the identity, is the state
    // the loop continues from.
    const bool stream_ident = !async && c == 1 && max_sweeps > 1 && n > 0 && m > 0;
    int32_t* L = nullptr;
    if ((async || stream_ident) && n > 0) {
        if (out_on_device && (reinterpret_cast<uintptr_t>(labels_out) & 15) == 0) {
            L = static_cast<int32_t*>(labels_out);
        } else {
            SH_CUDA(cc::dmalloc(&g->L, (size_t)n * sizeof(int32_t), s));
            L = static_cast<int32_t*>(g->L);
        }
        auto ki = cc::iota_kernel<int32_t>;
        ki<<<grid_for(ki, n), kThreads, 0, s>>>(L, nullptr, n);
        SH_CUDA(cudaGetLastError());
    }
    if (K > 0) {
        // Per chunk: the chunk is screened and oriented as soon as its copy
        // has landed and -- asynchronous solves -- swept once while later
        // chunks are in flight.  On graphs of average degree 8 or more the
        // copy lands in one of two staging pairs and is sorted from there
        // into its place in the edge arrays (the staging pair is then free
        // for the chunk two ahead): grouped by one endpoint, a thread's edges
        // share it and the loop's sweeps gather fewer scattered labels
        // (R-MAT 24: 15.5 -> 13.8 ms per call).  On sparser graphs the sort
        // costs more than it saves (grid 4096²: 3.26 vs 3.50 ms) and the
        // copies land in place.  (Sweeping the one to three chunks before
        // each landed one again as well left the loop's sweep count unchanged
        // and delayed the last chunk: R-MAT 24 14.1-16.1 ms vs 13.8 ms.)
        const bool sorted = m >= 4 * n;
        SH_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        evs.resize(2 * (size_t)K + 1, nullptr);
        for (auto& e : evs) SH_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        cudaEvent_t* landed = evs.data();
        cudaEvent_t* freed = evs.data() + K;
        const int64_t E = std::min<int64_t>(kStreamChunk, m);
        const int bits = cc::key_bits(n > 0 ? n : 1);
        int32_t* ds = static_cast<int32_t*>(g->src);
        int32_t* dd = static_cast<int32_t*>(g->dst);
        size_t tmp_bytes = 0;
        if (sorted) {
            for (int i = 0; i < 2; ++i) {
                SH_CUDA(cc::dmalloc(reinterpret_cast<void**>(&stg_s[i]), (size_t)E * sizeof(int32_t), s));
                SH_CUDA(cc::dmalloc(reinterpret_cast<void**>(&stg_d[i]), (size_t)E * sizeof(int32_t), s));
            }
            SH_CUDA(cc::sort_pairs_u32(nullptr, &tmp_bytes, (uint32_t*)stg_s[0], (uint32_t*)ds, (uint32_t*)stg_d[0],
                                       (uint32_t*)dd, E, bits, s, nullptr));
            SH_CUDA(cc::dmalloc(&sort_tmp, tmp_bytes > 0 ? tmp_bytes : 16, s));
        }
        // copies start once these buffers exist on the compute stream
        SH_CUDA(cudaEventRecord(evs[2 * K], s));
        SH_CUDA(cudaStreamWaitEvent(cs, evs[2 * K], 0));
        const int sweep = (async && n > 0) ? 1 : 0;
        SH_CUDA(cudaMemsetAsync(&g->ctl->flag, 0, sizeof(int32_t), s));
        const int h = order == CC_ORDER_FULL ? cc::kFullChainHops : order;
        for (int64_t k = 0; k < K; ++k) {
            const int64_t off = chunks[k].first;
            const int64_t len = chunks[k].second;
            const int b = (int)(k & 1);
            int32_t* cs_src = sorted ? stg_s[b] : ds + off;  // where the copy lands
            int32_t* cs_dst = sorted ? stg_d[b] : dd + off;
            if (sorted && k >= 2) SH_CUDA(cudaStreamWaitEvent(cs, freed[k - 2], 0));
            SH_CUDA(cudaMemcpyAsync(cs_src, src + off, (size_t)len * sizeof(int32_t), cudaMemcpyHostToDevice, cs));
            SH_CUDA(cudaMemcpyAsync(cs_dst, dst + off, (size_t)len * sizeof(int32_t), cudaMemcpyHostToDevice, cs));
            SH_CUDA(cudaEventRecord(landed[k], cs));
            SH_CUDA(cudaStreamWaitEvent(s, landed[k], 0));
            auto ko = cc::chunk_orient_kernel;
            ko<<<grid_for(ko, len / 4 + 1), kThreads, 0, s>>>(cs_src, cs_dst, len, off, n, g->ctl);
            SH_CUDA(cudaGetLastError());
            if (sorted) {
                bool in_second = false;
                size_t tb = tmp_bytes;
                SH_CUDA(cc::sort_pairs_u32(sort_tmp, &tb, (uint32_t*)stg_s[b], (uint32_t*)(ds + off),
                                           (uint32_t*)stg_d[b], (uint32_t*)(dd + off), len, bits, s, &in_second));
                if (!in_second) {
                    SH_CUDA(cudaMemcpyAsync(ds + off, stg_s[b], (size_t)len * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
                    SH_CUDA(cudaMemcpyAsync(dd + off, stg_d[b], (size_t)len * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
                }
                SH_CUDA(cudaEventRecord(freed[k], s));
            }
            if (sweep) {
                SH_CUDA(order == 1   ? launch_chunk<1>(ds + off, dd + off, len, L, h, s)
                        : order == 2 ? launch_chunk<2>(ds + off, dd + off, len, L, h, s)
                                     : launch_chunk<0>(ds + off, dd + off, len, L, h, s));
            } else if (stream_ident) {
                auto ki = cc::chunk_identity_kernel;
                ki<<<grid_for(ki, len / 4 + 1), kThreads, 0, s>>>(ds + off, dd + off, len, L, &g->ctl->flag);
                SH_CUDA(cudaGetLastError());
            }
        }
    }
    SH_CUDA(cudaMemcpyAsync(g->ctl_h, g->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    SH_CUDA(cudaStreamSynchronize(s));
    if (g->ctl_h->bad_count)
        return done(set_error(CC_EIDRANGE, "%llu edges with an endpoint outside [0, %lld) (first at edge %llu)",
                              g->ctl_h->bad_count, (long long)n, g->ctl_h->first_bad));
    // a streamed first iteration that saw only loops is Alg. 1's last one:
    // the loop then starts afresh and stops after its one (identity) sweep
    const bool streamed = async ? (n > 0 && m > 0) : (stream_ident && g->ctl_h->flag != 0);
    // the ordinary loop of checked sweeps (cc_run), from the streamed labels
    st = run_impl(g, order, mode, c, streamed ? max_sweeps - 1 : max_sweeps, streamed ? L : nullptr, labels_out,
                  out_on_device, stats, s);
    if (stats) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev_start, g->ev1) == cudaSuccess) stats->solve_ms = ms;
        else cudaGetLastError();  // the loop stopped before its last event: keep cc_run's time
        if (streamed) {
            stats->sweeps += 1;
            // one sweep's algorithmic bytes, counted as cc_run counts them
            stats->alg_bytes += 8.0 * (double)m + (async ? 4.0 : 16.0) * (double)n;
        }
        stats->edges_per_s = stats->solve_ms > 0 ? (double)m / (stats->solve_ms * 1e-3) : 0.0;
    }
#undef SH_CUDA
    return done(st);
}

extern "C" cc_status cc_graph_edges(const cc_graph* g, const void** src, const void** dst) {
    if (!g) return set_error(CC_EINVAL, "cc_graph_edges: g is NULL");
    if (g->layout == CC_CSR_NATIVE || g->layout == CC_CSR_NATIVE_SYM) {
        if (src) *src = g->off;
        if (dst) *dst = g->dst;
        return CC_OK;
    }
    if (src) *src = g->src;
    if (dst) *dst = g->dst;
    return CC_OK;
}

extern "C" cc_status cc_graph_set_launch(cc_graph* g, int launch) {
    if (!g) return set_error(CC_EINVAL, "cc_graph_set_launch: g is NULL");
    if (launch != CC_LAUNCH_GRAPH && launch != CC_LAUNCH_HOST)
        return set_error(CC_EINVAL, "cc_graph_set_launch: launch must be CC_LAUNCH_GRAPH or CC_LAUNCH_HOST");
    g->launch = launch;
    return CC_OK;
}

extern "C" cc_status cc_graph_hubs(const cc_graph* g, const int32_t** hubs, int32_t* k) {
    if (!g) return set_error(CC_EINVAL, "cc_graph_hubs: g is NULL");
    if (hubs) *hubs = g->hubs;
    if (k) *k = g->hub_k;
    return CC_OK;
}

extern "C" cc_status cc_graph_perm(const cc_graph* g, const int32_t** perm, const int32_t** inv) {
    if (!g) return set_error(CC_EINVAL, "cc_graph_perm: g is NULL");
    if (perm) *perm = g->perm;
    if (inv) *inv = g->inv;
    return CC_OK;
}

extern "C" cc_status cc_graph_info(const cc_graph* g, int64_t* n, int64_t* m) {
    if (!g) return set_error(CC_EINVAL, "cc_graph_info: g is NULL");
    if (n) *n = g->n;
    if (m) *m = g->m;
    return CC_OK;
}

extern "C" void cc_free(cc_graph* g) { destroy(g); }

extern "C" const char* cc_strerror(cc_status s) {
    switch (s) {
        case CC_OK: return "success";
        case CC_EINVAL: return "invalid argument";
        case CC_EIDRANGE: return "vertex id out of range";
        case CC_ENOMEM: return "out of memory";
        case CC_ECUDA: return "CUDA error";
        case CC_ENOTCONVERGED: return "not converged within max_sweeps";
        case CC_ETIMEOUT: return "device-side wait timed out";
    }
    return "unknown status";
}

extern "C" const char* cc_last_error(void) { return g_last_error.c_str(); }

// Internals shared with the other translation units.
namespace cc {
const void* graph_src(const cc_graph* g) { return g->src; }
const void* graph_dst(const cc_graph* g) { return g->dst; }
int graph_id_bits(const cc_graph* g) { return g->id_bits; }
int graph_layout(const cc_graph* g) { return g->layout; }
int graph_hub_count(const cc_graph* g) { return g->hub_k; }
const int32_t* graph_hubs(const cc_graph* g) { return g->hubs; }
void graph_set_hubs(cc_graph* g, int32_t* hubs, int k) {
    free_loops(g);  // loop graphs captured the plain sweep kernel
    dfree(g->hubs, g->stream);
    g->hubs = hubs;
    g->hub_k = k;
}
const int64_t* graph_csr_off(const cc_graph* g) { return g->off; }
cudaStream_t graph_stream(const cc_graph* g) { return g->stream; }
SchedCtx** graph_sched_slot(cc_graph* g) { return &g->sched; }
void graph_set_relabel(cc_graph* g, int32_t* perm, int32_t* inv, int k) {
    free_loops(g);  // loop graphs captured the previous sweep kernel
    dfree(g->perm, g->stream);
    dfree(g->inv, g->stream);
    g->perm = perm;
    g->inv = inv;
    g->hub_k = k;
}
bool graph_relabeled(const cc_graph* g) { return g->perm != nullptr; }
cc_status graph_replace_edges(cc_graph* g, void* src, void* dst) {
    // cached loop graphs and scheduler features refer to the old arrays
    free_loops(g);
    sched_ctx_free(g->sched);
    g->sched = nullptr;
    dfree(g->hubs, g->stream);
    g->hubs = nullptr;
    g->hub_k = 0;
    if (g->own_edges) {
        dfree(g->src, g->stream);
        dfree(g->dst, g->stream);
    }
    g->src = src;
    g->dst = dst;
    g->own_edges = true;
    return CC_OK;
}
cc_status graph_nm(const cc_graph* g, long long* n, long long* m) {
    *n = g->n;
    *m = g->m;
    return CC_OK;
}
}  // namespace cc
