// cc_graph_reorder: a one-time layout step that groups a handle's edges so
// that consecutive edges share (or neighbour) one endpoint.
//
// The operator is applied to every edge in any order (Alg. 1 processes the
// edge set with a parallel "forall"), so the order of the stored edges is a
// layout choice that never changes the result.  A sweep's cost is dominated
// by the first-level gathers L[w] and L[v]: with edges grouped by w the
// gathers of one warp fall into one or two cache lines, which roughly halves
// the scattered sectors per edge.
//
//   CC_REORDER_SRC     sort by src (stable radix sort of (src, dst) pairs)
//   CC_REORDER_LOWDEG  orient every edge from its lower-degree endpoint (ties:
//                      smaller id) to the other and sort by that endpoint, so
//                      the high-degree side -- whose labels stay hot in cache --
//                      is the scattered one
#include <cub/device/device_radix_sort.cuh>
#include <cuda_runtime.h>

#include "../../include/contour.h"
#include "cc_internal.h"

namespace {

__global__ void degree_kernel(const int32_t* src, const int32_t* dst, int64_t m, int32_t* deg) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        atomicAdd(deg + src[e], 1);
        atomicAdd(deg + dst[e], 1);
    }
}

// key = lower-degree endpoint, value = the other endpoint
__global__ void orient_kernel(const int32_t* src, const int32_t* dst, int64_t m, const int32_t* deg,
                              uint32_t* key, uint32_t* val) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const int32_t a = src[e], b = dst[e];
        const int32_t da = deg[a], db = deg[b];
        const bool swap = db < da || (db == da && b < a);
        key[e] = (uint32_t)(swap ? b : a);
        val[e] = (uint32_t)(swap ? a : b);
    }
}

__global__ void range_check_kernel(const uint32_t* a, const uint32_t* b, int64_t m, int64_t n,
                                   unsigned long long* bad) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long cnt = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride)
        cnt += ((int64_t)a[e] >= n) + ((int64_t)b[e] >= n);
    if (cnt) atomicAdd(bad, cnt);
}

int bits_for(int64_t n) {
    int b = 1;
    while (b < 31 && (int64_t(1) << b) < n) ++b;
    return b;
}

#define RCUDA(expr)                                                                  \
    do {                                                                             \
        cudaError_t e_ = (expr);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            st = cc::cuda_fail(e_, #expr, __FILE__, __LINE__);                       \
            goto done;                                                               \
        }                                                                            \
    } while (0)

}  // namespace

extern "C" cc_status cc_graph_reorder(cc_graph* g, int method) {
    cc::NvtxRange range("cc_graph_reorder");
    if (!g) return cc::set_error(CC_EINVAL, "cc_graph_reorder: g is NULL");
    if (method != CC_REORDER_SRC && method != CC_REORDER_LOWDEG)
        return cc::set_error(CC_EINVAL, "cc_graph_reorder: method must be CC_REORDER_SRC or CC_REORDER_LOWDEG");
    if (cc::graph_id_bits(g) != 32) return cc::set_error(CC_EINVAL, "cc_graph_reorder: int32 ids only");
    long long n = 0, m = 0;
    cc::graph_nm(g, &n, &m);
    if (m == 0) return CC_OK;
    cudaStream_t s = cc::graph_stream(g);
    const int32_t* src = static_cast<const int32_t*>(cc::graph_src(g));
    const int32_t* dst = static_cast<const int32_t*>(cc::graph_dst(g));
    cc_status st = CC_OK;
    uint32_t *k_in = nullptr, *v_in = nullptr, *k_out = nullptr, *v_out = nullptr;
    int32_t* deg = nullptr;
    void* tmp = nullptr;
    size_t tmp_bytes = 0;
    const int grid = cc::device_sms() * 8;
    RCUDA(cc::dmalloc(reinterpret_cast<void**>(&k_out), (size_t)m * sizeof(uint32_t), s));
    RCUDA(cc::dmalloc(reinterpret_cast<void**>(&v_out), (size_t)m * sizeof(uint32_t), s));
    if (method == CC_REORDER_LOWDEG) {
        RCUDA(cc::dmalloc(reinterpret_cast<void**>(&k_in), (size_t)m * sizeof(uint32_t), s));
        RCUDA(cc::dmalloc(reinterpret_cast<void**>(&v_in), (size_t)m * sizeof(uint32_t), s));
        RCUDA(cc::dmalloc(reinterpret_cast<void**>(&deg), (size_t)n * sizeof(int32_t), s));
        RCUDA(cudaMemsetAsync(deg, 0, (size_t)n * sizeof(int32_t), s));
        degree_kernel<<<grid, 256, 0, s>>>(src, dst, m, deg);
        RCUDA(cudaGetLastError());
        orient_kernel<<<grid, 256, 0, s>>>(src, dst, m, deg, k_in, v_in);
        RCUDA(cudaGetLastError());
    } else {
        k_in = reinterpret_cast<uint32_t*>(const_cast<int32_t*>(src));
        v_in = reinterpret_cast<uint32_t*>(const_cast<int32_t*>(dst));
    }
    RCUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, k_in, k_out, v_in, v_out, (long long)m, 0,
                                          bits_for(n), s));
    RCUDA(cc::dmalloc(&tmp, tmp_bytes, s));
    RCUDA(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, k_in, k_out, v_in, v_out, (long long)m, 0,
                                          bits_for(n), s));
    RCUDA(cudaStreamSynchronize(s));
    {
        // the sorted pairs must be a permutation of the oriented input: check
        // that every id is in range before the handle gathers with them
        unsigned long long* d_bad = nullptr;
        unsigned long long bad = 0;
        RCUDA(cc::dmalloc(reinterpret_cast<void**>(&d_bad), sizeof bad, s));
        RCUDA(cudaMemsetAsync(d_bad, 0, sizeof bad, s));
        range_check_kernel<<<grid, 256, 0, s>>>(k_out, v_out, m, n, d_bad);
        cudaError_t e2 = cudaGetLastError();
        if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(&bad, d_bad, sizeof bad, cudaMemcpyDeviceToHost, s);
        if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(s);
        cc::dfree(d_bad, s);
        RCUDA(e2);
        if (bad) {
            st = cc::set_error(CC_ECUDA, "cc_graph_reorder: internal error, %llu reordered ids out of range", bad);
            goto done;
        }
    }
    st = cc::graph_replace_edges(g, k_out, v_out);
    if (st == CC_OK) k_out = v_out = nullptr;  // now owned by the handle
done:
    if (method == CC_REORDER_LOWDEG) {
        cc::dfree(k_in, s);
        cc::dfree(v_in, s);
    }
    cc::dfree(deg, s);
    cc::dfree(tmp, s);
    cc::dfree(k_out, s);
    cc::dfree(v_out, s);
    return st;
}
