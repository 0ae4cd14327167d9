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
//   CC_REORDER_HUB     CC_REORDER_LOWDEG, then the (at most kHubMax) vertices
//                      of highest degree, if their degree is at least
//                      kHubMinDegree, become hubs: a dst entry naming hub
//                      number s is stored as ~s, and the sweep reads the hubs'
//                      labels from a shared-memory table (hub_kernels.cuh)
//   CC_REORDER_DEGREE  renumber the vertices in order of decreasing degree
//                      (ties: smaller id first), store every edge from its
//                      larger new id to its smaller and sort by the larger;
//                      the first (at most kHubMax) new ids of degree at least
//                      kHubMinDegree are read from shared memory at every
//                      step of a chain (relabel_kernels.cuh).  cc_run maps
//                      the labels back to the caller's ids.
#include <cub/device/device_radix_sort.cuh>
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "../../include/contour.h"
#include "cc_internal.h"
#include "hub_kernels.cuh"
#include "relabel_kernels.cuh"

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

// a[e] must be an id in [0, n); b[e] an id, or ~s for a hub slot s < K
__global__ void range_check_kernel(const uint32_t* a, const uint32_t* b, int64_t m, int64_t n, int64_t K,
                                   unsigned long long* bad) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long cnt = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const int32_t bv = (int32_t)b[e];
        cnt += ((int64_t)a[e] >= n) + (bv >= 0 ? (int64_t)bv >= n : (int64_t)(~bv) >= K);
    }
    if (cnt) atomicAdd(bad, cnt);
}

__global__ void iota_u32_kernel(uint32_t* x, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) x[i] = (uint32_t)i;
}

__global__ void hub_slots_kernel(const uint32_t* hubs, int K, int32_t* slot_of) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K; i += gridDim.x * blockDim.x)
        slot_of[hubs[i]] = i;
}

__global__ void hub_encode_kernel(uint32_t* v, int64_t m, const int32_t* slot_of) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const int32_t s = slot_of[v[e]];
        if (s >= 0) v[e] = (uint32_t)(~s);
    }
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

// The hubs: vertices sorted by degree (descending), the first ones of degree
// >= kHubMinDegree, at most kHubMax.  v (m high-side ids) is rewritten in
// place: an id that is hub number s becomes ~s.  *hubs_out (owned by the
// caller) receives the K hub ids; K = 0 leaves v unchanged.
cc_status select_and_encode_hubs(const int32_t* deg, int64_t n, uint32_t* v, int64_t m, cudaStream_t s,
                                 uint32_t** hubs_out, int* k_out) {
    *hubs_out = nullptr;
    *k_out = 0;
    cc_status st = CC_OK;
    uint32_t *ids = nullptr, *ids_sorted = nullptr;
    int32_t *deg_sorted = nullptr, *slot_of = nullptr;
    void* tmp = nullptr;
    size_t tmp_bytes = 0;
    const int grid = cc::device_sms() * 8;
    const int cap = (int)std::min<int64_t>(n, cc::kHubMax);
    std::vector<int32_t> top(cap > 0 ? cap : 1);
    int K = 0;
    RCUDA(cc::dmalloc(reinterpret_cast<void**>(&ids), (size_t)n * sizeof(uint32_t), s));
    RCUDA(cc::dmalloc(reinterpret_cast<void**>(&ids_sorted), (size_t)n * sizeof(uint32_t), s));
    RCUDA(cc::dmalloc(reinterpret_cast<void**>(&deg_sorted), (size_t)n * sizeof(int32_t), s));
    iota_u32_kernel<<<grid, 256, 0, s>>>(ids, n);
    RCUDA(cudaGetLastError());
    RCUDA(cub::DeviceRadixSort::SortPairsDescending(nullptr, tmp_bytes, deg, deg_sorted, ids, ids_sorted,
                                                    (long long)n, 0, 32, s));
    RCUDA(cc::dmalloc(&tmp, tmp_bytes, s));
    RCUDA(cub::DeviceRadixSort::SortPairsDescending(tmp, tmp_bytes, deg, deg_sorted, ids, ids_sorted,
                                                    (long long)n, 0, 32, s));
    if (cap > 0) RCUDA(cudaMemcpyAsync(top.data(), deg_sorted, (size_t)cap * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RCUDA(cudaStreamSynchronize(s));
    while (K < cap && top[K] >= cc::kHubMinDegree) ++K;
    if (K > 0) {
        RCUDA(cc::dmalloc(reinterpret_cast<void**>(&slot_of), (size_t)n * sizeof(int32_t), s));
        RCUDA(cudaMemsetAsync(slot_of, 0xff, (size_t)n * sizeof(int32_t), s));  // -1: not a hub
        hub_slots_kernel<<<(K + 255) / 256, 256, 0, s>>>(ids_sorted, K, slot_of);
        RCUDA(cudaGetLastError());
        hub_encode_kernel<<<grid, 256, 0, s>>>(v, m, slot_of);
        RCUDA(cudaGetLastError());
        RCUDA(cc::dmalloc(reinterpret_cast<void**>(hubs_out), (size_t)K * sizeof(uint32_t), s));
        RCUDA(cudaMemcpyAsync(*hubs_out, ids_sorted, (size_t)K * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
        RCUDA(cudaStreamSynchronize(s));
        *k_out = K;
    }
done:
    cc::dfree(ids, s);
    cc::dfree(ids_sorted, s);
    cc::dfree(deg_sorted, s);
    cc::dfree(slot_of, s);
    cc::dfree(tmp, s);
    if (st != CC_OK && *hubs_out) {
        cc::dfree(*hubs_out, s);
        *hubs_out = nullptr;
        *k_out = 0;
    }
    return st;
}

// CC_REORDER_DEGREE: renumber, orient, sort; hands the new edges, the two
// id maps and the shared-memory prefix length to the handle.
cc_status relabel_by_degree(cc_graph* g, const int32_t* src, const int32_t* dst, int64_t n, int64_t m,
                            cudaStream_t s) {
    cc_status st = CC_OK;
    int32_t *deg = nullptr, *deg_sorted = nullptr, *perm = nullptr;
    uint32_t *ids = nullptr, *inv = nullptr, *k_in = nullptr, *v_in = nullptr, *k_out = nullptr, *v_out = nullptr;
    void* tmp = nullptr;
    size_t tmp_bytes = 0, need = 0;
    const int grid = cc::device_sms() * 8;
    const int cap = (int)std::min<int64_t>(n, cc::kHubMax);
    std::vector<int32_t> top(cap > 0 ? cap : 1);
    int K = 0;
    RCUDA(cc::dmalloc(reinterpret_cast<void**>(&deg), (size_t)n * sizeof(int32_t), s));
    RCUDA(cc::dmalloc(reinterpret_cast<void**>(&deg_sorted), (size_t)n * sizeof(int32_t), s));
    RCUDA(cc::dmalloc(reinterpret_cast<void**>(&ids), (size_t)n * sizeof(uint32_t), s));
    RCUDA(cc::dmalloc(reinterpret_cast<void**>(&inv), (size_t)n * sizeof(uint32_t), s));
    RCUDA(cc::dmalloc(reinterpret_cast<void**>(&perm), (size_t)n * sizeof(int32_t), s));
    RCUDA(cudaMemsetAsync(deg, 0, (size_t)n * sizeof(int32_t), s));
    degree_kernel<<<grid, 256, 0, s>>>(src, dst, m, deg);
    RCUDA(cudaGetLastError());
    iota_u32_kernel<<<grid, 256, 0, s>>>(ids, n);
    RCUDA(cudaGetLastError());
    // stable: equal degrees keep increasing ids
    RCUDA(cub::DeviceRadixSort::SortPairsDescending(nullptr, need, deg, deg_sorted, ids, inv, (long long)n, 0, 32, s));
    tmp_bytes = need;
    RCUDA(cub::DeviceRadixSort::SortPairs(nullptr, need, k_in, k_out, v_in, v_out, (long long)m, 0, bits_for(n), s));
    tmp_bytes = std::max(tmp_bytes, need);
    RCUDA(cc::dmalloc(&tmp, tmp_bytes, s));
    RCUDA(cub::DeviceRadixSort::SortPairsDescending(tmp, tmp_bytes, deg, deg_sorted, ids, inv, (long long)n, 0, 32, s));
    if (cap > 0) RCUDA(cudaMemcpyAsync(top.data(), deg_sorted, (size_t)cap * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    cc::invert_perm_kernel<<<grid, 256, 0, s>>>(inv, n, perm);
    RCUDA(cudaGetLastError());
    cc::dfree(deg, s);
    cc::dfree(deg_sorted, s);
    cc::dfree(ids, s);
    deg = deg_sorted = nullptr;
    ids = nullptr;
    RCUDA(cc::dmalloc(reinterpret_cast<void**>(&k_in), (size_t)m * sizeof(uint32_t), s));
    RCUDA(cc::dmalloc(reinterpret_cast<void**>(&v_in), (size_t)m * sizeof(uint32_t), s));
    RCUDA(cc::dmalloc(reinterpret_cast<void**>(&k_out), (size_t)m * sizeof(uint32_t), s));
    RCUDA(cc::dmalloc(reinterpret_cast<void**>(&v_out), (size_t)m * sizeof(uint32_t), s));
    cc::relabel_orient_kernel<<<grid, 256, 0, s>>>(src, dst, m, perm, k_in, v_in);
    RCUDA(cudaGetLastError());
    RCUDA(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, k_in, k_out, v_in, v_out, (long long)m, 0, bits_for(n), s));
    RCUDA(cudaStreamSynchronize(s));
    while (K < cap && top[K] >= cc::kHubMinDegree) ++K;
    {
        // every stored id must be in range before the handle gathers with it
        unsigned long long* d_bad = nullptr;
        unsigned long long bad = 0;
        RCUDA(cc::dmalloc(reinterpret_cast<void**>(&d_bad), sizeof bad, s));
        RCUDA(cudaMemsetAsync(d_bad, 0, sizeof bad, s));
        range_check_kernel<<<grid, 256, 0, s>>>(k_out, v_out, m, n, 0, d_bad);
        cudaError_t e2 = cudaGetLastError();
        if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(&bad, d_bad, sizeof bad, cudaMemcpyDeviceToHost, s);
        if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(s);
        cc::dfree(d_bad, s);
        RCUDA(e2);
        if (bad) {
            st = cc::set_error(CC_ECUDA, "cc_graph_reorder: internal error, %llu renumbered ids out of range", bad);
            goto done;
        }
    }
    st = cc::graph_replace_edges(g, k_out, v_out);
    if (st == CC_OK) {
        k_out = v_out = nullptr;  // now owned by the handle
        cc::graph_set_relabel(g, perm, reinterpret_cast<int32_t*>(inv), K);
        perm = nullptr;
        inv = nullptr;
    }
done:
    cc::dfree(deg, s);
    cc::dfree(deg_sorted, s);
    cc::dfree(ids, s);
    cc::dfree(inv, s);
    cc::dfree(perm, s);
    cc::dfree(k_in, s);
    cc::dfree(v_in, s);
    cc::dfree(k_out, s);
    cc::dfree(v_out, s);
    cc::dfree(tmp, s);
    return st;
}

}  // namespace

namespace cc {

int key_bits(int64_t n) { return bits_for(n); }

cudaError_t sort_pairs_u32(void* temp, size_t* temp_bytes, uint32_t* k0, uint32_t* k1, uint32_t* v0, uint32_t* v1,
                           int64_t cnt, int end_bit, cudaStream_t s, bool* in_second) {
    cub::DoubleBuffer<uint32_t> keys(k0, k1), vals(v0, v1);
    cudaError_t e = cub::DeviceRadixSort::SortPairs(temp, *temp_bytes, keys, vals, (long long)cnt, 0, end_bit, s);
    if (in_second) *in_second = keys.Current() == k1;
    return e;
}

}  // namespace cc

extern "C" cc_status cc_graph_reorder(cc_graph* g, int method) {
    cc::NvtxRange range("cc_graph_reorder");
    if (!g) return cc::set_error(CC_EINVAL, "cc_graph_reorder: g is NULL");
    if (method != CC_REORDER_SRC && method != CC_REORDER_LOWDEG && method != CC_REORDER_HUB &&
        method != CC_REORDER_DEGREE)
        return cc::set_error(CC_EINVAL, "cc_graph_reorder: method must be CC_REORDER_SRC, CC_REORDER_LOWDEG, "
                                        "CC_REORDER_HUB or CC_REORDER_DEGREE");
    if (cc::graph_id_bits(g) != 32) return cc::set_error(CC_EINVAL, "cc_graph_reorder: int32 ids only");
    if (cc::graph_layout(g) != CC_COO)
        return cc::set_error(CC_EINVAL, "cc_graph_reorder: a native CSR handle keeps the caller's row order");
    if (cc::graph_hub_count(g) > 0)
        return cc::set_error(CC_EINVAL, "cc_graph_reorder: the edges are already hub-encoded (CC_REORDER_HUB)");
    if (cc::graph_relabeled(g))
        return cc::set_error(CC_EINVAL, "cc_graph_reorder: the vertices are already renumbered (CC_REORDER_DEGREE)");
    long long n = 0, m = 0;
    cc::graph_nm(g, &n, &m);
    if (m == 0) return CC_OK;
    cudaStream_t s = cc::graph_stream(g);
    const int32_t* src = static_cast<const int32_t*>(cc::graph_src(g));
    const int32_t* dst = static_cast<const int32_t*>(cc::graph_dst(g));
    if (method == CC_REORDER_DEGREE) return relabel_by_degree(g, src, dst, n, m, s);
    cc_status st = CC_OK;
    uint32_t *k_in = nullptr, *v_in = nullptr, *k_out = nullptr, *v_out = nullptr;
    int32_t* deg = nullptr;
    void* tmp = nullptr;
    size_t tmp_bytes = 0;
    uint32_t* hubs = nullptr;
    int hub_k = 0;
    const bool lowdeg = method != CC_REORDER_SRC;
    const int grid = cc::device_sms() * 8;
    RCUDA(cc::dmalloc(reinterpret_cast<void**>(&k_out), (size_t)m * sizeof(uint32_t), s));
    RCUDA(cc::dmalloc(reinterpret_cast<void**>(&v_out), (size_t)m * sizeof(uint32_t), s));
    if (lowdeg) {
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
    if (method == CC_REORDER_HUB) {
        st = select_and_encode_hubs(deg, n, v_out, m, s, &hubs, &hub_k);
        if (st != CC_OK) goto done;
    }
    {
        // the sorted pairs must be a permutation of the oriented input: check
        // that every id is in range before the handle gathers with them
        unsigned long long* d_bad = nullptr;
        unsigned long long bad = 0;
        RCUDA(cc::dmalloc(reinterpret_cast<void**>(&d_bad), sizeof bad, s));
        RCUDA(cudaMemsetAsync(d_bad, 0, sizeof bad, s));
        range_check_kernel<<<grid, 256, 0, s>>>(k_out, v_out, m, n, hub_k, d_bad);
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
    if (st == CC_OK) {
        k_out = v_out = nullptr;  // now owned by the handle
        if (hub_k > 0) {
            cc::graph_set_hubs(g, reinterpret_cast<int32_t*>(hubs), hub_k);
            hubs = nullptr;
        }
    }
done:
    cc::dfree(hubs, s);
    if (lowdeg) {
        cc::dfree(k_in, s);
        cc::dfree(v_in, s);
    }
    cc::dfree(deg, s);
    cc::dfree(tmp, s);
    cc::dfree(k_out, s);
    cc::dfree(v_out, s);
    return st;
}
