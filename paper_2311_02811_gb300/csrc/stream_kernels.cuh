// Sweeps of a streamed upload (cc_solve_host): the edge list crosses the host
// link in chunks, and each chunk is swept as soon as it has landed, while the
// chunks after it are still in flight.
//
// Why this is still Contour.  In the asynchronous iteration (Section III-B1)
// the operator may be applied to the edges in any order and at any time, and
// every application only lowers labels to ids of the same component (L[x] <= x
// and L[x] in x's component stay true).  Applying MM^h to the landed part of
// the list early is therefore one more legal order of applications; the loop
// of ordinary, checked sweeps that follows once the whole list is resident
// decides convergence exactly as cc_run does (Section III-B2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mm_kernels.cuh"

namespace cc {

// An edge whose endpoints are not both in [0, n) is counted (bad) and
// replaced by the self-loop <0, 0>, which reads L[0] and never writes it
// (L[0] = 0 always holds): no gather leaves the label array.
__device__ __forceinline__ void screen_edge(int32_t& w, int32_t& v, int64_t n, int64_t e, unsigned long long& bad,
                                            Ctl* ctl) {
    if ((uint32_t)w >= (uint64_t)n || (uint32_t)v >= (uint64_t)n) {
        ++bad;
        atomicMin(&ctl->first_bad, (unsigned long long)e);
        w = 0;
        v = 0;
    }
}

// A landed chunk in its staging arrays: every edge screened and stored in
// place as (smaller id, larger id), the chunk's sort keys and values.  Grouped
// by the smaller endpoint, the edges of a warp gather neighbouring labels on
// that side and a thread's edges often share it (one combined write).
__global__ void chunk_orient_kernel(int32_t* __restrict__ src, int32_t* __restrict__ dst, int64_t cnt,
                                    int64_t base, int64_t n, Ctl* ctl) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long bad = 0;
    const int64_t q4 = cnt / 4;
    for (int64_t g = tid; g < q4; g += stride) {
        int32_t w[4], v[4];
        load4(src + 4 * g, w);
        load4(dst + 4 * g, v);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            screen_edge(w[k], v[k], n, base + 4 * g + k, bad, ctl);
            const int32_t lo = w[k] < v[k] ? w[k] : v[k];
            v[k] = w[k] < v[k] ? v[k] : w[k];
            w[k] = lo;
        }
        reinterpret_cast<int4*>(src)[g] = make_int4(w[0], w[1], w[2], w[3]);
        reinterpret_cast<int4*>(dst)[g] = make_int4(v[0], v[1], v[2], v[3]);
    }
    const int64_t t = 4 * q4 + tid;
    if (t < cnt) {
        int32_t w = src[t], v = dst[t];
        screen_edge(w, v, n, base + t, bad, ctl);
        src[t] = w < v ? w : v;
        dst[t] = w < v ? v : w;
    }
    for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, o);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(&ctl->bad_count, bad);
}

// One chunk after its sort, at src/dst (16-byte aligned: chunks start at
// multiples of 4 edges of 256-byte aligned arrays; ids already screened by
// chunk_orient_kernel): MM^h (h = H, or h at run time for H = 0) applied once
// to every edge, asynchronously in place on L.
template <int H>
__global__ void __launch_bounds__(256, (H <= 2 && H > 0) ? 4 : 2)
chunk_sweep_kernel(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t cnt, int32_t* L,
                   int h) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t q4 = cnt / 4;
    for (int64_t g = tid; g < q4; g += stride) {
        int32_t w[4], v[4];
        load4(src + 4 * g, w);
        load4(dst + 4 * g, v);
        if constexpr (H > 0) mm_fixed<H, false, 4, int32_t>(w, v, L, nullptr);
        else mm_runtime_ilp<false, 4, int32_t>(w, v, h, L, nullptr);
    }
    const int64_t t = 4 * q4 + tid;
    if (t < cnt) {
        int32_t w[1] = {__ldcs(src + t)};
        int32_t v[1] = {__ldcs(dst + t)};
        if constexpr (H > 0) mm_fixed<H, false, 1, int32_t>(w, v, L, nullptr);
        else mm_runtime_ilp<false, 1, int32_t>(w, v, h, L, nullptr);
    }
}

// Alg. 1's first iteration on one chunk after its sort (synchronous solves):
// from L = id every chain is trivial, so each edge only lowers
// L_u[max(w, v)] to min(w, v) (see identity_pair).  The minima commute, so
// applying them chunk by chunk gives exactly the iteration's L_u.  target
// starts as the identity; *flag is raised if any edge is not a loop (the
// iteration's violation flag).
__global__ void chunk_identity_kernel(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t cnt,
                                      int32_t* target, int32_t* flag) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool viol = false;
    const int64_t q4 = cnt / 4;
    for (int64_t g = tid; g < q4; g += stride) {
        int32_t w[4], v[4];
        load4(src + 4 * g, w);
        load4(dst + 4 * g, v);
#pragma unroll
        for (int k = 0; k < 4; ++k) viol |= identity_pair(w[k], v[k], target);
    }
    const int64_t t = 4 * q4 + tid;
    if (t < cnt) viol |= identity_pair(__ldcs(src + t), __ldcs(dst + t), target);
    if (__syncthreads_or(viol) && threadIdx.x == 0) *flag = 1;
}

}  // namespace cc
