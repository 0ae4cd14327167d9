// Asynchronous full-chain sweeps with edge compaction (CC_ASYNC_COMPACT).
//
// With the full-chain operator an edge <w, v> walks both label chains to
// their roots r_w, r_v and lowers every chain entry above z = min(r_w, r_v)
// to z.  Once both walks of an edge end at the same root, the edge has, for
// now, nothing left to do: its endpoints lie in one tree of the pointer graph.
// Compacting sweeps drop such edges and append the others to a second edge
// list that the next compacting sweep reads, so later sweeps stream only the
// edges that still merge trees.
//
// Dropping is a heuristic, not a proof: in the asynchronous iteration a write
// walk that read a stale chain can stop below a tree's current root and move
// a vertex to another tree without its root (and a walk cut at the 1024-hop
// cap does the same), so a dropped edge can become active again.  The
// convergence test therefore stays the paper's (Section III-B2), over every
// edge: when a compacting sweep sees no violation among the edges it read,
// the next sweep is an ordinary full-chain sweep over all edges; if that one
// sees a violation, ordinary sweeps continue until one sees none.  The phase
// lives in Ctl::sched_h (1: compacting, kFullChainHops: ordinary), so the
// compacting kernel and the ordinary kernel are both in the loop body and
// only the one of the current phase runs.
//
// Edge lists: compacting sweep k of a run (k = 0, 1, ...; compacting sweeps
// come first) reads the caller's edges (k = 0) or list (k - 1) & 1 and
// appends the edges it keeps to list k & 1.  cnt[0..2] count the edges
// appended in sweeps k = 0, 1, 2 (mod 3); cnt[3] accumulates the edges read
// by the compacting sweeps of the run and cnt[4] counts those sweeps.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mm_kernels.cuh"

namespace cc {

struct CompactLists {
    int32_t* src[2];
    int32_t* dst[2];
    unsigned long long* cnt;  // 5 words (see above)
};

// Full-chain MM on K edges (lockstep walks as in mm_runtime_ilp, h = the cap)
// and, per edge, whether it may be dropped: both walks ended at a root and
// the roots are equal.
template <int K>
__device__ __forceinline__ bool mm_full_compact(const int32_t (&w)[K], const int32_t (&v)[K], int32_t* L,
                                                unsigned& drop) {
    constexpr int h = kFullChainHops;
    int32_t cur[2 * K], first[2 * K];
    unsigned act = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        cur[2 * k] = w[k];
        cur[2 * k + 1] = v[k];
    }
#pragma unroll
    for (int i = 0; i < 2 * K; ++i) {
        first[i] = L[cur[i]];
        if (first[i] != cur[i]) act |= 1u << i;
        cur[i] = first[i];
    }
    for (int j = 1; j < h && act; ++j) {
        int32_t y[2 * K];
#pragma unroll
        for (int i = 0; i < 2 * K; ++i) y[i] = (act >> i & 1u) ? L[cur[i]] : cur[i];
#pragma unroll
        for (int i = 0; i < 2 * K; ++i) {
            if (y[i] == cur[i]) act &= ~(1u << i);
            cur[i] = y[i];
        }
    }
    // act: chains that did not reach a root within the cap
    drop = 0;
    int32_t z[K];
    unsigned wact = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        z[k] = cur[2 * k] < cur[2 * k + 1] ? cur[2 * k] : cur[2 * k + 1];
        if (first[2 * k] > z[k]) wact |= 1u << (2 * k);
        if (first[2 * k + 1] > z[k]) wact |= 1u << (2 * k + 1);
        const bool roots = !(act >> (2 * k) & 1u) && !(act >> (2 * k + 1) & 1u);
        if (roots && cur[2 * k] == cur[2 * k + 1]) drop |= 1u << k;
    }
    const bool viol = wact != 0;
    int32_t x[2 * K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        x[2 * k] = w[k];
        x[2 * k + 1] = v[k];
    }
    for (int j = 0; j < h && wact; ++j) {
        int32_t y[2 * K];
#pragma unroll
        for (int i = 0; i < 2 * K; ++i) y[i] = (wact >> i & 1u) ? L[x[i]] : x[i];
#pragma unroll
        for (int i = 0; i < 2 * K; ++i) {
            if (!(wact >> i & 1u)) continue;
            const int32_t zi = z[i >> 1];
            if (y[i] <= zi) {
                wact &= ~(1u << i);
                continue;
            }
            red_min(L + x[i], zi);
            if (y[i] == x[i]) wact &= ~(1u << i);
            x[i] = y[i];
        }
    }
    return viol;
}

// Append the kept edges of this lane (keep bit i for edge i of n) to the
// output list, one atomic per warp.
template <int K>
__device__ __forceinline__ void append_kept(const int32_t (&w)[K], const int32_t (&v)[K], unsigned keep,
                                            int32_t* os, int32_t* od, unsigned long long* ocnt) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned mine = __popc(keep);
    unsigned incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(full, incl, o);
        if (lane >= o) incl += y;
    }
    const unsigned total = __shfl_sync(full, incl, 31);
    unsigned long long base = 0;
    if (lane == 31 && total) base = atomicAdd(ocnt, (unsigned long long)total);
    base = __shfl_sync(full, base, 31);
    unsigned long long pos = base + (incl - mine);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (keep >> k & 1u) {
            os[pos] = w[k];
            od[pos] = v[k];
            ++pos;
        }
    }
}

// One compacting sweep (k = ctl->sweeps); returns at once outside the
// compacting phase.
__global__ void __launch_bounds__(256)
mm_sweep_compact_kernel(const int32_t* __restrict__ src0, const int32_t* __restrict__ dst0, int64_t m0,
                        CompactLists lists, int32_t* L, int32_t* flag, const Ctl* ctl) {
    if (ctl->sched_h != 1) return;
    const int32_t k = ctl->sweeps;
    const int32_t* src = k == 0 ? src0 : lists.src[(k - 1) & 1];
    const int32_t* dst = k == 0 ? dst0 : lists.dst[(k - 1) & 1];
    const int64_t m = k == 0 ? m0 : (int64_t)lists.cnt[(k + 2) % 3];
    int32_t* os = lists.src[k & 1];
    int32_t* od = lists.dst[k & 1];
    unsigned long long* ocnt = lists.cnt + (k % 3);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        lists.cnt[(k + 1) % 3] = 0;  // the list the next sweep appends to
        lists.cnt[3] += (unsigned long long)m;
        lists.cnt[4] += 1;
    }
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t q4 = m / 4;
    // every lane of a warp runs the same number of iterations (the warp-wide
    // append needs all 32 lanes): the loop bound is rounded up to whole warps
    const int64_t iters = (q4 + stride - 1) / stride;
    bool viol = false;
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t g = tid + it * stride;
        int32_t w[4] = {0, 0, 0, 0}, v[4] = {0, 0, 0, 0};
        unsigned drop = 0xfu;
        if (g < q4) {
            load4(src + g * 4, w);
            load4(dst + g * 4, v);
            viol |= mm_full_compact<4>(w, v, L, drop);
        }
        append_kept<4>(w, v, ~drop & 0xfu, os, od, ocnt);
    }
    {
        const int64_t t = q4 * 4 + tid;
        int32_t w[1] = {0}, v[1] = {0};
        unsigned drop = 1u;
        if (t < m) {
            w[0] = __ldcs(src + t);
            v[0] = __ldcs(dst + t);
            viol |= mm_full_compact<1>(w, v, L, drop);
        }
        // only the first warps hold tail edges; every lane of a warp takes part
        if (tid - (threadIdx.x & 31) < m - q4 * 4) append_kept<1>(w, v, ~drop & 1u, os, od, ocnt);
    }
    if (flag != nullptr) {
        if (__syncthreads_or(viol) && threadIdx.x == 0) *flag = 1;
    }
}

// End of a loop iteration of a compacting run: a clean compacting sweep
// switches to an ordinary sweep over all edges; an ordinary sweep ends the
// run when it saw no violation.  loop_cond == nullptr: host-polled run (the
// host reads ctl).
__device__ __forceinline__ int compact_check(Ctl* ctl) {
    const int32_t f = ctl->flag;
    ctl->flag = 0;
    ctl->sweeps += 1;
    if (ctl->sched_h == 1) {
        if (f == 0) ctl->sched_h = kFullChainHops;
        ctl->converged = 0;
        return ctl->sweeps < ctl->max_sweeps;
    }
    ctl->converged = (f == 0);
    return f != 0 && ctl->sweeps < ctl->max_sweeps;
}

static __global__ void compact_check_kernel(Ctl* ctl, cudaGraphConditionalHandle loop) {
    if (threadIdx.x == 0) cudaGraphSetConditional(loop, compact_check(ctl) ? 1u : 0u);
}

static __global__ void compact_check_host_kernel(Ctl* ctl) {
    if (threadIdx.x == 0) compact_check(ctl);
}

}  // namespace cc
