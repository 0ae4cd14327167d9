// Sweep with the labels of the highest-degree vertices ("hubs") held in
// shared memory (int32 ids, edge lists written by cc_graph_reorder with
// CC_REORDER_HUB).
//
// After that reorder every edge <w, v> is oriented from its lower-degree
// endpoint w, the list is sorted by w, and a v that is one of the K hubs is
// stored as ~slot (a negative value) with hubs[slot] = v.  On a power-law
// graph most edges end at a hub, and those label reads are the scattered
// half of the sweep's gathers: served from a shared-memory table, a warp's
// 32 reads cost a few bank cycles instead of up to 32 L1 tag lookups.
//
// The table holds the hubs' labels only (4 bytes each, 96 KB at most), so
// that most of the SM's L1 stays with the other gathers -- above all the
// second-level ones, whose targets (roots) are few and hot.  A hub's id is
// read from the global table (hubs) only when the sweep writes its label.
//
// The table is loaded from L at the start of every sweep.  Synchronous sweeps
// never write L, so it is exact.  Asynchronous sweeps may read a table entry
// that another block has lowered in L meanwhile; that is one more stale read
// of the kind the asynchronous iteration already has (Section III-B1): every
// value in the table is a label that the vertex held during the sweep, and a
// sweep without any write saw the current labels everywhere, so the
// convergence test stays exact.  A block lowers its own copy together with L.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mm_kernels.cuh"

namespace cc {

constexpr int kHubThreads = 1024;   // one block per SM
constexpr int kHubMax = 24576;      // table entries: one label each -> 96 KB
constexpr int kHubMinDegree = 16;   // vertices of lower degree are not worth a slot

// The block's view of the hubs: their labels in shared memory (lab[0..K)),
// their ids in global memory.
struct HubTab {
    int32_t* lab;
    const int32_t* id;
};

// x <- z for hub `slot` after a read saw its label above z.  Synchronous
// sweeps write L_u (tested at L2 first, see wr); asynchronous ones write L
// and lower the block's copy with it.  (A second table collecting the
// block's L_u minima for the hubs, as the renumbered layout keeps, made the
// synchronous sweeps of this layout slower: R-MAT 24 7.0 -> 9.1 ms, with the
// label table cut to half the hubs to make room.)
template <bool SYNC>
__device__ __forceinline__ void hub_write(int32_t* L, int32_t* Lu, const HubTab& T, int slot, int32_t z) {
    wr<SYNC>(L, Lu, T.id[slot], z);
    if constexpr (!SYNC) atomicMin(T.lab + slot, z);  // the block's copy follows L
}

// MM^h (h = H) on K edges whose v side may be a hub slot (see mm_fixed).
template <int H, bool SYNC, int K>
__device__ __forceinline__ bool mm_fixed_hub(const int32_t (&w)[K], const int32_t (&venc)[K], int32_t* L,
                                             int32_t* Lu, const HubTab& T) {
    int32_t cw[K][H + 1], cv[K][H + 1];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        cw[k][0] = w[k];
        cw[k][1] = rd<SYNC>(L, w[k]);
        if (venc[k] < 0) {
            cv[k][0] = -1;  // id read from the global table only if written
            cv[k][1] = T.lab[~venc[k]];
        } else {
            cv[k][0] = venc[k];
            cv[k][1] = rd<SYNC>(L, venc[k]);
        }
    }
#pragma unroll
    for (int j = 2; j <= H; ++j) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            cw[k][j] = (cw[k][j - 1] == cw[k][j - 2]) ? cw[k][j - 1] : rd<SYNC>(L, cw[k][j - 1]);
            cv[k][j] = (cv[k][j - 1] == cv[k][j - 2]) ? cv[k][j - 1] : rd<SYNC>(L, cv[k][j - 1]);
        }
    }
    bool viol = false;
    int32_t z[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        z[k] = cw[k][H] < cv[k][H] ? cw[k][H] : cv[k][H];
        viol |= (cw[k][1] > z[k]) | (cv[k][1] > z[k]);
    }
    // chains never increase, so no write is due unless some first label
    // exceeds z: the common case of a late sweep skips the write logic
    if (!viol) return false;
    // w side: the edges are sorted by w, so a thread's edges often share w
    // (and then their chains).  Equal chain vertices are adjacent; each run
    // of them gets one write of the run's smallest z.  That equals the
    // run's separate writes applied back to back: the conditional
    // assignments of Def. 1 commute, and the smallest one wins.
#pragma unroll
    for (int j = 0; j < H; ++j) {
        int32_t zr = z[0];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (k > 0) zr = (cw[k][j] == cw[k - 1][j]) ? (zr < z[k] ? zr : z[k]) : z[k];
            const bool last = (k == K - 1) || (cw[k + (k < K - 1)][j] != cw[k][j]);
            if (last && cw[k][j + 1] > zr) wr<SYNC>(L, Lu, cw[k][j], zr);
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
        for (int j = 0; j < H; ++j) {
            if (cv[k][j + 1] <= z[k]) continue;
            if (j == 0 && venc[k] < 0) hub_write<SYNC>(L, Lu, T, ~venc[k], z[k]);
            else wr<SYNC>(L, Lu, cv[k][j], z[k]);
        }
    }
    return viol;
}

// Run-time order h on K edges (see mm_runtime_ilp): only the first label of
// a hub's chain comes from the table.
template <bool SYNC, int K>
__device__ __forceinline__ bool mm_runtime_hub(const int32_t (&w)[K], const int32_t (&venc)[K], int h, int32_t* L,
                                               int32_t* Lu, const HubTab& T) {
    int32_t cur[2 * K], first[2 * K], x[2 * K];
    unsigned act = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        x[2 * k] = w[k];
        first[2 * k] = rd<SYNC>(L, w[k]);
        if (venc[k] < 0) {
            x[2 * k + 1] = -1;  // id read from the global table only if written
            first[2 * k + 1] = T.lab[~venc[k]];
        } else {
            x[2 * k + 1] = venc[k];
            first[2 * k + 1] = rd<SYNC>(L, venc[k]);
        }
    }
#pragma unroll
    for (int i = 0; i < 2 * K; ++i) {
        if (first[i] != x[i]) act |= 1u << i;
        cur[i] = first[i];
    }
    for (int j = 1; j < h && act; ++j) {
        int32_t y[2 * K];
#pragma unroll
        for (int i = 0; i < 2 * K; ++i) y[i] = (act >> i & 1u) ? rd<SYNC>(L, cur[i]) : cur[i];
#pragma unroll
        for (int i = 0; i < 2 * K; ++i) {
            if (y[i] == cur[i]) act &= ~(1u << i);
            cur[i] = y[i];
        }
    }
    int32_t z[K];
    unsigned wact = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        z[k] = cur[2 * k] < cur[2 * k + 1] ? cur[2 * k] : cur[2 * k + 1];
        if (first[2 * k] > z[k]) wact |= 1u << (2 * k);
        if (first[2 * k + 1] > z[k]) {
            if (venc[k] < 0) x[2 * k + 1] = T.id[~venc[k]];
            wact |= 1u << (2 * k + 1);
            if constexpr (!SYNC) {
                if (venc[k] < 0) atomicMin(T.lab + ~venc[k], z[k]);
            }
        }
    }
    const bool viol = wact != 0;
    for (int j = 0; j < h && wact; ++j) {
        int32_t y[2 * K];
#pragma unroll
        for (int i = 0; i < 2 * K; ++i) y[i] = (wact >> i & 1u) ? rd<SYNC>(L, x[i]) : x[i];
#pragma unroll
        for (int i = 0; i < 2 * K; ++i) {
            if (!(wact >> i & 1u)) continue;
            const int32_t zi = z[i >> 1];
            if (y[i] <= zi) {
                wact &= ~(1u << i);
                continue;
            }
            wr<SYNC>(L, Lu, x[i], zi);
            if (y[i] == x[i]) wact &= ~(1u << i);
            x[i] = y[i];
        }
    }
    return viol;
}

// The sweep (see mm_sweep_kernel for first / gate / flag).  One block of
// kHubThreads per SM; dynamic shared memory: 4 * K bytes (the labels).
template <int H, bool SYNC>
__global__ void __launch_bounds__(kHubThreads, 1)
mm_sweep_hub_kernel(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m, int32_t* L,
                    int32_t* Lu, int h, int32_t* flag, const Ctl* ctl, int first, int gate,
                    const int32_t* __restrict__ hubs, int K) {
    if (gate != 0 && ctl->sched_h != gate) return;
    extern __shared__ int32_t hub_smem[];
    const HubTab T{hub_smem, hubs};  // ids stay in global memory
    for (int i = threadIdx.x; i < K; i += blockDim.x) hub_smem[i] = rd<SYNC>(L, hubs[i]);
    __syncthreads();
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool viol = false;
    const bool ident = first == 2 || (first == 1 && ctl->sweeps == 0 && ctl->fresh != 0);
    if (ident) {
        int32_t* target = SYNC ? Lu : L;
        const int64_t q4 = m / 4;
        for (int64_t g = tid; g < q4; g += stride) {
            int32_t w[4], v[4];
            load4(src + g * 4, w);
            load4(dst + g * 4, v);
#pragma unroll
            for (int k = 0; k < 4; ++k) viol |= identity_pair(w[k], v[k] < 0 ? T.id[~v[k]] : v[k], target);
        }
        const int64_t t = q4 * 4 + tid;
        if (t < m) {
            const int32_t v = __ldcs(dst + t);
            viol |= identity_pair(__ldcs(src + t), v < 0 ? T.id[~v] : v, target);
        }
    } else {
        // The next group's edges are loaded before this group's gathers, so
        // the stream's DRAM latency overlaps the dependent label gathers.
        const int64_t q4 = m / 4;
        int32_t wn[4], vn[4];
        if (tid < q4) {
            load4(src + tid * 4, wn);
            load4(dst + tid * 4, vn);
        }
        for (int64_t g = tid; g < q4; g += stride) {
            int32_t w[4], v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                w[k] = wn[k];
                v[k] = vn[k];
            }
            const int64_t gn = g + stride;
            if (gn < q4) {
                load4(src + gn * 4, wn);
                load4(dst + gn * 4, vn);
            }
            if constexpr (H > 0) viol |= mm_fixed_hub<H, SYNC, 4>(w, v, L, Lu, T);
            else viol |= mm_runtime_hub<SYNC, 4>(w, v, h, L, Lu, T);
        }
        const int64_t t = q4 * 4 + tid;
        if (t < m) {
            int32_t w[1] = {__ldcs(src + t)};
            int32_t v[1] = {__ldcs(dst + t)};
            if constexpr (H > 0) viol |= mm_fixed_hub<H, SYNC, 1>(w, v, L, Lu, T);
            else viol |= mm_runtime_hub<SYNC, 1>(w, v, h, L, Lu, T);
        }
    }
    if (flag != nullptr) {
        if (__syncthreads_or(viol) && threadIdx.x == 0) *flag = 1;
    }
}

// Decoded (src, dst) pairs of S edges spread evenly over the m edges (edge
// floor(j * m / S)), for the scheduler's feature pass.
static __global__ void hub_sample_kernel(const int32_t* src, const int32_t* dst, int64_t m, int64_t S,
                                         const int32_t* hubs, int32_t* su, int32_t* sv) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < S; j += stride) {
        const int64_t e = (m <= S) ? j : (j * m) / S;
        const int32_t v = dst[e];
        su[j] = src[e];
        sv[j] = v < 0 ? hubs[~v] : v;
    }
}

}  // namespace cc
