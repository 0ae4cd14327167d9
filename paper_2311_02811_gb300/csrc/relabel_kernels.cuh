// Sweep and label mapping for handles whose vertices were renumbered in order
// of decreasing degree (cc_graph_reorder with CC_REORDER_DEGREE).
//
// Layout.  Vertex x of the caller becomes perm[x]; inv is the inverse.  Ids
// are given by decreasing degree (ties: smaller id first), so the labels most
// edges touch are packed at the front of L, where a few hundred KB of cache
// lines serve most gathers and the label array's hot part stays in L2 even
// when the whole array (537 MB at R-MAT scale 27) does not.  Every edge <w, v>
// is stored with w > v (w the lower-degree endpoint), sorted by w.  The K
// highest-degree vertices are ids 0..K-1: a label x < K is read from a
// shared-memory copy of L[0..K), and no id table or edge encoding is needed.
//
// The iteration itself is Contour on the renumbered graph, which is the
// caller's graph up to isomorphism: Def. 3 and Alg. 1 apply unchanged and
// reach, per component, the star rooted at its smallest NEW id.  The caller's
// labels are recovered by one more pass: each tree of the final (or stopped)
// state is labelled by the smallest ORIGINAL id among its members.  At the
// fixed point a tree is a component, so that is the component's minimum id,
// the unique result of reading 1; for a stopped run it is a valid resume
// snapshot (every label is an id of the same component, not above the vertex's
// own id).  A snapshot passed back in is mapped the other way: each tree of
// it is labelled by its smallest new id.
//
// The shared-memory copy.  It is loaded from L at the start of every sweep.
// Synchronous sweeps never write L, so it is exact.  In an asynchronous sweep
// a block lowers its copy together with L, and may read an entry that another
// block has lowered in L meanwhile: a stale read of the kind Section III-B1
// already allows (the value is a label the vertex held during the sweep), and
// a sweep without any write saw the current labels everywhere, so the early
// convergence test stays exact.  The copy is never below L[x] (L takes every
// write the copy takes), so a write that the copy already holds is a no-op on
// L and is not issued.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hub_kernels.cuh"
#include "mm_kernels.cuh"

namespace cc {

// Label of x: the shared-memory copy for ids below K.
template <bool SYNC>
__device__ __forceinline__ int32_t plab(const int32_t* L, const int32_t* tab, int K, int32_t x) {
    return x < K ? tab[x] : rd<SYNC>(L, x);
}

// Conditional assignment x <- z after a read saw a label of x above z.
// Synchronous sweeps (L read-only, every write into L_u) keep a second table
// tab[K..2K) that collects the block's minima for L_u[0..K); the sweep's end
// merges it into L_u (flush_prefix_lu), so the hottest targets take no
// global atomics during the sweep.  The result is the same minimum.
template <bool SYNC>
__device__ __forceinline__ void pwr(int32_t* L, int32_t* Lu, int32_t* tab, int K, int32_t x, int32_t z) {
    if constexpr (SYNC) {
        if (x < K) atomicMin(tab + K + x, z);
        else wr<true>(L, Lu, x, z);
    } else {
        if (x < K && atomicMin(tab + x, z) <= z) return;  // L[x] <= copy <= z already
        red_min(L + x, z);
    }
}

// MM^h (h = H) on K edges (see mm_fixed): the first label of each chain
// through plab, the later ones from L -- they are mostly roots, few and hot,
// which L1 serves as well as the table, and the select costs registers
// (measured: synchronous R-MAT 24 4.07 -> 3.80 ms, R-MAT 27 36.6 -> 33.7 ms).
// The w-side writes are combined per run of equal chain vertices as in
// mm_fixed_hub.
template <int H, bool SYNC, int K>
__device__ __forceinline__ bool mm_fixed_prefix(const int32_t (&w)[K], const int32_t (&v)[K], int32_t* L,
                                                int32_t* Lu, int32_t* tab, int KH) {
    int32_t cw[K][H + 1], cv[K][H + 1];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        cw[k][0] = w[k];
        cv[k][0] = v[k];
        cw[k][1] = plab<SYNC>(L, tab, KH, w[k]);
        cv[k][1] = plab<SYNC>(L, tab, KH, v[k]);
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
    if (!viol) return false;  // no write is due (see mm_fixed_hub)
#pragma unroll
    for (int j = 0; j < H; ++j) {
        int32_t zr = z[0];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (k > 0) zr = (cw[k][j] == cw[k - 1][j]) ? (zr < z[k] ? zr : z[k]) : z[k];
            const bool last = (k == K - 1) || (cw[k + (k < K - 1)][j] != cw[k][j]);
            if (last && cw[k][j + 1] > zr) pwr<SYNC>(L, Lu, tab, KH, cw[k][j], zr);
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
        for (int j = 0; j < H; ++j)
            if (cv[k][j + 1] > z[k]) pwr<SYNC>(L, Lu, tab, KH, cv[k][j], z[k]);
    }
    return viol;
}

// Run-time order h (orders other than 1, 2, 4, and the full chain) on K edges:
// the 2K chains advance in lockstep and stop at their roots (mm_runtime_ilp).
template <bool SYNC, int K>
__device__ __forceinline__ bool mm_runtime_prefix(const int32_t (&w)[K], const int32_t (&v)[K], int h, int32_t* L,
                                                  int32_t* Lu, int32_t* tab, int KH) {
    int32_t cur[2 * K], first[2 * K], x[2 * K];
    unsigned act = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        x[2 * k] = w[k];
        x[2 * k + 1] = v[k];
    }
#pragma unroll
    for (int i = 0; i < 2 * K; ++i) {
        first[i] = plab<SYNC>(L, tab, KH, x[i]);
        if (first[i] != x[i]) act |= 1u << i;
        cur[i] = first[i];
    }
    for (int j = 1; j < h && act; ++j) {
        int32_t y[2 * K];
#pragma unroll
        for (int i = 0; i < 2 * K; ++i) y[i] = (act >> i & 1u) ? plab<SYNC>(L, tab, KH, cur[i]) : cur[i];
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
        if (first[2 * k + 1] > z[k]) wact |= 1u << (2 * k + 1);
    }
    const bool viol = wact != 0;
    for (int j = 0; j < h && wact; ++j) {
        int32_t y[2 * K];
#pragma unroll
        for (int i = 0; i < 2 * K; ++i) y[i] = (wact >> i & 1u) ? plab<SYNC>(L, tab, KH, x[i]) : x[i];
#pragma unroll
        for (int i = 0; i < 2 * K; ++i) {
            if (!(wact >> i & 1u)) continue;
            const int32_t zi = z[i >> 1];
            if (y[i] <= zi) {  // labels further down the chain are <= y
                wact &= ~(1u << i);
                continue;
            }
            pwr<SYNC>(L, Lu, tab, KH, x[i], zi);
            if (y[i] == x[i]) wact &= ~(1u << i);  // root
            x[i] = y[i];
        }
    }
    return viol;
}

// End of a synchronous sweep: the block's minima for L_u[0..K) go to L_u.
__device__ __forceinline__ void flush_prefix_lu(int32_t* Lu, const int32_t* tab, int K) {
    __syncthreads();
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
        const int32_t u = tab[K + i];
        if (u < tab[i] && __ldcg(Lu + i) > u) red_min(Lu + i, u);
    }
}

// The sweep (see mm_sweep_kernel for first / gate / flag).  One block of
// kHubThreads per SM; dynamic shared memory: 4 * KH bytes (labels of ids
// below KH), twice that for synchronous sweeps (the L_u minima).  The next
// group's edges are loaded before this group's gathers.
template <int H, bool SYNC>
__global__ void __launch_bounds__(kHubThreads, 1)
mm_sweep_prefix_kernel(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m, int32_t* L,
                       int32_t* Lu, int h, int32_t* flag, const Ctl* ctl, int first, int gate, int KH) {
    if (gate != 0 && ctl->sched_h != gate) return;
    extern __shared__ int32_t prefix_smem[];
    int32_t* tab = prefix_smem;
    for (int i = threadIdx.x; i < KH; i += blockDim.x) {
        tab[i] = rd<SYNC>(L, i);
        if constexpr (SYNC) tab[KH + i] = tab[i];  // L_u = L at the start of a sweep
    }
    __syncthreads();
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool viol = false;
    const bool ident = first == 2 || (first == 1 && ctl->sweeps == 0 && ctl->fresh != 0);
    const int64_t q4 = m / 4;
    if (ident) {
        // from L = id every chain is trivial: the larger endpoint (stored
        // first) takes the smaller id (see mm_sweep_kernel); one write per run
        // of equal w with the run's smallest v (a loop has v == w: no write)
        for (int64_t g = tid; g < q4; g += stride) {
            int32_t w[4], v[4];
            load4(src + g * 4, w);
            load4(dst + g * 4, v);
            int32_t zr = v[0];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (k > 0) zr = (w[k] == w[k - 1]) ? (zr < v[k] ? zr : v[k]) : v[k];
                const bool last = (k == 3) || (w[k + (k < 3)] != w[k]);
                if (last && zr < w[k]) {
                    pwr<SYNC>(L, Lu, tab, KH, w[k], zr);
                    viol = true;
                }
            }
        }
        const int64_t t = q4 * 4 + tid;
        if (t < m) {
            const int32_t w = __ldcs(src + t), v = __ldcs(dst + t);
            if (w != v) {
                pwr<SYNC>(L, Lu, tab, KH, w, v);
                viol = true;
            }
        }
    } else {
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
            if constexpr (H > 0) viol |= mm_fixed_prefix<H, SYNC, 4>(w, v, L, Lu, tab, KH);
            else viol |= mm_runtime_prefix<SYNC, 4>(w, v, h, L, Lu, tab, KH);
        }
        const int64_t t = q4 * 4 + tid;
        if (t < m) {
            int32_t w[1] = {__ldcs(src + t)};
            int32_t v[1] = {__ldcs(dst + t)};
            if constexpr (H > 0) viol |= mm_fixed_prefix<H, SYNC, 1>(w, v, L, Lu, tab, KH);
            else viol |= mm_runtime_prefix<SYNC, 1>(w, v, h, L, Lu, tab, KH);
        }
    }
    if constexpr (SYNC) flush_prefix_lu(Lu, tab, KH);
    if (flag != nullptr) {
        if (__syncthreads_or(viol) && threadIdx.x == 0) *flag = 1;
    }
}

// ---------------------------------------------------------------------------
// label mapping between the caller's ids and the renumbered ids
// ---------------------------------------------------------------------------

constexpr int kMapChaseCap = 1 << 24;  // chains strictly decrease; the walk is capped all the same

// Root of x's tree in a label array whose chains never increase.
__device__ __forceinline__ int32_t chase_root(const int32_t* L, int32_t x, unsigned long long* overflow) {
    int32_t r = L[x];
    for (int guard = 0; guard < kMapChaseCap; ++guard) {
        const int32_t p = L[r];
        if (p == r) return r;
        r = p;
    }
    atomicAdd(overflow, 1ull);
    return r;
}

// tree_min[root(y)] = min over the tree's members y of key[y].  tree_min must
// hold INT32_MAX at every root beforehand.  Most members of a power-law graph
// share one root (the giant component's), so each lane keeps a running
// minimum per run of equal roots over its slice of a warp tile and issues one
// atomic per run; a warp whose lanes all end on the same root issues one.
// ctl != nullptr and ctl->converged: the compress has made L a set of stars,
// root(y) = L[y], and a lane's loads are independent (4 in flight per step);
// otherwise every chain is walked to its root.
static __global__ void tree_min_kernel(const int32_t* L, const int32_t* key, int64_t n, int32_t* tree_min,
                                       const Ctl* ctl, unsigned long long* overflow) {
    constexpr int kPerLane = 64;
    const bool stars = ctl != nullptr && ctl->converged != 0;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t tile = 32 * kPerLane;
    int32_t racc = -1, kacc = 0x7fffffff;
    auto take = [&](int32_t r, int32_t kv) {
        if (r == racc) {
            kacc = kv < kacc ? kv : kacc;
        } else {
            if (racc >= 0) atomicMin(tree_min + racc, kacc);
            racc = r;
            kacc = kv;
        }
    };
    for (int64_t base = warp * tile; base < n; base += nwarps * tile) {
        if (stars && base + tile <= n) {
            for (int i = 0; i < kPerLane; i += 4) {
                int32_t r[4], kv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t y = base + (int64_t)(i + u) * 32 + lane;
                    r[u] = L[y];
                    kv[u] = key[y];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) take(r[u], kv[u]);
            }
            continue;
        }
        for (int i = 0; i < kPerLane; ++i) {
            const int64_t y = base + (int64_t)i * 32 + lane;
            if (y >= n) break;
            take(stars ? L[y] : chase_root(L, (int32_t)y, overflow), key[y]);
        }
    }
    const int32_t r0 = __shfl_sync(0xffffffffu, racc, 0);
    if (__all_sync(0xffffffffu, racc == r0)) {
        for (int o = 16; o > 0; o >>= 1) {
            const int32_t other = __shfl_xor_sync(0xffffffffu, kacc, o);
            kacc = other < kacc ? other : kacc;
        }
        if (lane == 0 && racc >= 0) atomicMin(tree_min + racc, kacc);
    } else if (racc >= 0) {
        atomicMin(tree_min + racc, kacc);
    }
}

// out[x] = tree_min[root(map[x])]: labels of one id space from a label array
// of the other (map: caller id -> renumbered id, or the reverse); stars as
// for tree_min_kernel.
static __global__ void map_labels_kernel(const int32_t* L, const int32_t* map, const int32_t* tree_min, int64_t n,
                                         int32_t* out, const Ctl* ctl, unsigned long long* overflow) {
    const bool stars = ctl != nullptr && ctl->converged != 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
        const int32_t y = map[x];
        const int32_t r = stars ? L[y] : chase_root(L, y, overflow);
        out[x] = tree_min[r];
    }
}

// The renumbering: inv[r] = the r-th vertex in order of decreasing degree
// (from a stable sort), perm = its inverse.
static __global__ void invert_perm_kernel(const uint32_t* inv, int64_t n, int32_t* perm) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) perm[inv[r]] = (int32_t)r;
}

// key = the larger renumbered endpoint (the lower-degree one), value = the other.
static __global__ void relabel_orient_kernel(const int32_t* src, const int32_t* dst, int64_t m, const int32_t* perm,
                                             uint32_t* key, uint32_t* val) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const int32_t a = perm[src[e]], b = perm[dst[e]];
        key[e] = (uint32_t)(a > b ? a : b);
        val[e] = (uint32_t)(a > b ? b : a);
    }
}

}  // namespace cc
