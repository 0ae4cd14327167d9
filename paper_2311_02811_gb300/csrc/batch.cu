// Batched Contour: thousands of independent graphs, concatenated, solved by
// one CUDA-graph launch (include/contour.h: cc_batch_init / cc_batch_run).
//
// Each graph g owns vertices [off_v[g], off_v[g+1]) of the label array and
// edges [off_e[g], off_e[g+1]) of src/dst, whose ids are local (0..n_g-1).
// Every graph runs its own Contour iteration (Alg. 1 / Section III-B) with
// its own operator order, mode, check interval, flag and sweep count.
//
// Work is split by size:
//  * small graphs (labels fit the shared-memory budget) are solved whole by
//    one CTA each: labels live in shared memory for all sweeps, edges are
//    streamed from global memory; a persistent kernel pulls graphs, largest
//    first, from an atomic counter;
//  * large graphs run in rounds inside a conditional WHILE node: one sweep
//    per round for every active large graph, as tiles of kWarpTile edges,
//    each warp taking a contiguous range of tiles of the persistent grid (one
//    kernel per operator-order class; no block-wide barrier), then a
//    one-block check kernel that applies each graph's convergence test
//    (Section III-B2), retires converged graphs and rebuilds the active
//    lists and tile prefix sums for the next round.
//    The large graphs are split into waves whose labels together fit in L2
//    (kWaveBytes); the next wave is admitted once the active work left falls
//    below what keeps the grid busy (a wave's last rounds hold only its
//    slowest graphs).  Every graph still runs its own iteration from its own
//    first sweep (its start round is recorded), so waves change nothing but
//    which graphs share a round: with all large graphs in one round, their
//    labels (gigabytes for a big batch) would not stay in L2 and every
//    scattered label gather would go to DRAM.
// No kernel waits on another CTA; rounds are separated by kernel boundaries.
#include <cub/device/device_radix_sort.cuh>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/contour.h"
#include "cc_internal.h"
#include "mm_kernels.cuh"

namespace {

using cc::red_min;

constexpr int kClasses = 4;        // order classes: 0: h=1, 1: h=2, 2: h=4, 3: run-time h
constexpr int kLargeThreads = 256;
constexpr int kEPT = 4;            // edges per thread per tile
constexpr int kTile = kLargeThreads * kEPT;   // edges per tile of validation and reorder passes
constexpr int kWarpTile = 32 * kEPT;          // edges per round-kernel tile (one warp)
constexpr int kVTile = 1024;       // vertices per tile (init, copy, compress)
constexpr int kCheckThreads = 1024;
constexpr long long kWaveBytes = 64ll << 20;  // label (and L_u) bytes of the large graphs of one wave

enum : int32_t { kActive = 0, kConverged = 1, kStopped = 2 };

int order_class(int order) {
    switch (order) {
        case 1: return 0;
        case 2: return 1;
        case 4: return 2;
        default: return 3;
    }
}

struct BatchCtl {
    int32_t round;       // rounds completed
    int32_t wave;        // last wave of large graphs admitted
    int32_t n_waves;
    long long admit_tiles;  // admit the next wave while fewer tiles are active
    int32_t max_sweeps;
    int32_t small_next;  // queue head of the small-graph kernel
    int32_t sact_cnt;    // active synchronous large graphs
    int32_t act_cnt[kClasses];
    long long tiles[kClasses];
    long long vtiles;    // vertex tiles of active synchronous large graphs
    unsigned long long compress_changes;
    unsigned long long bad_count;
    unsigned long long first_bad;
};

// Device view of a batch plan.
struct Dev {
    int32_t G;
    const int64_t* off_v;
    const int64_t* off_e;
    const int32_t* src;
    const int32_t* dst;
    int32_t* L;   // labels (caller's output)
    int32_t* Lu;  // update array for synchronous graphs (nullptr if none)
    // per graph
    const int32_t* h;     // operator order (1024 for the full chain)
    const int32_t* sync;  // 1 = synchronous
    const int32_t* c;     // check interval
    int32_t* flag;
    int32_t* sweeps;
    int32_t* state;
    const int32_t* wave;  // wave of each large graph
    int32_t* start;       // rounds completed when the graph's wave was admitted
    // small graphs
    const int32_t* small_list;
    int32_t n_small;
    // large graphs
    const int32_t* large_cls[kClasses];  // static lists per class (setup)
    int32_t large_cls_cnt[kClasses];
    int32_t* act[kClasses];
    long long* tpre[kClasses];  // tile prefix over act[k]
    int32_t* sact;
    long long* vpre;            // vertex-tile prefix over sact
    // all large graphs, for init and compress
    const int32_t* large_all;
    const long long* large_vpre;
    int32_t n_large;
    long long large_vtiles;
    BatchCtl* ctl;
};

__device__ __forceinline__ int find_tile(const long long* pre, int cnt, long long t) {
    // largest i with pre[i] <= t (pre[0] = 0, pre[cnt] = total)
    int lo = 0, hi = cnt;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= t) lo = mid; else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// block scan helpers (one block of kCheckThreads)
// ---------------------------------------------------------------------------

template <typename T>
__device__ T block_exclusive_scan(T v, T* total, T* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        T s = lane < nw ? sh[lane] : T(0);
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) sh[lane] = s;
    }
    __syncthreads();
    const T warp_excl = warp ? sh[warp - 1] : T(0);
    *total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_excl + x - v;
}

// ---------------------------------------------------------------------------
// check / setup kernel: per-graph convergence decision and list rebuild
// ---------------------------------------------------------------------------

__device__ void rebuild_lists(const Dev& d, bool setup) {
    __shared__ long long shl[32];
    __shared__ int32_t shi[32];
    __shared__ int32_t sact_base;
    __shared__ long long vbase;
    if (threadIdx.x == 0) {
        sact_base = 0;
        vbase = 0;
    }
    __syncthreads();
    for (int k = 0; k < kClasses; ++k) {
        const int32_t* srcl = setup ? d.large_cls[k] : d.act[k];
        const int32_t cnt = setup ? d.large_cls_cnt[k] : d.ctl->act_cnt[k];
        int32_t out = 0;
        long long tiles = 0;
        if (threadIdx.x == 0) d.tpre[k][0] = 0;
        for (int32_t base = 0; base < cnt; base += blockDim.x) {
            const int32_t i = base + threadIdx.x;
            int32_t g = -1;
            if (i < cnt) g = srcl[i];
            // the static lists hold every large graph: take the admitted waves'
            const bool keep = g >= 0 && d.state[g] == kActive && (!setup || d.wave[g] <= d.ctl->wave);
            __syncthreads();  // every read of this chunk precedes the writes below
            int32_t kept_total;
            const int32_t pos = block_exclusive_scan<int32_t>(keep ? 1 : 0, &kept_total, shi);
            long long nt = 0;
            if (keep) nt = (d.off_e[g + 1] - d.off_e[g] + kWarpTile - 1) / kWarpTile;
            long long tiles_total;
            const long long tpos = block_exclusive_scan<long long>(nt, &tiles_total, shl);
            if (keep) {
                d.act[k][out + pos] = g;
                d.tpre[k][out + pos + 1] = tiles + tpos + nt;
            }
            // synchronous graphs also need their vertices copied each round
            const bool sk = keep && d.sync[g];
            int32_t s_total;
            const int32_t spos = block_exclusive_scan<int32_t>(sk ? 1 : 0, &s_total, shi);
            long long nv = 0;
            if (sk) nv = (d.off_v[g + 1] - d.off_v[g] + kVTile - 1) / kVTile;
            long long v_total;
            const long long vpos = block_exclusive_scan<long long>(nv, &v_total, shl);
            if (sk) {
                d.sact[sact_base + spos] = g;
                d.vpre[sact_base + spos + 1] = vbase + vpos + nv;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                sact_base += s_total;
                vbase += v_total;
            }
            out += kept_total;
            tiles += tiles_total;
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            d.ctl->act_cnt[k] = out;
            d.ctl->tiles[k] = tiles;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        d.vpre[0] = 0;
        d.ctl->sact_cnt = sact_base;
        d.ctl->vtiles = vbase;
    }
}

// While the active large graphs hold fewer than admit_tiles tiles, admit the
// next wave: its graphs start counting sweeps at round `done`.
__device__ void admit_waves(const Dev& d, int32_t done) {
    __shared__ int admit;
    for (int iter = 0; iter < (1 << 20); ++iter) {  // ends: each pass admits one of finitely many waves
        if (threadIdx.x == 0) {
            long long tiles = 0;
            for (int k = 0; k < kClasses; ++k) tiles += d.ctl->tiles[k];
            admit = tiles < d.ctl->admit_tiles && d.ctl->wave + 1 < d.ctl->n_waves;
            if (admit) d.ctl->wave += 1;
        }
        __syncthreads();
        if (!admit) break;
        const int32_t w = d.ctl->wave;
        for (int32_t g = threadIdx.x; g < d.G; g += blockDim.x)
            if (d.wave[g] == w) d.start[g] = done;
        __syncthreads();
        rebuild_lists(d, true);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kCheckThreads) batch_setup_kernel(Dev d, int32_t max_sweeps, int32_t n_waves,
                                                                   long long admit_tiles) {
    if (threadIdx.x == 0) {
        d.ctl->round = 0;
        d.ctl->wave = 0;
        d.ctl->n_waves = n_waves;
        d.ctl->admit_tiles = admit_tiles;
        d.ctl->max_sweeps = max_sweeps;
        d.ctl->small_next = 0;
        d.ctl->compress_changes = 0;
    }
    for (int32_t g = threadIdx.x; g < d.G; g += blockDim.x) {
        d.flag[g] = 0;
        d.sweeps[g] = 0;
        d.state[g] = kActive;
        d.start[g] = 0;
    }
    __syncthreads();
    rebuild_lists(d, true);
    __syncthreads();
    admit_waves(d, 0);
}

__global__ void __launch_bounds__(kCheckThreads) batch_check_kernel(Dev d, cudaGraphConditionalHandle loop) {
    const int32_t done = d.ctl->round + 1;  // rounds completed including this one
    const int32_t maxs = d.ctl->max_sweeps;
    for (int k = 0; k < kClasses; ++k) {
        const int32_t cnt = d.ctl->act_cnt[k];
        for (int32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
            const int32_t g = d.act[k][i];
            const int32_t round = done - d.start[g];  // sweeps of graph g so far
            if (round % d.c[g] == 0) {
                if (d.flag[g] == 0) {
                    d.state[g] = kConverged;
                    d.sweeps[g] = round;
                    continue;
                }
                d.flag[g] = 0;
            }
            if (round >= maxs) {
                d.state[g] = kStopped;
                d.sweeps[g] = round;
            }
        }
    }
    __syncthreads();
    rebuild_lists(d, false);
    __syncthreads();
    if (threadIdx.x == 0) d.ctl->round = done;
    admit_waves(d, done);
    if (threadIdx.x == 0) {
        int any = 0;
        for (int k = 0; k < kClasses; ++k) any |= d.ctl->act_cnt[k] > 0;
        cudaGraphSetConditional(loop, any ? 1u : 0u);
    }
}

// ---------------------------------------------------------------------------
// large graphs: one sweep of every active graph of one order class
// ---------------------------------------------------------------------------

template <int H>
__global__ void __launch_bounds__(kLargeThreads) batch_round_kernel(Dev d, int cls) {
    const long long total = d.ctl->tiles[cls];
    const int32_t cnt = d.ctl->act_cnt[cls];
    const int32_t done = d.ctl->round;  // rounds completed before this one
    // every warp takes an equal, contiguous range of tiles and walks the
    // active graphs along it (one search per warp, then sequential steps).
    // Walking a graph's sorted edges in order lets labels travel far within
    // one asynchronous sweep: long-diameter graphs converge in fewer sweeps
    // than with warp-strided tiles (measured on the 4,096-graph mix).
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (kLargeThreads / 32);
    const long long wid = (long long)blockIdx.x * (kLargeThreads / 32) + (threadIdx.x >> 5);
    const long long t_begin = total * wid / warps;
    const long long t_end = total * (wid + 1) / warps;
    if (t_begin >= t_end) return;
    int i = find_tile(d.tpre[cls], cnt, t_begin);
    long long t0 = d.tpre[cls][i], t1 = d.tpre[cls][i + 1];
    int32_t g = d.act[cls][i];
    // the flag of graph g is raised once per warp and graph span, not per
    // tile: per-tile stores from every warp to the same word serialise in L2
    bool pending = false;
    auto flush = [&](int32_t gg) {
        const int32_t r = done - d.start[gg];  // sweep index of graph gg in this round
        if (__any_sync(0xffffffffu, pending) && lane == 0 && ((r + 1) % d.c[gg]) == 0) d.flag[gg] = 1;
        pending = false;
    };
    for (long long t = t_begin; t < t_end; ++t) {
        while (t >= t1) {
            flush(g);
            ++i;
            t0 = t1;
            t1 = d.tpre[cls][i + 1];
            g = d.act[cls][i];
        }
        const long long e_begin = d.off_e[g] + (t - t0) * kWarpTile;
        const long long e_end = d.off_e[g + 1];
        int32_t* L = d.L + d.off_v[g];
        const bool sync = d.sync[g] != 0;
        int32_t* Lu = sync ? d.Lu + d.off_v[g] : nullptr;
        const int32_t round = done - d.start[g];  // sweep index of graph g
        // edges of this lane: kEPT consecutive ones, so that edges sharing
        // their w side (the lists are grouped by w after cc_batch_reorder)
        // meet in one thread and the fixed-order operator writes each run of
        // them once (4,096-graph mix, C-2: 84.6 -> 79.2 ms); lanes past the
        // graph's end take the self-loop <0, 0>, which never writes (L[0] = 0
        // always holds)
        int32_t w[kEPT], v[kEPT];
#pragma unroll
        for (int k = 0; k < kEPT; ++k) {
            const long long e = e_begin + kEPT * lane + k;
            const bool ok = e < e_end;
            w[k] = ok ? __ldcs(d.src + e) : 0;
            v[k] = ok ? __ldcs(d.dst + e) : 0;
        }
        bool viol = false;
        if (sync && round == 0) {
            // first iteration of Alg. 1 from L[i] = i: gather-free
#pragma unroll
            for (int k = 0; k < kEPT; ++k) viol |= cc::identity_pair(w[k], v[k], Lu);
        } else if constexpr (H > 0) {
            viol = sync ? cc::mm_fixed<H, true, kEPT>(w, v, L, Lu) : cc::mm_fixed<H, false, kEPT>(w, v, L, Lu);
        } else {
            const int h = d.h[g];
            viol = sync ? cc::mm_runtime_ilp<true, kEPT>(w, v, h, L, Lu) : cc::mm_runtime_ilp<false, kEPT>(w, v, h, L, Lu);
        }
        pending |= viol;
    }
    flush(g);
}

// L = L_u for the vertices of active synchronous large graphs (Alg. 1 copy).
__global__ void __launch_bounds__(256) batch_sync_copy_kernel(Dev d) {
    __shared__ int32_t s_g;
    __shared__ long long s_t0;
    const long long total = d.ctl->vtiles;
    const int32_t cnt = d.ctl->sact_cnt;
    for (long long t = blockIdx.x; t < total; t += gridDim.x) {
        if (threadIdx.x == 0) {
            const int i = find_tile(d.vpre, cnt, t);
            s_g = d.sact[i];
            s_t0 = d.vpre[i];
        }
        __syncthreads();
        const int32_t g = s_g;
        const long long v0 = d.off_v[g] + (t - s_t0) * kVTile;
        const long long v1 = min((long long)d.off_v[g + 1], v0 + kVTile);
        for (long long x = v0 + threadIdx.x; x < v1; x += blockDim.x) d.L[x] = d.Lu[x];
        __syncthreads();
    }
}

// Vertex tiles over all large graphs: L[x] = local id (and L_u for sync).
__global__ void __launch_bounds__(256) batch_large_init_kernel(Dev d) {
    __shared__ int32_t s_g;
    __shared__ long long s_t0;
    for (long long t = blockIdx.x; t < d.large_vtiles; t += gridDim.x) {
        if (threadIdx.x == 0) {
            const int i = find_tile(d.large_vpre, d.n_large, t);
            s_g = d.large_all[i];
            s_t0 = d.large_vpre[i];
        }
        __syncthreads();
        const int32_t g = s_g;
        const long long base = d.off_v[g];
        const long long l0 = (t - s_t0) * kVTile;
        const long long l1 = min(d.off_v[g + 1] - base, l0 + kVTile);
        const bool sync = d.sync[g] != 0;
        for (long long x = l0 + threadIdx.x; x < l1; x += blockDim.x) {
            d.L[base + x] = (int32_t)x;
            if (sync) d.Lu[base + x] = (int32_t)x;
        }
        __syncthreads();
    }
}

// Compress converged large graphs to stars (a no-op at the fixed point; moved
// labels are counted).  Graphs stopped at max_sweeps keep their raw state.
__global__ void __launch_bounds__(256) batch_large_compress_kernel(Dev d) {
    __shared__ int32_t s_g;
    __shared__ long long s_t0;
    unsigned long long changes = 0;
    for (long long t = blockIdx.x; t < d.large_vtiles; t += gridDim.x) {
        if (threadIdx.x == 0) {
            const int i = find_tile(d.large_vpre, d.n_large, t);
            s_g = d.large_all[i];
            s_t0 = d.large_vpre[i];
        }
        __syncthreads();
        const int32_t g = s_g;
        if (d.state[g] == kConverged) {
            int32_t* L = d.L + d.off_v[g];
            const long long n = d.off_v[g + 1] - d.off_v[g];
            const long long l0 = (t - s_t0) * kVTile;
            const long long l1 = min(n, l0 + kVTile);
            for (long long x = l0 + threadIdx.x; x < l1; x += blockDim.x) {
                const int32_t l = L[x];
                int32_t r = l, p = L[r];
                for (int guard = 0; p != r && guard < (1 << 24); ++guard) {
                    r = p;
                    p = L[r];
                }
                if (r != l) {
                    L[x] = r;
                    ++changes;
                }
            }
        }
        __syncthreads();
    }
    for (int o = 16; o > 0; o >>= 1) changes += __shfl_xor_sync(0xffffffffu, changes, o);
    if ((threadIdx.x & 31) == 0 && changes) atomicAdd(&d.ctl->compress_changes, changes);
}

// ---------------------------------------------------------------------------
// small graphs: one CTA solves one graph with labels in shared memory
// ---------------------------------------------------------------------------

// MM^h on shared-memory labels with a run-time order (walk, then rewalk).
template <bool SYNC>
__device__ __forceinline__ bool smem_mm(int32_t w, int32_t v, int h, int32_t* Ls, int32_t* Lus) {
    int32_t ew = w, ev = v;
    const int32_t fw = Ls[w], fv = Ls[v];
    {
        int32_t y = fw;
        for (int j = 1; j < h && y != ew; ++j) {
            ew = y;
            y = Ls[ew];
        }
        ew = y;
        y = fv;
        for (int j = 1; j < h && y != ev; ++j) {
            ev = y;
            y = Ls[ev];
        }
        ev = y;
    }
    const int32_t z = ew < ev ? ew : ev;
    if (fw <= z && fv <= z) return false;
    for (int side = 0; side < 2; ++side) {
        int32_t x = side ? v : w;
        for (int j = 0; j < h; ++j) {
            const int32_t y = Ls[x];
            if (y <= z) break;
            if constexpr (SYNC) {
                if (Lus[x] > z) atomicMin(Lus + x, z);
            } else {
                atomicMin(Ls + x, z);  // never raises a label another thread lowered
            }
            if (y == x) break;
            x = y;
        }
    }
    return true;
}

template <bool SYNC>
__device__ void small_solve(const Dev& d, int32_t g, int32_t* Ls, int32_t* Lus, int ept) {
    const long long base_v = d.off_v[g];
    const int32_t n = (int32_t)(d.off_v[g + 1] - base_v);
    const long long e0 = d.off_e[g];
    const long long m = d.off_e[g + 1] - e0;
    const int h = d.h[g];
    const int32_t cg = d.c[g];
    const int32_t maxs = d.ctl->max_sweeps;
    for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
        Ls[i] = i;
        if (SYNC) Lus[i] = i;
    }
    __syncthreads();
    int32_t sweeps = 0;
    int32_t state = kActive;
    while (state == kActive) {
        int any = 0;
        for (int j = 0; j < cg; ++j) {
            bool viol = false;
            const bool ident = SYNC && sweeps == 0 && j == 0;
            for (long long e = threadIdx.x; e < m; e += (long long)blockDim.x * ept) {
                int32_t w[4], v[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const long long q = e + (long long)k * blockDim.x;
                    const bool ok = k < ept && q < m;
                    w[k] = ok ? __ldcs(d.src + e0 + q) : 0;
                    v[k] = ok ? __ldcs(d.dst + e0 + q) : 0;
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (ident) {
                        if (w[k] != v[k]) {
                            const int32_t lo = min(w[k], v[k]), hi = max(w[k], v[k]);
                            if (Lus[hi] > lo) atomicMin(Lus + hi, lo);
                            viol = true;
                        }
                    } else {
                        viol |= smem_mm<SYNC>(w[k], v[k], h, Ls, Lus);
                    }
                }
            }
            if (SYNC) {
                __syncthreads();
                for (int32_t i = threadIdx.x; i < n; i += blockDim.x) Ls[i] = Lus[i];
            }
            any = __syncthreads_or(viol);
        }
        sweeps += cg;
        if (!any) state = kConverged;
        else if (sweeps >= maxs) state = kStopped;
    }
    if (state == kConverged) {
        for (int32_t x = threadIdx.x; x < n; x += blockDim.x) {
            int32_t r = Ls[x];
            for (int guard = 0; Ls[r] != r && guard < (1 << 24); ++guard) r = Ls[r];
            Ls[x] = r;
        }
        __syncthreads();
    }
    for (int32_t i = threadIdx.x; i < n; i += blockDim.x) d.L[base_v + i] = Ls[i];
    if (threadIdx.x == 0) {
        d.sweeps[g] = sweeps;
        d.state[g] = state;
    }
}

__global__ void batch_small_kernel(Dev d, int ept) {
    extern __shared__ int32_t smem[];
    __shared__ int32_t s_idx;
    for (;;) {
        if (threadIdx.x == 0) s_idx = atomicAdd(&d.ctl->small_next, 1);
        __syncthreads();
        const int32_t idx = s_idx;
        __syncthreads();
        if (idx >= d.n_small) break;
        const int32_t g = d.small_list[idx];
        const int32_t n = (int32_t)(d.off_v[g + 1] - d.off_v[g]);
        if (d.sync[g]) small_solve<true>(d, g, smem, smem + n, ept);
        else small_solve<false>(d, g, smem, nullptr, ept);
        __syncthreads();
    }
}

// Edge ids of every graph must lie in [0, n_g): tiles over all graphs.
__global__ void __launch_bounds__(256) batch_validate_kernel(const int64_t* off_v, const int64_t* off_e,
                                                            const int32_t* src, const int32_t* dst,
                                                            const long long* epre, int32_t G, long long total,
                                                            BatchCtl* ctl) {
    __shared__ int32_t s_g;
    __shared__ long long s_t0;
    unsigned long long bad = 0;
    for (long long t = blockIdx.x; t < total; t += gridDim.x) {
        if (threadIdx.x == 0) {
            int lo = 0, hi = G;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (epre[mid] <= t) lo = mid; else hi = mid;
            }
            s_g = lo;
            s_t0 = epre[lo];
        }
        __syncthreads();
        const int32_t g = s_g;
        const long long n = off_v[g + 1] - off_v[g];
        const long long e0 = off_e[g] + (t - s_t0) * kTile;
        const long long e1 = min((long long)off_e[g + 1], e0 + kTile);
        for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            const int32_t a = __ldcs(src + e), b = __ldcs(dst + e);
            if (a < 0 || a >= n || b < 0 || b >= n) {
                ++bad;
                atomicMin(&ctl->first_bad, (unsigned long long)e);
            }
        }
        __syncthreads();
    }
    for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, o);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(&ctl->bad_count, bad);
}

// Edge tiles over all graphs (epre = tile prefix per graph): the graph of a
// tile and the local edge range it covers.
__device__ __forceinline__ void tile_range(const int64_t* off_e, const long long* epre, int32_t G, long long t,
                                           int32_t* g_out, long long* e0, long long* e1) {
    int lo = 0, hi = G;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (epre[mid] <= t) lo = mid; else hi = mid;
    }
    *g_out = lo;
    *e0 = off_e[lo] + (t - epre[lo]) * kTile;
    *e1 = min((long long)off_e[lo + 1], *e0 + kTile);
}

// degrees of every vertex of the batch, indexed by global vertex id
__global__ void __launch_bounds__(256) batch_degree_kernel(const int64_t* off_v, const int64_t* off_e,
                                                          const int32_t* src, const int32_t* dst,
                                                          const long long* epre, int32_t G, long long total,
                                                          int32_t* deg) {
    __shared__ int32_t s_g;
    __shared__ long long s_e0, s_e1;
    for (long long t = blockIdx.x; t < total; t += gridDim.x) {
        if (threadIdx.x == 0) {
            int32_t g;
            long long e0, e1;
            tile_range(off_e, epre, G, t, &g, &e0, &e1);
            s_g = g;
            s_e0 = e0;
            s_e1 = e1;
        }
        __syncthreads();
        const long long base = off_v[s_g];
        for (long long e = s_e0 + threadIdx.x; e < s_e1; e += blockDim.x) {
            atomicAdd(deg + base + src[e], 1);
            atomicAdd(deg + base + dst[e], 1);
        }
        __syncthreads();
    }
}

// key = global id of the lower-degree endpoint (ties: smaller id), value = the
// other endpoint's local id.  Sorting by key keeps every graph's edges inside
// its own edge range, because graphs own consecutive vertex ranges.
__global__ void __launch_bounds__(256) batch_orient_kernel(const int64_t* off_v, const int64_t* off_e,
                                                          const int32_t* src, const int32_t* dst,
                                                          const long long* epre, int32_t G, long long total,
                                                          const int32_t* deg, uint32_t* key, uint32_t* val) {
    __shared__ int32_t s_g;
    __shared__ long long s_e0, s_e1;
    for (long long t = blockIdx.x; t < total; t += gridDim.x) {
        if (threadIdx.x == 0) {
            int32_t g;
            long long e0, e1;
            tile_range(off_e, epre, G, t, &g, &e0, &e1);
            s_g = g;
            s_e0 = e0;
            s_e1 = e1;
        }
        __syncthreads();
        const long long base = off_v[s_g];
        for (long long e = s_e0 + threadIdx.x; e < s_e1; e += blockDim.x) {
            const int32_t a = src[e], b = dst[e];
            const int32_t da = deg[base + a], db = deg[base + b];
            const bool swap = db < da || (db == da && b < a);
            key[e] = (uint32_t)(base + (swap ? b : a));
            val[e] = (uint32_t)(swap ? a : b);
        }
        __syncthreads();
    }
}

// key (global id) -> local id of the graph that owns edge e
__global__ void __launch_bounds__(256) batch_localize_kernel(const int64_t* off_v, const int64_t* off_e,
                                                            const long long* epre, int32_t G, long long total,
                                                            uint32_t* key) {
    __shared__ int32_t s_g;
    __shared__ long long s_e0, s_e1;
    for (long long t = blockIdx.x; t < total; t += gridDim.x) {
        if (threadIdx.x == 0) {
            int32_t g;
            long long e0, e1;
            tile_range(off_e, epre, G, t, &g, &e0, &e1);
            s_g = g;
            s_e0 = e0;
            s_e1 = e1;
        }
        __syncthreads();
        const long long base = off_v[s_g];
        for (long long e = s_e0 + threadIdx.x; e < s_e1; e += blockDim.x) key[e] = (uint32_t)((long long)key[e] - base);
        __syncthreads();
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct BatchLoop {
    int32_t* L = nullptr;
    unsigned long long sched_hash = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

struct cc_batch_plan {
    int32_t G = 0;
    std::vector<int64_t> off_v, off_e;
    int64_t total_n = 0, total_m = 0;
    const int32_t* src = nullptr;
    const int32_t* dst = nullptr;
    bool own_edges = false;  // after cc_batch_reorder
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    cudaStream_t aux[kClasses - 1] = {};  // capture branches for concurrent class kernels
    cudaEvent_t fork = nullptr, join[kClasses] = {};
    // device buffers
    int64_t* d_off_v = nullptr;
    int64_t* d_off_e = nullptr;
    int32_t* d_pg = nullptr;  // per-graph block: h, sync, c, flag, sweeps, state
    int32_t* d_lists = nullptr;
    long long* d_pre = nullptr;
    BatchCtl* d_ctl = nullptr;
    BatchCtl* h_ctl = nullptr;
    int32_t* d_Lu = nullptr;
    // current schedule (host copies)
    std::vector<int32_t> h_h, h_sync, h_c;
    // tuning
    int small_budget = 0;  // bytes of shared memory per small-graph CTA
    int small_threads = 512;
    int small_ept = 4;
    bool tuned = false;
    std::vector<BatchLoop> loops;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int sms = 0;
    cc::SchedCtx* sched = nullptr;  // CC_ORDER_AUTO buffers
};

namespace {

#define BCUDA(expr)                                                                  \
    do {                                                                             \
        cudaError_t e_ = (expr);                                                     \
        if (e_ != cudaSuccess) return cc::cuda_fail(e_, #expr, __FILE__, __LINE__); \
    } while (0)

void destroy_batch(cc_batch_plan* b) {
    if (!b) return;
    cc::sched_ctx_free(b->sched);
    for (auto& l : b->loops) {
        if (l.exec) cudaGraphExecDestroy(l.exec);
        if (l.graph) cudaGraphDestroy(l.graph);
    }
    if (b->own_edges) {
        cudaFree(const_cast<int32_t*>(b->src));
        cudaFree(const_cast<int32_t*>(b->dst));
    }
    cudaFree(b->d_off_v);
    cudaFree(b->d_off_e);
    cudaFree(b->d_pg);
    cudaFree(b->d_lists);
    cudaFree(b->d_pre);
    cudaFree(b->d_ctl);
    cudaFree(b->d_Lu);
    if (b->h_ctl) cudaFreeHost(b->h_ctl);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (auto& a : b->aux)
        if (a) cudaStreamDestroy(a);
    if (b->fork) cudaEventDestroy(b->fork);
    for (auto& j : b->join)
        if (j) cudaEventDestroy(j);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    delete b;
}

// Sizes of the per-graph and list regions.
struct Layout {
    size_t pg_ints;     // 8 * G
    size_t list_ints;   // small list + 4 static class lists + 4 active + sact + large_all
    size_t pre_longs;   // 4 tile prefixes + vpre + large_vpre + edge-tile prefix (G+1 each)
};

Layout layout_for(int32_t G) {
    Layout l;
    l.pg_ints = 8ull * G;
    l.list_ints = 12ull * (G + 1);
    l.pre_longs = 7ull * (G + 1);
    return l;
}

// Is graph g solved in shared memory under this budget?
bool is_small(const cc_batch_plan* b, int32_t g, int budget, bool sync) {
    const int64_t n = b->off_v[g + 1] - b->off_v[g];
    const int64_t bytes = n * (sync ? 8 : 4);
    return bytes <= budget;
}

Dev make_dev(const cc_batch_plan* b, int32_t* L, std::vector<int32_t>& lists_h, std::vector<long long>& pre_h,
             int32_t* counts_small, int32_t cls_cnt[kClasses], int32_t* n_large, long long* large_vtiles,
             std::vector<int32_t>& wave_h, int32_t* n_waves) {
    const int32_t G = b->G;
    Dev d = {};
    d.G = G;
    d.off_v = b->d_off_v;
    d.off_e = b->d_off_e;
    d.src = b->src;
    d.dst = b->dst;
    d.L = L;
    d.Lu = b->d_Lu;
    d.h = b->d_pg;
    d.sync = b->d_pg + G;
    d.c = b->d_pg + 2 * G;
    d.flag = b->d_pg + 3 * G;
    d.sweeps = b->d_pg + 4 * G;
    d.state = b->d_pg + 5 * G;
    d.wave = b->d_pg + 6 * G;
    d.start = b->d_pg + 7 * G;
    d.ctl = b->d_ctl;

    // host-side classification (lists are uploaded by the caller)
    const size_t S = G + 1;
    lists_h.assign(12 * S, 0);
    // slots 0-5 of the prefix buffer (slot 6 holds the edge-tile prefix of
    // all graphs, written once by cc_batch_init and never overwritten)
    pre_h.assign(6 * S, 0);
    std::vector<int32_t> small, large_all, cls[kClasses];
    for (int32_t g = 0; g < G; ++g) {
        if (is_small(b, g, b->small_budget, b->h_sync[g] != 0)) small.push_back(g);
        else {
            large_all.push_back(g);
            cls[order_class(b->h_h[g])].push_back(g);
        }
    }
    // waves: large graphs in order of mean degree (sparse, long-diameter
    // graphs -- which need the most sweeps -- share waves), cut whenever the
    // wave's label bytes would exceed kWaveBytes
    {
        std::vector<int32_t> byd = large_all;
        auto deg = [&](int32_t g) {
            const double n = (double)(b->off_v[g + 1] - b->off_v[g]);
            return n > 0 ? (double)(b->off_e[g + 1] - b->off_e[g]) / n : 0.0;
        };
        std::stable_sort(byd.begin(), byd.end(), [&](int32_t x, int32_t y) { return deg(x) < deg(y); });
        wave_h.assign(G, 0);
        int32_t w = 0;
        long long bytes = 0;
        for (int32_t g : byd) {
            const long long nb = (b->off_v[g + 1] - b->off_v[g]) * (b->h_sync[g] ? 8ll : 4ll);
            if (bytes > 0 && bytes + nb > kWaveBytes) {
                ++w;
                bytes = 0;
            }
            wave_h[g] = w;
            bytes += nb;
        }
        *n_waves = byd.empty() ? 0 : w + 1;
    }
    // largest small graphs first (longest-processing-time order)
    std::stable_sort(small.begin(), small.end(), [&](int32_t x, int32_t y) {
        return (b->off_e[x + 1] - b->off_e[x]) > (b->off_e[y + 1] - b->off_e[y]);
    });
    int32_t* D = b->d_lists;
    auto put = [&](int slot, const std::vector<int32_t>& v) {
        std::copy(v.begin(), v.end(), lists_h.begin() + slot * S);
        return D + slot * S;
    };
    d.small_list = put(0, small);
    d.n_small = (int32_t)small.size();
    for (int k = 0; k < kClasses; ++k) {
        d.large_cls[k] = put(1 + k, cls[k]);
        d.large_cls_cnt[k] = (int32_t)cls[k].size();
        cls_cnt[k] = d.large_cls_cnt[k];
        d.act[k] = D + (5 + k) * S;
    }
    d.sact = D + 9 * S;
    d.large_all = put(10, large_all);
    d.n_large = (int32_t)large_all.size();
    long long* P = b->d_pre;
    for (int k = 0; k < kClasses; ++k) d.tpre[k] = P + k * S;
    d.vpre = P + 4 * S;
    long long vt = 0;
    pre_h[5 * S] = 0;
    for (size_t i = 0; i < large_all.size(); ++i) {
        const int32_t g = large_all[i];
        vt += (b->off_v[g + 1] - b->off_v[g] + kVTile - 1) / kVTile;
        pre_h[5 * S + i + 1] = vt;
    }
    d.large_vpre = P + 5 * S;
    d.large_vtiles = vt;
    *counts_small = d.n_small;
    *n_large = d.n_large;
    *large_vtiles = vt;
    return d;
}

// Largest dynamic shared-memory size the small-graph kernel can be given
// (the opt-in per-block limit minus its static shared memory).
int small_kernel_max_dynamic() {
    static int v = -1;
    if (v < 0) {
        int max_smem = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes attr;
        if (cudaFuncGetAttributes(&attr, batch_small_kernel) != cudaSuccess) attr.sharedSizeBytes = 1024;
        v = max_smem - (int)attr.sharedSizeBytes;
        if (v < 0) v = 0;
    }
    return v;
}

int persistent_grid(const void* fn, int threads, size_t smem) {
    return cc::persistent_blocks(fn, threads, smem);
}

cc_status build_loop(cc_batch_plan* b, const Dev& d, BatchLoop* out) {
    BatchLoop l;
    BCUDA(cudaGraphCreate(&l.graph, 0));
    cudaGraphConditionalHandle handle;
    cudaError_t e = cudaGraphConditionalHandleCreate(&handle, l.graph, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams p = {};
    cudaGraphNode_t node;
    if (e == cudaSuccess) {
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = handle;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        e = cudaGraphAddNode(&node, l.graph, nullptr, nullptr, 0, &p);
    }
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(b->cap, p.conditional.phGraph_out[0], nullptr,
                                                            nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const int g1 = persistent_grid(reinterpret_cast<const void*>(batch_round_kernel<1>), kLargeThreads, 0);
        const int g2 = persistent_grid(reinterpret_cast<const void*>(batch_round_kernel<2>), kLargeThreads, 0);
        const int g4 = persistent_grid(reinterpret_cast<const void*>(batch_round_kernel<4>), kLargeThreads, 0);
        const int g0 = persistent_grid(reinterpret_cast<const void*>(batch_round_kernel<0>), kLargeThreads, 0);
        // the order classes touch disjoint graphs: their kernels are parallel
        // branches of the round (joined before the copy and the check)
        cudaStream_t branch[kClasses];
        int used = 0;
        cudaError_t eb = cudaEventRecord(b->fork, b->cap);
        auto next_stream = [&]() {
            cudaStream_t st = used == 0 ? b->cap : b->aux[used - 1];
            if (used > 0 && eb == cudaSuccess) eb = cudaStreamWaitEvent(st, b->fork, 0);
            branch[used++] = st;
            return st;
        };
        if (d.large_cls_cnt[0]) batch_round_kernel<1><<<g1, kLargeThreads, 0, next_stream()>>>(d, 0);
        if (d.large_cls_cnt[1]) batch_round_kernel<2><<<g2, kLargeThreads, 0, next_stream()>>>(d, 1);
        if (d.large_cls_cnt[2]) batch_round_kernel<4><<<g4, kLargeThreads, 0, next_stream()>>>(d, 2);
        if (d.large_cls_cnt[3]) batch_round_kernel<0><<<g0, kLargeThreads, 0, next_stream()>>>(d, 3);
        for (int i = 1; i < used && eb == cudaSuccess; ++i) {
            eb = cudaEventRecord(b->join[i], branch[i]);
            if (eb == cudaSuccess) eb = cudaStreamWaitEvent(b->cap, b->join[i], 0);
        }
        if (d.Lu) {
            const int gc = persistent_grid(reinterpret_cast<const void*>(batch_sync_copy_kernel), 256, 0);
            batch_sync_copy_kernel<<<gc, 256, 0, b->cap>>>(d);
        }
        batch_check_kernel<<<1, kCheckThreads, 0, b->cap>>>(d, handle);
        cudaError_t ek = cudaGetLastError();
        if (ek == cudaSuccess) ek = eb;
        cudaGraph_t captured = nullptr;
        e = cudaStreamEndCapture(b->cap, &captured);
        if (ek != cudaSuccess) e = ek;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&l.exec, l.graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(l.graph);
        return cc::cuda_fail(e, "building the batch round graph", __FILE__, __LINE__);
    }
    *out = l;
    return CC_OK;
}

unsigned long long sched_hash(const cc_batch_plan* b, int32_t* L) {
    unsigned long long hsh = 1469598103934665603ull ^ (unsigned long long)(uintptr_t)L;
    auto mix = [&](int32_t x) { hsh = (hsh ^ (unsigned)x) * 1099511628211ull; };
    for (int32_t g = 0; g < b->G; ++g) {
        mix(b->h_h[g]);
        mix(b->h_sync[g]);
        mix(b->h_c[g]);
    }
    mix(b->small_budget);
    mix(b->small_threads);
    mix(b->small_ept);
    return hsh;
}

}  // namespace

namespace cc {

// Runs one solve of the batch with the schedule in b->h_h/h_sync/h_c.
cc_status batch_solve(cc_batch_plan* b, int32_t max_sweeps, int32_t* labels_out, int32_t* sweeps_out,
                      double* solve_ms) {
    NvtxRange range("cc_batch_run");
    const int32_t G = b->G;
    cudaStream_t s = b->stream;
    const bool any_sync = std::any_of(b->h_sync.begin(), b->h_sync.end(), [](int32_t x) { return x != 0; });
    if (any_sync && !b->d_Lu && b->total_n > 0) BCUDA(cudaMalloc(&b->d_Lu, b->total_n * sizeof(int32_t)));

    std::vector<int32_t> lists_h;
    std::vector<long long> pre_h;
    int32_t n_small = 0, cls_cnt[kClasses], n_large = 0, n_waves = 0;
    long long large_vtiles = 0;
    std::vector<int32_t> wave_h;
    Dev d = make_dev(b, labels_out, lists_h, pre_h, &n_small, cls_cnt, &n_large, &large_vtiles, wave_h, &n_waves);
    if (!any_sync) d.Lu = nullptr;

    // schedule and static lists to the device
    std::vector<int32_t> pg(3 * (size_t)G);
    std::copy(b->h_h.begin(), b->h_h.end(), pg.begin());
    std::copy(b->h_sync.begin(), b->h_sync.end(), pg.begin() + G);
    std::copy(b->h_c.begin(), b->h_c.end(), pg.begin() + 2 * G);
    BCUDA(cudaMemcpyAsync(b->d_pg, pg.data(), pg.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    BCUDA(cudaMemcpyAsync(b->d_pg + 6 * (size_t)G, wave_h.data(), (size_t)G * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    BCUDA(cudaMemcpyAsync(b->d_lists, lists_h.data(), lists_h.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    BCUDA(cudaMemcpyAsync(b->d_pre, pre_h.data(), pre_h.size() * sizeof(long long), cudaMemcpyHostToDevice, s));

    BatchLoop* loop = nullptr;
    if (n_large > 0) {
        const unsigned long long hs = sched_hash(b, labels_out);
        for (auto& l : b->loops)
            if (l.L == labels_out && l.sched_hash == hs) loop = &l;
        if (!loop) {
            if (b->loops.size() >= 4) {
                cudaGraphExecDestroy(b->loops.front().exec);
                cudaGraphDestroy(b->loops.front().graph);
                b->loops.erase(b->loops.begin());
            }
            BatchLoop nl;
            cc_status st = build_loop(b, d, &nl);
            if (st != CC_OK) return st;
            nl.L = labels_out;
            nl.sched_hash = hs;
            b->loops.push_back(nl);
            loop = &b->loops.back();
        }
    }

    BCUDA(cudaEventRecord(b->ev0, s));
    // admit waves while the active large graphs hold fewer tiles than 8 per
    // warp of the round kernels' persistent grid
    const long long admit_tiles =
        8ll * (kLargeThreads / 32) *
        persistent_grid(reinterpret_cast<const void*>(batch_round_kernel<2>), kLargeThreads, 0);
    batch_setup_kernel<<<1, kCheckThreads, 0, s>>>(d, max_sweeps, n_waves, admit_tiles);
    BCUDA(cudaGetLastError());
    if (n_small > 0) {
        const size_t smem = (size_t)b->small_budget;
        auto k = batch_small_kernel;
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, b->small_threads, smem) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        const int grid = std::min<int>(n_small, per_sm * cc::device_sms());
        k<<<grid, b->small_threads, smem, s>>>(d, b->small_ept);
        BCUDA(cudaGetLastError());
    }
    if (n_large > 0) {
        const int gi = persistent_grid(reinterpret_cast<const void*>(batch_large_init_kernel), 256, 0);
        batch_large_init_kernel<<<gi, 256, 0, s>>>(d);
        BCUDA(cudaGetLastError());
        BCUDA(cudaGraphLaunch(loop->exec, s));
        const int gc = persistent_grid(reinterpret_cast<const void*>(batch_large_compress_kernel), 256, 0);
        batch_large_compress_kernel<<<gc, 256, 0, s>>>(d);
        BCUDA(cudaGetLastError());
    }
    BCUDA(cudaEventRecord(b->ev1, s));
    std::vector<int32_t> tail(2 * (size_t)G);
    BCUDA(cudaMemcpyAsync(tail.data(), d.sweeps, 2 * (size_t)G * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    BCUDA(cudaMemcpyAsync(b->h_ctl, b->d_ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, s));
    BCUDA(cudaStreamSynchronize(s));
    if (solve_ms) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, b->ev0, b->ev1);
        *solve_ms = ms;
    }
    if (sweeps_out) std::memcpy(sweeps_out, tail.data(), (size_t)G * sizeof(int32_t));
    if (b->h_ctl->compress_changes)
        return set_error(CC_ECUDA, "cc_batch_run: a converged graph was not a set of stars (%llu labels moved)",
                         b->h_ctl->compress_changes);
    for (int32_t g = 0; g < G; ++g)
        if (tail[G + g] != kConverged)
            return set_error(CC_ENOTCONVERGED, "cc_batch_run: graph %d not converged within %d sweeps", g, max_sweeps);
    return CC_OK;
}

int32_t batch_graph_count(const cc_batch_plan* b) { return b->G; }
const int64_t* batch_off_v(const cc_batch_plan* b) { return b->off_v.data(); }
const int64_t* batch_off_e(const cc_batch_plan* b) { return b->off_e.data(); }
const int32_t* batch_src(const cc_batch_plan* b) { return b->src; }
const int32_t* batch_dst(const cc_batch_plan* b) { return b->dst; }
cudaStream_t batch_stream(const cc_batch_plan* b) { return b->stream; }
SchedCtx** batch_sched_slot(cc_batch_plan* b) { return &b->sched; }
void batch_set_schedule(cc_batch_plan* b, const int32_t* h, const int32_t* sync, const int32_t* c) {
    std::copy(h, h + b->G, b->h_h.begin());
    std::copy(sync, sync + b->G, b->h_sync.begin());
    std::copy(c, c + b->G, b->h_c.begin());
}

}  // namespace cc

// ---------------------------------------------------------------------------
// autotuner: shared-memory budget, CTA size and edges per thread of the
// small-graph kernel, timed on the batch itself and cached by a size key
// ---------------------------------------------------------------------------

namespace {

struct Tuning {
    int budget, threads, ept;
};

std::mutex g_tune_mu;
std::map<unsigned long long, Tuning> g_tune_cache;

unsigned long long size_key(const cc_batch_plan* b) {
    // histogram of log2(n) and log2(m/n) classes, hashed
    unsigned long long hsh = 1469598103934665603ull;
    int hist[64] = {0};
    for (int32_t g = 0; g < b->G; ++g) {
        const int64_t n = std::max<int64_t>(1, b->off_v[g + 1] - b->off_v[g]);
        const int64_t m = b->off_e[g + 1] - b->off_e[g];
        int ln = 0;
        while ((1ll << ln) < n && ln < 40) ++ln;
        const int dm = m / n >= 8 ? 2 : (m / n >= 2 ? 1 : 0);
        hist[(ln / 2) * 3 % 63 + dm]++;
    }
    for (int i = 0; i < 64; ++i) {
        int q = 0;
        while ((1 << q) <= hist[i] && q < 30) ++q;  // bucket counts by powers of two
        hsh = (hsh ^ (unsigned long long)(i * 31 + q)) * 1099511628211ull;
    }
    return hsh;
}

}  // namespace

namespace cc {

cc_status batch_autotune(cc_batch_plan* b, int force) {
    const unsigned long long key = size_key(b);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end() && !force) {
            b->small_budget = it->second.budget;
            b->small_threads = it->second.threads;
            b->small_ept = it->second.ept;
            b->tuned = true;
            return CC_OK;
        }
    }
    const int max_smem = small_kernel_max_dynamic();
    int32_t* L = nullptr;
    BCUDA(cudaMalloc(&L, std::max<int64_t>(1, b->total_n) * sizeof(int32_t)));
    std::vector<int32_t> sw(b->G);
    Tuning best = {b->small_budget, b->small_threads, b->small_ept};
    double best_ms = 1e30;
    const int budgets[] = {32 * 1024, 64 * 1024, 112 * 1024, max_smem};
    const int threads[] = {256, 512, 1024};
    const int epts[] = {2, 4};
    cc_status st = CC_OK;
    for (int bu : budgets) {
        if (bu > max_smem) continue;
        for (int th : threads)
            for (int ep : epts) {
                b->small_budget = bu;
                b->small_threads = th;
                b->small_ept = ep;
                double ms = 0;
                st = batch_solve(b, 1 << 20, L, sw.data(), &ms);
                if (st != CC_OK && st != CC_ENOTCONVERGED) {
                    cudaFree(L);
                    return st;
                }
                if (ms < best_ms) {
                    best_ms = ms;
                    best = {bu, th, ep};
                }
            }
    }
    cudaFree(L);
    b->small_budget = best.budget;
    b->small_threads = best.threads;
    b->small_ept = best.ept;
    b->tuned = true;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = best;
    return CC_OK;
}

}  // namespace cc

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" cc_status cc_batch_init(cc_batch_plan** out, int32_t n_graphs, const int64_t* vtx_off,
                                   const int64_t* edge_off, const int32_t* src, const int32_t* dst,
                                   int autotune, void* cuda_stream) {
    if (!out) return cc::set_error(CC_EINVAL, "cc_batch_init: out is NULL");
    *out = nullptr;
    if (n_graphs < 0) return cc::set_error(CC_EINVAL, "cc_batch_init: n_graphs < 0");
    if (n_graphs > 0 && (!vtx_off || !edge_off)) return cc::set_error(CC_EINVAL, "cc_batch_init: offsets are NULL");
    for (int32_t g = 0; g < n_graphs; ++g) {
        if (vtx_off[g + 1] < vtx_off[g] || edge_off[g + 1] < edge_off[g])
            return cc::set_error(CC_EINVAL, "cc_batch_init: offsets decrease at graph %d", g);
        if (vtx_off[g + 1] - vtx_off[g] > 0x7fffffffLL)
            return cc::set_error(CC_EINVAL, "cc_batch_init: graph %d has >= 2^31 vertices", g);
    }
    if (n_graphs > 0 && (vtx_off[0] != 0 || edge_off[0] != 0))
        return cc::set_error(CC_EINVAL, "cc_batch_init: offsets must start at 0");
    const int64_t total_m = n_graphs ? edge_off[n_graphs] : 0;
    if (total_m > 0 && (!src || !dst)) return cc::set_error(CC_EINVAL, "cc_batch_init: edge arrays are NULL");

    cc_batch_plan* b = new (std::nothrow) cc_batch_plan();
    if (!b) return cc::set_error(CC_ENOMEM, "cc_batch_init: host allocation failed");
    auto fail = [&](cc_status st) {
        destroy_batch(b);
        return st;
    };
    b->G = n_graphs;
    b->off_v.assign(vtx_off, vtx_off + n_graphs + 1);
    b->off_e.assign(edge_off, edge_off + n_graphs + 1);
    if (n_graphs == 0) {
        b->off_v.assign(1, 0);
        b->off_e.assign(1, 0);
    }
    b->total_n = b->off_v.back();
    b->total_m = b->off_e.back();
    b->src = src;
    b->dst = dst;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    b->h_h.assign(n_graphs, 2);
    b->h_sync.assign(n_graphs, 0);
    b->h_c.assign(n_graphs, 1);
    const int max_smem = small_kernel_max_dynamic();
    b->small_budget = std::min(112 * 1024, max_smem);
    const Layout lay = layout_for(std::max(n_graphs, 1));
    cudaError_t e = cudaMalloc(&b->d_off_v, (n_graphs + 1) * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_off_e, (n_graphs + 1) * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_pg, lay.pg_ints * sizeof(int32_t) + 16);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_lists, lay.list_ints * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_pre, lay.pre_longs * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_ctl, sizeof(BatchCtl));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_ctl, sizeof(BatchCtl));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    for (auto& a : b->aux)
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (auto& j : b->join)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev1);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(batch_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e != cudaSuccess) return fail(cc::cuda_fail(e, "cc_batch_init allocation", __FILE__, __LINE__));
    cudaStream_t s = b->stream;
    e = cudaMemcpyAsync(b->d_off_v, b->off_v.data(), b->off_v.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_off_e, b->off_e.data(), b->off_e.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(cc::cuda_fail(e, "cc_batch_init upload", __FILE__, __LINE__));
    // validate every edge id against its own graph
    if (b->total_m > 0) {
        std::vector<long long> epre(n_graphs + 1, 0);
        for (int32_t g = 0; g < n_graphs; ++g)
            epre[g + 1] = epre[g] + (b->off_e[g + 1] - b->off_e[g] + kTile - 1) / kTile;
        long long* d_epre = b->d_pre + 6ull * (n_graphs + 1);
        BatchCtl zero = {};
        zero.first_bad = ~0ull;
        e = cudaMemcpyAsync(d_epre, epre.data(), epre.size() * sizeof(long long), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_ctl, &zero, sizeof zero, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) {
            const int grid = persistent_grid(reinterpret_cast<const void*>(batch_validate_kernel), 256, 0);
            batch_validate_kernel<<<grid, 256, 0, s>>>(b->d_off_v, b->d_off_e, src, dst, d_epre, n_graphs,
                                                       epre[n_graphs], b->d_ctl);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_ctl, b->d_ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(cc::cuda_fail(e, "cc_batch_init validation", __FILE__, __LINE__));
        if (b->h_ctl->bad_count)
            return fail(cc::set_error(CC_EIDRANGE, "cc_batch_init: %llu endpoints outside their graph's [0, n) (first at edge %llu)",
                                      b->h_ctl->bad_count, b->h_ctl->first_bad));
    } else {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(cc::cuda_fail(e, "cc_batch_init", __FILE__, __LINE__));
    }
    if (autotune && n_graphs > 0) {
        cc_status st = cc::batch_autotune(b, autotune > 1);
        if (st != CC_OK) return fail(st);
    }
    *out = b;
    return CC_OK;
}

extern "C" cc_status cc_batch_run(cc_batch_plan* b, int order, int mode, int check_interval, int32_t max_sweeps,
                                  int32_t* labels_out, int32_t* sweeps_out, double* solve_ms) {
    if (!b) return cc::set_error(CC_EINVAL, "cc_batch_run: batch is NULL");
    if (b->total_n > 0 && !labels_out) return cc::set_error(CC_EINVAL, "cc_batch_run: labels_out is NULL");
    if (max_sweeps < 1) return cc::set_error(CC_EINVAL, "cc_batch_run: max_sweeps must be >= 1");
    if (order == CC_ORDER_AUTO) {
        cc_status st = cc::batch_resolve_schedule(b, mode, check_interval);
        if (st != CC_OK) return st;
    } else {
        if (order < 0 || order > CC_MAX_ORDER) return cc::set_error(CC_EINVAL, "cc_batch_run: bad order");
        if (mode != CC_SYNC && mode != CC_ASYNC) return cc::set_error(CC_EINVAL, "cc_batch_run: bad mode");
        if (check_interval < 1 || check_interval > 64) return cc::set_error(CC_EINVAL, "cc_batch_run: check_interval must be 1..64");
        const int h = order == CC_ORDER_FULL ? cc::kFullChainHops : order;
        std::fill(b->h_h.begin(), b->h_h.end(), h);
        std::fill(b->h_sync.begin(), b->h_sync.end(), mode == CC_SYNC ? 1 : 0);
        std::fill(b->h_c.begin(), b->h_c.end(), check_interval);
    }
    if (b->G == 0) {
        if (solve_ms) *solve_ms = 0;
        return CC_OK;
    }
    return cc::batch_solve(b, max_sweeps, labels_out, sweeps_out, solve_ms);
}

extern "C" cc_status cc_batch_set_schedule(cc_batch_plan* b, const int32_t* order, const int32_t* mode,
                                           const int32_t* check_interval) {
    if (!b || !order || !mode || !check_interval) return cc::set_error(CC_EINVAL, "cc_batch_set_schedule: NULL argument");
    for (int32_t g = 0; g < b->G; ++g) {
        if (order[g] < 0 || order[g] > CC_MAX_ORDER || (mode[g] != CC_SYNC && mode[g] != CC_ASYNC) ||
            check_interval[g] < 1 || check_interval[g] > 64)
            return cc::set_error(CC_EINVAL, "cc_batch_set_schedule: bad schedule for graph %d", g);
        b->h_h[g] = order[g] == CC_ORDER_FULL ? cc::kFullChainHops : order[g];
        b->h_sync[g] = mode[g] == CC_SYNC;
        b->h_c[g] = check_interval[g];
    }
    return CC_OK;
}

extern "C" cc_status cc_batch_run_scheduled(cc_batch_plan* b, int32_t max_sweeps, int32_t* labels_out,
                                            int32_t* sweeps_out, double* solve_ms) {
    if (!b) return cc::set_error(CC_EINVAL, "cc_batch_run_scheduled: batch is NULL");
    if (b->total_n > 0 && !labels_out) return cc::set_error(CC_EINVAL, "cc_batch_run_scheduled: labels_out is NULL");
    if (max_sweeps < 1) return cc::set_error(CC_EINVAL, "cc_batch_run_scheduled: max_sweeps must be >= 1");
    if (b->G == 0) return CC_OK;
    return cc::batch_solve(b, max_sweeps, labels_out, sweeps_out, solve_ms);
}

extern "C" cc_status cc_batch_tuning(const cc_batch_plan* b, int32_t* smem_budget, int32_t* threads, int32_t* ept) {
    if (!b) return cc::set_error(CC_EINVAL, "cc_batch_tuning: batch is NULL");
    if (smem_budget) *smem_budget = b->small_budget;
    if (threads) *threads = b->small_threads;
    if (ept) *ept = b->small_ept;
    return CC_OK;
}

extern "C" cc_status cc_batch_set_tuning(cc_batch_plan* b, int32_t smem_budget, int32_t threads, int32_t ept) {
    if (!b) return cc::set_error(CC_EINVAL, "cc_batch_set_tuning: batch is NULL");
    const int max_smem = small_kernel_max_dynamic();
    if (smem_budget < 0 || smem_budget > max_smem || (threads != 256 && threads != 512 && threads != 1024) ||
        ept < 1 || ept > 4)
        return cc::set_error(CC_EINVAL, "cc_batch_set_tuning: budget 0..%d bytes, threads 256/512/1024, ept 1..4", max_smem);
    b->small_budget = smem_budget;
    b->small_threads = threads;
    b->small_ept = ept;
    return CC_OK;
}

extern "C" cc_status cc_batch_reorder(cc_batch_plan* b) {
    cc::NvtxRange range("cc_batch_reorder");
    if (!b) return cc::set_error(CC_EINVAL, "cc_batch_reorder: batch is NULL");
    if (b->total_m == 0) return CC_OK;
    if (b->total_n >= (1ll << 32)) return cc::set_error(CC_EINVAL, "cc_batch_reorder: batches of >= 2^32 vertices are not supported");
    const int32_t G = b->G;
    const long long m = b->total_m;
    cudaStream_t s = b->stream;
    // edge-tile prefix of all graphs, rebuilt from the host offsets
    long long* d_epre = b->d_pre + 6ull * (G + 1);
    std::vector<long long> epre(G + 1, 0);
    for (int32_t g = 0; g < G; ++g) epre[g + 1] = epre[g] + (b->off_e[g + 1] - b->off_e[g] + kTile - 1) / kTile;
    const long long total_tiles = epre[G];
    {
        cudaError_t e0 = cudaMemcpyAsync(d_epre, epre.data(), (G + 1) * sizeof(long long), cudaMemcpyHostToDevice, s);
        if (e0 != cudaSuccess) return cc::cuda_fail(e0, "cc_batch_reorder", __FILE__, __LINE__);
    }
    int bits = 1;
    while (bits < 32 && (1ll << bits) < b->total_n) ++bits;
    cc_status st = CC_OK;
    uint32_t *k_in = nullptr, *v_in = nullptr, *k_out = nullptr, *v_out = nullptr;
    int32_t* deg = nullptr;
    void* tmp = nullptr;
    size_t tmp_bytes = 0;
    const int grid = cc::device_sms() * 8;
    cudaError_t e = cudaMalloc(&k_in, (size_t)m * 4);
    if (e == cudaSuccess) e = cudaMalloc(&v_in, (size_t)m * 4);
    if (e == cudaSuccess) e = cudaMalloc(&k_out, (size_t)m * 4);
    if (e == cudaSuccess) e = cudaMalloc(&v_out, (size_t)m * 4);
    if (e == cudaSuccess) e = cudaMalloc(&deg, (size_t)b->total_n * 4);
    if (e == cudaSuccess) e = cudaMemsetAsync(deg, 0, (size_t)b->total_n * 4, s);
    if (e == cudaSuccess) {
        batch_degree_kernel<<<grid, 256, 0, s>>>(b->d_off_v, b->d_off_e, b->src, b->dst, d_epre, G, total_tiles, deg);
        batch_orient_kernel<<<grid, 256, 0, s>>>(b->d_off_v, b->d_off_e, b->src, b->dst, d_epre, G, total_tiles, deg,
                                                 k_in, v_in);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, k_in, k_out, v_in, v_out, m, 0, bits, s);
    if (e == cudaSuccess) e = cudaMalloc(&tmp, tmp_bytes);
    if (e == cudaSuccess) e = cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, k_in, k_out, v_in, v_out, m, 0, bits, s);
    if (e == cudaSuccess) {
        batch_localize_kernel<<<grid, 256, 0, s>>>(b->d_off_v, b->d_off_e, d_epre, G, total_tiles, k_out);
        e = cudaGetLastError();
    }
    // every reordered id must still lie in its graph's [0, n) before any
    // sweep gathers with it
    if (e == cudaSuccess) {
        BatchCtl zero = {};
        zero.first_bad = ~0ull;
        e = cudaMemcpyAsync(b->d_ctl, &zero, sizeof zero, cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) {
        const int gv = persistent_grid(reinterpret_cast<const void*>(batch_validate_kernel), 256, 0);
        batch_validate_kernel<<<gv, 256, 0, s>>>(b->d_off_v, b->d_off_e, reinterpret_cast<const int32_t*>(k_out),
                                                 reinterpret_cast<const int32_t*>(v_out), d_epre, G, total_tiles, b->d_ctl);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_ctl, b->d_ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cc::cuda_fail(e, "cc_batch_reorder", __FILE__, __LINE__);
    if (st == CC_OK && b->h_ctl->bad_count)
        st = cc::set_error(CC_ECUDA, "cc_batch_reorder: internal error, %llu reordered ids out of range",
                           b->h_ctl->bad_count);
    cudaFree(k_in);
    cudaFree(v_in);
    cudaFree(deg);
    cudaFree(tmp);
    if (st != CC_OK) {
        cudaFree(k_out);
        cudaFree(v_out);
        return st;
    }
    // the plan now owns the reordered arrays; cached round graphs and
    // scheduler features referred to the old ones
    if (b->own_edges) {
        cudaFree(const_cast<int32_t*>(b->src));
        cudaFree(const_cast<int32_t*>(b->dst));
    }
    b->src = reinterpret_cast<const int32_t*>(k_out);
    b->dst = reinterpret_cast<const int32_t*>(v_out);
    b->own_edges = true;
    for (auto& l : b->loops) {
        if (l.exec) cudaGraphExecDestroy(l.exec);
        if (l.graph) cudaGraphDestroy(l.graph);
    }
    b->loops.clear();
    cc::sched_ctx_free(b->sched);
    b->sched = nullptr;
    return CC_OK;
}

extern "C" cc_status cc_batch_edges(const cc_batch_plan* b, const int32_t** src, const int32_t** dst) {
    if (!b) return cc::set_error(CC_EINVAL, "cc_batch_edges: batch is NULL");
    if (src) *src = b->src;
    if (dst) *dst = b->dst;
    return CC_OK;
}

extern "C" void cc_batch_free(cc_batch_plan* b) { destroy_batch(b); }

extern "C" cc_status cc_batch(int32_t n_graphs, const int64_t* vtx_off, const int64_t* edge_off,
                              const int32_t* src, const int32_t* dst, int order, int mode, int check_interval,
                              int32_t* labels_out, int32_t* sweeps_out, void* cuda_stream) {
    cc_batch_plan* b = nullptr;
    cc_status st = cc_batch_init(&b, n_graphs, vtx_off, edge_off, src, dst, 0, cuda_stream);
    if (st != CC_OK) return st;
    st = cc_batch_run(b, order, mode, check_interval, 1 << 20, labels_out, sweeps_out, nullptr);
    destroy_batch(b);
    return st;
}
