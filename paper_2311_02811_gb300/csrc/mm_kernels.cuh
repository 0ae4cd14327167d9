// Device kernels of the single-graph Contour path (sm_103a).
//
// Every kernel here works on a label array L[0..n-1] of vertex ids (int32_t or
// int64_t) and on an edge list given as two id arrays src[m], dst[m].
//
// Invariant relied on for memory safety: every value ever stored in L lies in
// [0, n) and satisfies L[x] <= x.  Labels start as ids (Alg. 1) or as a
// validated snapshot, and every store writes a value that was read from L, so
// every gather L[y] below is in bounds and every label chain strictly
// decreases until it reaches a root (L[r] == r).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cc {

// Device-side control block of one graph handle.
struct Ctl {
    int32_t flag;        // 1 if the checked sweep saw an edge that lowers a label
    int32_t sweeps;      // sweeps executed so far
    int32_t max_sweeps;  // stop after this many sweeps
    int32_t converged;   // 1 once a checked sweep saw no such edge
    unsigned long long bad_count;         // validation failures
    unsigned long long first_bad;         // smallest failing index
    unsigned long long compress_changes;  // labels changed by the final compress
    int32_t fresh;       // 1 when the run started from L[i] = i (no snapshot)
    int32_t sched_h;     // order of the next sweep under a per-iteration order schedule
};

constexpr int kFullChainHops = 1024;  // cap of the full-chain operator ("C-m", m = 1024)

// ---------------------------------------------------------------------------
// memory access helpers
// ---------------------------------------------------------------------------

// Edge stream: read once per sweep, never reused -> evict-first at L1 and L2.
__device__ __forceinline__ void load4(const int32_t* p, int32_t (&o)[4]) {
    int4 v = __ldcs(reinterpret_cast<const int4*>(p));
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void load4(const int64_t* p, int64_t (&o)[4]) {
    longlong2 a = __ldcs(reinterpret_cast<const longlong2*>(p));
    longlong2 b = __ldcs(reinterpret_cast<const longlong2*>(p) + 1);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}

// Label gather.  Synchronous sweeps never write L, so its reads may use the
// read-only path; asynchronous sweeps read L while other threads store into it.
template <bool SYNC, typename IdT>
__device__ __forceinline__ IdT rd(const IdT* L, IdT x) {
    if constexpr (SYNC) return __ldg(L + x);
    else return L[x];
}

// Conditional assignment x <- z (Def. 1).  The caller has already seen the
// old value exceed z.  Synchronous: atomic minimum into L_u (the CAS loop of
// Eq. "cas" collapses to one reduction).  Asynchronous: an atomic minimum
// into L as well.  Section III-B3 replaces atomics with plain stores because
// a lost write only costs iterations; on sm_103a the opposite holds: a plain
// store issued after a stale (L1-cached) read can raise a label that another
// SM has just lowered, and such stores measured up to 8x slower per solve
// than the fire-and-forget reduction (red.global.min) on 1e5-1e6 vertex
// graphs, with the same sweep counts.
template <typename IdT>
__device__ __forceinline__ void red_min(IdT* a, IdT z) {
    if constexpr (sizeof(IdT) == 4) atomicMin(reinterpret_cast<int*>(a), (int)z);
    else atomicMin(reinterpret_cast<long long*>(a), (long long)z);
}

template <bool SYNC, typename IdT>
__device__ __forceinline__ void wr(IdT* L, IdT* Lu, IdT x, IdT z) {
    if constexpr (SYNC) {
        // Read L_u at L2 first: hub vertices receive many candidate minima in
        // one sweep, and once one has landed most others are not smaller, so
        // the test removes most same-address atomics.
        if (__ldcg(Lu + x) > z) red_min(Lu + x, z);
    } else {
        red_min(L + x, z);
    }
}

// ---------------------------------------------------------------------------
// MM^h on K edges held in registers (h = H fixed at compile time)
// ---------------------------------------------------------------------------
//
// For edge <w, v>: chain c[0] = w, c[j] = L[c[j-1]] (j = 1..H);
// z = min(cw[H], cv[H]); every chain vertex c[j], j < H, whose label c[j+1]
// exceeds z is set to z (Def. 3).  Chains never increase (L[x] <= x), so some
// write is due exactly when max(L[w], L[v]) > z; for H = 2 that is the
// early-convergence test of Section III-B2 (L[v] != L^2[v] || L[w] != L^2[w]
// || L[v] != L[w]).  All loads of the K edges are issued before any store so
// that their latencies overlap.
template <int H, bool SYNC, int K, typename IdT>
__device__ __forceinline__ bool mm_fixed(const IdT (&w)[K], const IdT (&v)[K], IdT* L, IdT* Lu) {
    IdT cw[K][H + 1], cv[K][H + 1];
#pragma unroll
    for (int k = 0; k < K; ++k) { cw[k][0] = w[k]; cv[k][0] = v[k]; }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        cw[k][1] = rd<SYNC>(L, cw[k][0]);
        cv[k][1] = rd<SYNC>(L, cv[k][0]);
    }
    // Once a chain has reached a root (c[j] == c[j-1]) it only repeats it;
    // the repeat is taken from the register instead of another gather.
#pragma unroll
    for (int j = 2; j <= H; ++j) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            cw[k][j] = (cw[k][j - 1] == cw[k][j - 2]) ? cw[k][j - 1] : rd<SYNC>(L, cw[k][j - 1]);
            cv[k][j] = (cv[k][j - 1] == cv[k][j - 2]) ? cv[k][j - 1] : rd<SYNC>(L, cv[k][j - 1]);
        }
    }
    bool viol = false;
    IdT z[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        z[k] = cw[k][H] < cv[k][H] ? cw[k][H] : cv[k][H];
        viol |= (cw[k][1] > z[k]) | (cv[k][1] > z[k]);
    }
    if (!viol) return false;  // the common case of a late sweep: no write is due
    // w side: after cc_graph_reorder the edges are sorted by w, so a thread's
    // edges often share w (and then their chains).  Equal chain vertices are
    // adjacent; each run of them gets one write of the run's smallest z, which
    // equals the run's separate writes applied back to back (the conditional
    // assignments of Def. 1 commute, and the smallest wins).
#pragma unroll
    for (int j = 0; j < H; ++j) {
        IdT zr = z[0];
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
        for (int j = 0; j < H; ++j)
            if (cv[k][j + 1] > z[k]) wr<SYNC>(L, Lu, cv[k][j], z[k]);
    }
    return true;
}

// ---------------------------------------------------------------------------
// MM^h with h chosen at run time (orders other than 1, 2, 4, and the full
// chain).  The chain is walked twice: once to find z, once to write.  A walk
// stops early at a root (L[r] == r), where the chain would only repeat r.
// ---------------------------------------------------------------------------
template <bool SYNC, typename IdT>
__device__ __forceinline__ void rewalk(IdT x, IdT z, int h, IdT* L, IdT* Lu) {
    for (int j = 0; j < h; ++j) {
        const IdT y = rd<SYNC>(L, x);
        if (y <= z) break;  // labels further down the chain are <= y
        wr<SYNC>(L, Lu, x, z);
        if (y == x) break;  // root
        x = y;
    }
}

template <bool SYNC, typename IdT>
__device__ __forceinline__ bool mm_runtime(IdT w, IdT v, int h, IdT* L, IdT* Lu) {
    IdT ew = w, ev = v, fw = w, fv = v;
    bool dw = false, dv = false;
    for (int j = 0; j < h && !(dw && dv); ++j) {
        if (!dw) {
            const IdT y = rd<SYNC>(L, ew);
            if (j == 0) fw = y;
            dw = (y == ew);
            ew = y;
        }
        if (!dv) {
            const IdT y = rd<SYNC>(L, ev);
            if (j == 0) fv = y;
            dv = (y == ev);
            ev = y;
        }
    }
    const IdT z = ew < ev ? ew : ev;
    const bool viol = (fw > z) | (fv > z);
    if (fw > z) rewalk<SYNC>(w, z, h, L, Lu);
    if (fv > z) rewalk<SYNC>(v, z, h, L, Lu);
    return viol;
}

// The same run-time order for K edges at once: the 2K chains advance in
// lockstep, so each step issues up to 2K independent gathers; a chain stops
// at its root.  The write-back walks the chains again in lockstep.
template <bool SYNC, int K, typename IdT>
__device__ __forceinline__ bool mm_runtime_ilp(const IdT (&w)[K], const IdT (&v)[K], int h, IdT* L, IdT* Lu) {
    IdT cur[2 * K], first[2 * K];
    unsigned act = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        cur[2 * k] = w[k];
        cur[2 * k + 1] = v[k];
    }
#pragma unroll
    for (int i = 0; i < 2 * K; ++i) {
        first[i] = rd<SYNC>(L, cur[i]);
        if (first[i] != cur[i]) act |= 1u << i;
        cur[i] = first[i];
    }
    for (int j = 1; j < h && act; ++j) {
        IdT y[2 * K];
#pragma unroll
        for (int i = 0; i < 2 * K; ++i) y[i] = (act >> i & 1u) ? rd<SYNC>(L, cur[i]) : cur[i];
#pragma unroll
        for (int i = 0; i < 2 * K; ++i) {
            if (y[i] == cur[i]) act &= ~(1u << i);
            cur[i] = y[i];
        }
    }
    bool viol = false;
    IdT z[K];
    unsigned wact = 0;  // chains that must be written
#pragma unroll
    for (int k = 0; k < K; ++k) {
        z[k] = cur[2 * k] < cur[2 * k + 1] ? cur[2 * k] : cur[2 * k + 1];
        if (first[2 * k] > z[k]) wact |= 1u << (2 * k);
        if (first[2 * k + 1] > z[k]) wact |= 1u << (2 * k + 1);
    }
    viol = wact != 0;
    IdT x[2 * K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        x[2 * k] = w[k];
        x[2 * k + 1] = v[k];
    }
    for (int j = 0; j < h && wact; ++j) {
        IdT y[2 * K];
#pragma unroll
        for (int i = 0; i < 2 * K; ++i) y[i] = (wact >> i & 1u) ? rd<SYNC>(L, x[i]) : x[i];
#pragma unroll
        for (int i = 0; i < 2 * K; ++i) {
            if (!(wact >> i & 1u)) continue;
            const IdT zi = z[i >> 1];
            if (y[i] <= zi) {  // labels further down the chain are <= y
                wact &= ~(1u << i);
                continue;
            }
            wr<SYNC>(L, Lu, x[i], zi);
            if (y[i] == x[i]) wact &= ~(1u << i);  // root
            x[i] = y[i];
        }
    }
    return viol;
}

// ---------------------------------------------------------------------------
// the sweep: every edge once (Alg. 1 edge loop)
// ---------------------------------------------------------------------------
//
// Grid-stride over groups of 4 edges loaded with 16-byte streaming loads
// (src and dst are 16-byte aligned); the m % 4 tail edges are taken by the
// first threads of the grid.  H = 0 selects the run-time order h.
// flag == nullptr: sweep without convergence check (inside a check block).
//
// The first sweep of a run that starts from L[i] = i needs no gathers: every
// chain of the identity state is trivial (L^j[x] = x), so MM^h reduces to
// z = min(w, v) and one conditional assignment to max(w, v).  That sweep
// ("identity sweep") applies it with an atomic minimum, which gives exactly
// the state after the first iteration of Alg. 1 in both modes.
//   first == 0: ordinary sweep
//   first == 1: identity sweep iff ctl->sweeps == 0 and ctl->fresh
//   first == 2: identity sweep
// gate != 0: the sweep belongs to a per-iteration order schedule (the C-11mm
// and C-1m1m variants of Section III-B4) and runs only when ctl->sched_h ==
// gate; otherwise it returns at once.
// The target is read at L2 first: a hub receives one candidate from each of
// its edges, and once a small one has landed the others need no atomic
// (synchronous R-MAT 24: identity sweep 2.36 -> 1.24 ms).
template <typename IdT>
__device__ __forceinline__ bool identity_pair(IdT w, IdT v, IdT* target) {
    if (w == v) return false;
    const IdT lo = w < v ? w : v;
    const IdT hi = w < v ? v : w;
    if (__ldcg(target + hi) > lo) red_min(target + hi, lo);
    return true;
}

// Four resident blocks (64 registers) for int32 ids, 4 edges per thread and
// h <= 2; two for the wider cases, which would spill under that cap.
template <int H, bool SYNC, int G, typename IdT>
__global__ void __launch_bounds__(256, (sizeof(IdT) == 4 && G == 1 && H <= 2 && H > 0) ? 4 : 2)
mm_sweep_kernel(const IdT* __restrict__ src, const IdT* __restrict__ dst, int64_t m,
                IdT* L, IdT* Lu, int h, int32_t* flag, const Ctl* ctl, int first, int gate) {
    if (gate != 0 && ctl->sched_h != gate) return;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t ngroups = m / (4 * G);
    bool viol = false;
    const bool ident = first == 2 || (first == 1 && ctl->sweeps == 0 && ctl->fresh != 0);
    if (ident) {
        IdT* target = SYNC ? Lu : L;
        const int64_t q4 = m / 4;
        for (int64_t g = tid; g < q4; g += stride) {
            IdT w[4], v[4];
            load4(src + g * 4, w);
            load4(dst + g * 4, v);
#pragma unroll
            for (int k = 0; k < 4; ++k) viol |= identity_pair(w[k], v[k], target);
        }
        const int64_t t = q4 * 4 + tid;
        if (t < m) viol |= identity_pair(__ldcs(src + t), __ldcs(dst + t), target);
        if (flag != nullptr) {
            if (__syncthreads_or(viol) && threadIdx.x == 0) *flag = 1;
        }
        return;
    }
    // The next group's edges are loaded before this group's gathers, so the
    // stream's DRAM latency overlaps the dependent label gathers.
    IdT wn[4 * G], vn[4 * G];
    auto load_group = [&](int64_t gg) {
#pragma unroll
        for (int q = 0; q < G; ++q) {
            IdT t[4];
            load4(src + (gg * G + q) * 4, t);
#pragma unroll
            for (int i = 0; i < 4; ++i) wn[4 * q + i] = t[i];
            load4(dst + (gg * G + q) * 4, t);
#pragma unroll
            for (int i = 0; i < 4; ++i) vn[4 * q + i] = t[i];
        }
    };
    if (tid < ngroups) load_group(tid);
    for (int64_t g = tid; g < ngroups; g += stride) {
        IdT w[4 * G], v[4 * G];
#pragma unroll
        for (int i = 0; i < 4 * G; ++i) {
            w[i] = wn[i];
            v[i] = vn[i];
        }
        if (g + stride < ngroups) load_group(g + stride);
        if constexpr (H > 0) {
            viol |= mm_fixed<H, SYNC, 4 * G>(w, v, L, Lu);
        } else {
            viol |= mm_runtime_ilp<SYNC, 4 * G>(w, v, h, L, Lu);
        }
    }
    const int64_t tail0 = ngroups * 4 * G;
    if (tid < m - tail0) {
        IdT w[1] = {__ldcs(src + tail0 + tid)};
        IdT v[1] = {__ldcs(dst + tail0 + tid)};
        if constexpr (H > 0) viol |= mm_fixed<H, SYNC, 1>(w, v, L, Lu);
        else viol |= mm_runtime<SYNC>(w[0], v[0], h, L, Lu);
    }
    if (flag != nullptr) {
        // one store per block, only when some edge of the block could lower a label
        if (__syncthreads_or(viol) && threadIdx.x == 0) *flag = 1;
    }
}

// ---------------------------------------------------------------------------
// label initialisation, copy, compress, validation
// ---------------------------------------------------------------------------

// L[i] = i and, for synchronous runs, L_u[i] = i (Alg. 1 initialisation).
template <typename IdT>
__global__ void iota_kernel(IdT* L, IdT* Lu, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        L[i] = (IdT)i;
        if (Lu) Lu[i] = (IdT)i;
    }
}

// dst[i] = src[i] for i < count ids, 16-byte vectors plus a scalar tail
// (L = L_u of Alg. 1; both arrays are 256-byte aligned device allocations or
// the caller's 16-byte aligned output).
template <typename IdT>
__global__ void copy_kernel(IdT* __restrict__ dst, const IdT* __restrict__ src, int64_t count) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    constexpr int per = 16 / sizeof(IdT);
    const int64_t nv = count / per;
    const int4* s4 = reinterpret_cast<const int4*>(src);
    int4* d4 = reinterpret_cast<int4*>(dst);
    for (int64_t i = tid; i < nv; i += stride) d4[i] = s4[i];
    const int64_t t = nv * per + tid;
    if (t < count) dst[t] = src[t];
}

// Final compress: L[x] becomes the root of x's chain, so the pointer graph is
// a set of stars (Section II-A).  At a fixed point of the sweep this changes
// nothing; the number of changed labels is reported for checking.  Chains
// strictly decrease, so each walk ends; the walk is still capped.
// Runs only after a converged loop; a partial state (max_sweeps reached) is
// left exactly as the last sweep wrote it, so that it resumes bit-exactly.
template <typename IdT>
__global__ void compress_kernel(IdT* L, int64_t n, Ctl* ctl) {
    if (!ctl->converged) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long changes = 0;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
        const IdT l = L[x];
        IdT r = l;
        IdT p = L[r];
        for (int guard = 0; p != r && guard < (1 << 24); ++guard) {
            r = p;
            p = L[r];
        }
        if (r != l) {
            L[x] = r;
            ++changes;
        }
    }
    for (int o = 16; o > 0; o >>= 1) changes += __shfl_xor_sync(0xffffffffu, changes, o);
    if ((threadIdx.x & 31) == 0 && changes) atomicAdd(&ctl->compress_changes, changes);
}

// Count endpoints of src[count] and dst[count] outside [0, n) and record the
// smallest failing edge index.  Both arrays are 16-byte aligned; they are read
// as 4-id vectors (the count % 4 tail with scalar loads).
template <typename IdT>
__device__ __forceinline__ void check_id(IdT x, int64_t n, int64_t e, unsigned long long& bad, Ctl* ctl) {
    if (x < 0 || (int64_t)x >= n) {
        ++bad;
        atomicMin(&ctl->first_bad, (unsigned long long)e);
    }
}

template <typename IdT>
__global__ void validate_ids_kernel(const IdT* src, const IdT* dst, int64_t count, int64_t n, Ctl* ctl) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long bad = 0;
    const int64_t q4 = count / 4;
    for (int64_t g = tid; g < q4; g += stride) {
        IdT a[4], b[4];
        load4(src + 4 * g, a);
        load4(dst + 4 * g, b);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            check_id(a[k], n, 4 * g + k, bad, ctl);
            check_id(b[k], n, 4 * g + k, bad, ctl);
        }
    }
    const int64_t t = 4 * q4 + tid;
    if (t < count) {
        check_id(src[t], n, t, bad, ctl);
        check_id(dst[t], n, t, bad, ctl);
    }
    for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, o);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(&ctl->bad_count, bad);
}

// A resume snapshot must satisfy 0 <= L[x] <= x (labels never exceed ids).
template <typename IdT>
__global__ void validate_snapshot_kernel(const IdT* L, int64_t n, Ctl* ctl) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const IdT x = L[i];
        if (x < 0 || (int64_t)x > i) {
            ++bad;
            atomicMin(&ctl->first_bad, (unsigned long long)i);
        }
    }
    for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, o);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(&ctl->bad_count, bad);
}

// CSR offsets must run from 0 to nnz without decreasing.
static __global__ void validate_offsets_kernel(const int64_t* off, int64_t n, int64_t nnz, Ctl* ctl) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += stride) {
        const int64_t o = off[i];
        bool ok = (i == 0) ? (o == 0) : (o >= off[i - 1]);
        if (i == n) ok = ok && (o == nnz);
        if (!ok) {
            ++bad;
            atomicMin(&ctl->first_bad, (unsigned long long)i);
        }
    }
    for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, o);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(&ctl->bad_count, bad);
}

// CSR -> COO: entry k belongs to the row r with off[r] <= k < off[r+1].
template <typename IdT>
__global__ void csr_rows_kernel(const int64_t* off, int64_t n, int64_t nnz, IdT* rows) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += stride) {
        int64_t lo = 0, hi = n;  // largest r with off[r] <= k
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (off[mid] <= k) lo = mid; else hi = mid;
        }
        rows[k] = (IdT)lo;
    }
}

static __global__ void ctl_reset_kernel(Ctl* ctl, int32_t max_sweeps, int32_t fresh, int32_t sched_h = 0) {
    if (threadIdx.x == 0) {
        ctl->fresh = fresh;
        ctl->sched_h = sched_h;
        ctl->flag = 0;
        ctl->sweeps = 0;
        ctl->max_sweeps = max_sweeps;
        ctl->converged = 0;
        ctl->bad_count = 0;
        ctl->first_bad = ~0ull;
        ctl->compress_changes = 0;
    }
}

// End of one check block inside the conditional WHILE body: read and clear the
// flag, count the block's sweeps, and decide whether the loop runs again.
// sched: 0 none; 1 C-11mm (order 1 for two sweeps, then the full chain);
// 2 C-1m1m (order 1 and the full chain alternately).
static __global__ void check_kernel(Ctl* ctl, int32_t block_sweeps, cudaGraphConditionalHandle loop,
                                    int sched = 0) {
    if (threadIdx.x == 0) {
        const int32_t f = ctl->flag;
        ctl->flag = 0;
        ctl->sweeps += block_sweeps;
        if (sched == 1) ctl->sched_h = ctl->sweeps < 2 ? 1 : kFullChainHops;
        if (sched == 2) ctl->sched_h = (ctl->sweeps % 2 == 0) ? 1 : kFullChainHops;
        ctl->converged = (f == 0);
        cudaGraphSetConditional(loop, (f != 0 && ctl->sweeps < ctl->max_sweeps) ? 1u : 0u);
    }
}

}  // namespace cc
