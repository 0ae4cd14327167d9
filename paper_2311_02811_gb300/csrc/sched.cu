// Learned schedule selection (CC_ORDER_AUTO): graph features -> a small MLP
// -> (operator order, sync/async mode, check interval).
//
// The paper picks operators by hand from graph size and diameter (Section
// IV-E: C-1 for small low-diameter graphs, C-m for large or long-diameter
// ones, C-2 as the stable default); this file learns that choice from
// measured solve times.  Every schedule returns identical labels, so the
// choice only changes the run time.
//
// Features (12 per graph, log2(1 + x) of each quantity):
//   0 n, 1 m,
//   2 degree variance, 3 maximum degree   (estimated from an edge sample),
//   4..11 eccentricities of 8 sources in the sampled graph (BFS, capped).
// The sample is every edge when m <= kSample, else the kSample edges at
// positions floor(j * m / kSample).  Degrees are counted on the sample and
// scaled by m / |sample|.  Sources are the src endpoints of sample positions
// floor((2i+1) * |sample| / 16).  BFS runs level by level on the sample graph
// from all 8 sources at once (one bit per source) for at most kLevels levels.
//
// MLP: 12 -> 64 -> 64 -> 64 -> 18, ReLU, inputs standardised with the
// training mean/std; weights BF16, biases and accumulation FP32.
// Output class k = order_idx * 6 + async * 3 + interval_idx with orders
// {2, 4, full chain} and intervals {1, 2, 4}.
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/contour.h"
#include "cc_internal.h"
#include "csr_kernels.cuh"
#include "hub_kernels.cuh"

namespace {

constexpr int kFeat = CC_SCHED_FEATURES;
constexpr int kHidden = 64;
constexpr int kOut = CC_SCHED_CLASSES;
constexpr int kSample = 16384;
constexpr int kLevels = 16;
constexpr int kFeatThreads = 1024;

// ---------------------------------------------------------------------------
// weights blob
// ---------------------------------------------------------------------------

struct BlobHeader {
    char magic[8];  // "CCMLP01"
    int32_t n_in, n_hidden, n_layers, n_out;
    float mean[kFeat];
    float std_[kFeat];
};

// parameter counts of the four layers
constexpr int kW1 = kHidden * kFeat, kW2 = kHidden * kHidden, kW3 = kHidden * kHidden, kW4 = kOut * kHidden;
constexpr size_t kBlobBytes = sizeof(BlobHeader) + 2 * (kW1 + kW2 + kW3 + kW4) + 4 * (3 * kHidden + kOut);

// Device-side model: bf16 weights and fp32 biases, plus normalisation.
struct Model {
    float mean[kFeat], inv_std[kFeat];
    __nv_bfloat16 w1[kW1], w2[kW2], w3[kW3], w4[kW4];
    float b1[kHidden], b2[kHidden], b3[kHidden], b4[kOut];
};

std::mutex g_mu;
Model* g_model = nullptr;  // device copy, nullptr when nothing is loaded
Model* g_model_batch = nullptr;  // weights for batched solves (cc_sched_load_batch), optional
long long g_model_version = 0;  // bumped by every cc_sched_load / cc_sched_load_batch
std::vector<unsigned char> g_blob, g_blob_batch;

// ---------------------------------------------------------------------------
// features
// ---------------------------------------------------------------------------

// Per-CTA scratch of the feature kernel: an open-addressing table from the
// sample's vertices to slots (at most 2 * kSample distinct vertices, so a
// table of 4 * kSample slots stays at most half full), per-slot degree and
// BFS words, the sample's edges as slot pairs, and the list of used slots.
// The kernel returns every slot it used to empty, so the scratch is cleared
// once when allocated and never again.
constexpr int kSlots = 4 * kSample;

struct FeatArgs {
    int32_t G;
    const int64_t* off_v;
    const int64_t* off_e;
    const int32_t* src;
    const int32_t* dst;
    int32_t* keys;       // kSlots per CTA, -1 = empty
    int32_t* deg;        // kSlots per CTA
    uint32_t* word;      // kSlots per CTA: bits 0-7 visited, 8-15 frontier, 16-23 next
    int32_t* su;         // kSample per CTA: slot of the sample edge's src
    int32_t* sv;         // kSample per CTA: slot of its dst
    int32_t* owned;      // 2 * kSample per CTA: slots in use
    float* out;          // G x kFeat
};

__device__ __forceinline__ long long sample_pos(long long j, long long m, long long S) {
    return (m <= S) ? j : (j * m) / S;
}

// Slot of vertex x; a new slot is appended to the used list.
__device__ __forceinline__ int32_t table_slot(int32_t* keys, int32_t x, int32_t* owned, int32_t* n_owned) {
    uint32_t h = ((uint32_t)x * 2654435761u) & (kSlots - 1);
    for (int probe = 0; probe < kSlots; ++probe) {
        const int32_t k = atomicCAS(keys + h, -1, x);
        if (k == -1) {
            owned[atomicAdd(n_owned, 1)] = (int32_t)h;
            return (int32_t)h;
        }
        if (k == x) return (int32_t)h;
        h = (h + 1) & (kSlots - 1);
    }
    return -1;  // unreachable: the table is at most half full
}

__global__ void __launch_bounds__(kFeatThreads) features_kernel(FeatArgs a) {
    __shared__ int32_t s_owned;
    __shared__ unsigned long long s_sumsq;
    __shared__ int32_t s_max;
    __shared__ int32_t s_ecc[8];
    int32_t* keys = a.keys + (size_t)blockIdx.x * kSlots;
    int32_t* deg = a.deg + (size_t)blockIdx.x * kSlots;
    uint32_t* word = a.word + (size_t)blockIdx.x * kSlots;
    int32_t* su = a.su + (size_t)blockIdx.x * kSample;
    int32_t* sv = a.sv + (size_t)blockIdx.x * kSample;
    int32_t* owned = a.owned + (size_t)blockIdx.x * 2 * kSample;
    for (int32_t g = blockIdx.x; g < a.G; g += gridDim.x) {
        const long long n = a.off_v[g + 1] - a.off_v[g];
        const long long e0 = a.off_e[g];
        const long long m = a.off_e[g + 1] - e0;
        const long long S = m < kSample ? m : kSample;
        if (threadIdx.x == 0) {
            s_owned = 0;
            s_sumsq = 0;
            s_max = 0;
        }
        if (threadIdx.x < 8) s_ecc[threadIdx.x] = 0;
        __syncthreads();
        // sample edges -> slots; degrees on the sample
        for (long long j0 = threadIdx.x; j0 < S; j0 += (long long)blockDim.x * 4) {
            int32_t eu[4], ev[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const long long j = j0 + (long long)k * blockDim.x;
                const long long e = e0 + sample_pos(j < S ? j : 0, m, S);
                eu[k] = a.src[e];
                ev[k] = a.dst[e];
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const long long j = j0 + (long long)k * blockDim.x;
                if (j >= S) continue;
                const int32_t pu = table_slot(keys, eu[k], owned, &s_owned);
                const int32_t pv = table_slot(keys, ev[k], owned, &s_owned);
                su[j] = pu;
                sv[j] = pv;
                atomicAdd(deg + pu, 1);
                atomicAdd(deg + pv, 1);
            }
        }
        __syncthreads();
        const int32_t no = s_owned;
        unsigned long long sq = 0;
        int32_t mx = 0;
        for (int32_t i = threadIdx.x; i < no; i += blockDim.x) {
            const long long dd = deg[owned[i]];
            sq += (unsigned long long)(dd * dd);
            mx = max(mx, (int32_t)dd);
        }
        atomicAdd(&s_sumsq, sq);
        atomicMax(&s_max, mx);
        // 8 BFS sources: the src endpoints of sample positions floor((2i+1) S / 16)
        if (threadIdx.x < 8 && S > 0) {
            const long long j = ((2ll * threadIdx.x + 1) * S) / 16;
            atomicOr(word + su[j], (1u << threadIdx.x) | (1u << (8 + threadIdx.x)));
        }
        __syncthreads();
        // Level-synchronous BFS; each thread takes 4 items per step and issues
        // all their loads before any atomic so that the latencies overlap.
        constexpr int U = 4;
        for (int level = 1; level <= kLevels; ++level) {
            for (long long j0 = threadIdx.x; j0 < S; j0 += (long long)blockDim.x * U) {
                int32_t pu[U], pv[U];
                uint32_t wu[U], wv[U];
#pragma unroll
                for (int k = 0; k < U; ++k) {
                    const long long j = j0 + (long long)k * blockDim.x;
                    pu[k] = j < S ? su[j] : -1;
                    pv[k] = j < S ? sv[j] : -1;
                }
#pragma unroll
                for (int k = 0; k < U; ++k) {
                    wu[k] = pu[k] >= 0 ? word[pu[k]] : 0u;
                    wv[k] = pv[k] >= 0 ? word[pv[k]] : 0u;
                }
#pragma unroll
                for (int k = 0; k < U; ++k) {
                    if (pu[k] < 0) continue;
                    const uint32_t to_v = ((wu[k] >> 8) & 0xffu) & ~(wv[k] & 0xffu);
                    const uint32_t to_u = ((wv[k] >> 8) & 0xffu) & ~(wu[k] & 0xffu);
                    if (to_v) atomicOr(word + pv[k], to_v << 16);
                    if (to_u) atomicOr(word + pu[k], to_u << 16);
                }
            }
            __syncthreads();
            int any = 0;
            for (int32_t i0 = threadIdx.x; i0 < no; i0 += blockDim.x * U) {
                int32_t x[U];
                uint32_t w[U];
#pragma unroll
                for (int k = 0; k < U; ++k) {
                    const int32_t i = i0 + k * blockDim.x;
                    x[k] = i < no ? owned[i] : -1;
                }
#pragma unroll
                for (int k = 0; k < U; ++k) w[k] = x[k] >= 0 ? word[x[k]] : 0u;
#pragma unroll
                for (int k = 0; k < U; ++k) {
                    if (x[k] < 0) continue;
                    const uint32_t fresh = ((w[k] >> 16) & 0xffu) & ~(w[k] & 0xffu);
                    word[x[k]] = (w[k] & 0xffu) | fresh | (fresh << 8);
                    if (fresh) {
                        any = 1;
                        for (int b = 0; b < 8; ++b)
                            if (fresh >> b & 1u) atomicMax(&s_ecc[b], level);
                    }
                }
            }
            if (__syncthreads_or(any) == 0) break;
        }
        // return every used slot to empty for the next graph / call
        for (int32_t i = threadIdx.x; i < no; i += blockDim.x) {
            const int32_t x = owned[i];
            keys[x] = -1;
            deg[x] = 0;
            word[x] = 0;
        }
        if (threadIdx.x == 0) {
            float* f = a.out + (size_t)g * kFeat;
            const double scale = S > 0 ? (double)m / (double)S : 0.0;
            const double nn = n > 0 ? (double)n : 1.0;
            const double mean = 2.0 * (double)S / nn;
            const double var_s = (double)s_sumsq / nn - mean * mean;
            const double var_est = (var_s > 0 ? var_s : 0.0) * scale * scale;
            const double max_est = (double)s_max * scale;
            f[0] = (float)log2(1.0 + (double)n);
            f[1] = (float)log2(1.0 + (double)m);
            f[2] = (float)log2(1.0 + var_est);
            f[3] = (float)log2(1.0 + max_est);
            for (int b = 0; b < 8; ++b) f[4 + b] = (float)log2(1.0 + (double)s_ecc[b]);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// features of ONE graph on a thread-block cluster of 8 CTAs (8 SMs)
// ---------------------------------------------------------------------------
//
// Same definition as features_kernel, computed with the vertex table spread
// over the shared memory of the 8 CTAs of a cluster (distributed shared
// memory): a vertex's slot lives in CTA (hash >> 29), each CTA takes 1/8 of
// the sample edges, and remote slots are read and updated with DSMEM loads
// and atomics.  Phases and BFS levels are separated by cluster barriers.

namespace cgx = cooperative_groups;

constexpr int kCl = 8;                         // CTAs per cluster
constexpr int kPart = kSlots / kCl;            // slots per CTA
constexpr int kClEdges = kSample / kCl;        // sample edges per CTA
static_assert((kPart & (kPart - 1)) == 0, "slot partition must be a power of two");
constexpr int kPartBits = 13;
static_assert((1 << kPartBits) == kPart, "kPartBits");

struct ClusterSmem {
    int32_t keys[kPart];
    int32_t deg[kPart];
    uint32_t word[kPart];
    int32_t owned[kPart];   // local slots in use
    int32_t su[kClEdges];   // global slot id (owner << kPartBits | local) of this CTA's edges
    int32_t sv[kClEdges];
    int32_t n_owned;
    int32_t maxdeg;                     // rank-0 accumulators
    unsigned long long sumsq;
    int32_t ecc[8];
    int32_t any[kLevels + 2];
};

__device__ __forceinline__ int32_t cl_slot(cgx::cluster_group& cl, ClusterSmem* me, int32_t x) {
    const uint32_t h = (uint32_t)x * 2654435761u;
    const int owner = (int)(h >> 29);
    uint32_t loc = (h >> 13) & (kPart - 1);
    ClusterSmem* o = cl.map_shared_rank(me, owner);
    for (int probe = 0; probe < kPart; ++probe) {
        const int32_t k = atomicCAS(&o->keys[loc], -1, x);
        if (k == -1) {
            o->owned[atomicAdd(&o->n_owned, 1)] = (int32_t)loc;
            return (owner << kPartBits) | (int32_t)loc;
        }
        if (k == x) return (owner << kPartBits) | (int32_t)loc;
        loc = (loc + 1) & (kPart - 1);
    }
    return -1;  // unreachable: at most 2 * kSample vertices in 8 * kPart slots
}

__device__ __forceinline__ uint32_t* cl_word(cgx::cluster_group& cl, ClusterSmem* me, int32_t slot) {
    return &cl.map_shared_rank(me, slot >> kPartBits)->word[slot & (kPart - 1)];
}

// m_feat < 0: the sample is taken from the m = off_e[1] - off_e[0] edges
// src/dst.  m_feat >= 0: src/dst already hold the S sampled pairs (S =
// off_e[1] - off_e[0] <= kSample) of a graph with m_feat edges.
__global__ void __launch_bounds__(kFeatThreads) features_cluster_kernel(const int64_t* off_v, const int64_t* off_e,
                                                                     const int32_t* src, const int32_t* dst,
                                                                     long long m_feat, float* out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ClusterSmem* me = reinterpret_cast<ClusterSmem*>(smem_raw);
    cgx::cluster_group cl = cgx::this_cluster();
    const int rank = (int)cl.block_rank();
    ClusterSmem* r0 = cl.map_shared_rank(me, 0);
    const long long n = off_v[1] - off_v[0];
    const long long e0 = off_e[0];
    const bool pre = m_feat >= 0;
    const long long m = pre ? m_feat : off_e[1] - e0;
    const long long S = pre ? off_e[1] - e0 : (m < kSample ? m : kSample);
    const long long per = (S + kCl - 1) / kCl;
    const long long jb = rank * per;
    const long long je = min(S, jb + per);
    for (int i = threadIdx.x; i < kPart; i += blockDim.x) {
        me->keys[i] = -1;
        me->deg[i] = 0;
        me->word[i] = 0;
    }
    if (threadIdx.x == 0) {
        me->n_owned = 0;
        me->maxdeg = 0;
        me->sumsq = 0;
    }
    if (threadIdx.x < 8) me->ecc[threadIdx.x] = 0;
    if (threadIdx.x < kLevels + 2) me->any[threadIdx.x] = 0;
    cl.sync();
    // this CTA's share of the sample: slots and degrees
    for (long long j = jb + threadIdx.x; j < je; j += blockDim.x) {
        const long long e = e0 + (pre ? j : sample_pos(j, m, S));
        const int32_t pu = cl_slot(cl, me, src[e]);
        const int32_t pv = cl_slot(cl, me, dst[e]);
        me->su[j - jb] = pu;
        me->sv[j - jb] = pv;
        atomicAdd(&cl.map_shared_rank(me, pu >> kPartBits)->deg[pu & (kPart - 1)], 1);
        atomicAdd(&cl.map_shared_rank(me, pv >> kPartBits)->deg[pv & (kPart - 1)], 1);
    }
    cl.sync();
    {
        unsigned long long sq = 0;
        int32_t mx = 0;
        for (int32_t i = threadIdx.x; i < me->n_owned; i += blockDim.x) {
            const long long dd = me->deg[me->owned[i]];
            sq += (unsigned long long)(dd * dd);
            mx = max(mx, (int32_t)dd);
        }
        if (sq) atomicAdd(&r0->sumsq, sq);
        if (mx) atomicMax(&r0->maxdeg, mx);
    }
    // the 8 BFS sources: src endpoints of sample positions floor((2i+1) S / 16)
    if (threadIdx.x < 8 && S > 0) {
        const long long j = ((2ll * threadIdx.x + 1) * S) / 16;
        if (j >= jb && j < je)
            atomicOr(cl_word(cl, me, me->su[j - jb]), (1u << threadIdx.x) | (1u << (8 + threadIdx.x)));
    }
    cl.sync();
    for (int level = 1; level <= kLevels; ++level) {
        for (long long j = jb + threadIdx.x; j < je; j += blockDim.x) {
            const int32_t pu = me->su[j - jb], pv = me->sv[j - jb];
            uint32_t* au = cl_word(cl, me, pu);
            uint32_t* av = cl_word(cl, me, pv);
            const uint32_t wu = *au, wv = *av;
            const uint32_t to_v = ((wu >> 8) & 0xffu) & ~(wv & 0xffu);
            const uint32_t to_u = ((wv >> 8) & 0xffu) & ~(wu & 0xffu);
            if (to_v) atomicOr(av, to_v << 16);
            if (to_u) atomicOr(au, to_u << 16);
        }
        cl.sync();
        int any = 0;
        for (int32_t i = threadIdx.x; i < me->n_owned; i += blockDim.x) {
            const int32_t x = me->owned[i];
            const uint32_t w = me->word[x];
            const uint32_t fresh = ((w >> 16) & 0xffu) & ~(w & 0xffu);
            me->word[x] = (w & 0xffu) | fresh | (fresh << 8);
            if (fresh) {
                any = 1;
                for (int b = 0; b < 8; ++b)
                    if (fresh >> b & 1u) atomicMax(&r0->ecc[b], level);
            }
        }
        if (any) atomicOr(&r0->any[level], 1);
        cl.sync();
        if (r0->any[level] == 0) break;
    }
    cl.sync();
    if (rank == 0 && threadIdx.x == 0) {
        const double scale = S > 0 ? (double)m / (double)S : 0.0;
        const double nn = n > 0 ? (double)n : 1.0;
        const double mean = 2.0 * (double)S / nn;
        const double var_s = (double)me->sumsq / nn - mean * mean;
        const double var_est = (var_s > 0 ? var_s : 0.0) * scale * scale;
        const double max_est = (double)me->maxdeg * scale;
        out[0] = (float)log2(1.0 + (double)n);
        out[1] = (float)log2(1.0 + (double)m);
        out[2] = (float)log2(1.0 + var_est);
        out[3] = (float)log2(1.0 + max_est);
        for (int b = 0; b < 8; ++b) out[4 + b] = (float)log2(1.0 + (double)me->ecc[b]);
    }
}

// ---------------------------------------------------------------------------
// MLP inference: one warp per graph, FP32 accumulation of BF16 weights
// ---------------------------------------------------------------------------

__device__ __forceinline__ float dense_unit(const __nv_bfloat16* w, const float* b, const float* x, int n_in, int unit) {
    float acc = b[unit];
    for (int i = 0; i < n_in; ++i) acc += __bfloat162float(w[unit * n_in + i]) * x[i];
    return acc;
}

__global__ void mlp_infer_kernel(const Model* M, const float* feats, int32_t G, int32_t* cls, float* logits) {
    __shared__ float sh[8][3][kHidden];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int32_t g = blockIdx.x * 8 + warp;
    if (g >= G) return;
    float* x0 = sh[warp][0];
    float* h1 = sh[warp][1];
    float* h2 = sh[warp][2];
    if (lane < kFeat) x0[lane] = (feats[(size_t)g * kFeat + lane] - M->mean[lane]) * M->inv_std[lane];
    __syncwarp();
    for (int u = lane; u < kHidden; u += 32) h1[u] = fmaxf(dense_unit(M->w1, M->b1, x0, kFeat, u), 0.f);
    __syncwarp();
    for (int u = lane; u < kHidden; u += 32) h2[u] = fmaxf(dense_unit(M->w2, M->b2, h1, kHidden, u), 0.f);
    __syncwarp();
    float h3v[2];
    for (int r = 0; r < 2; ++r) h3v[r] = fmaxf(dense_unit(M->w3, M->b3, h2, kHidden, lane + 32 * r), 0.f);
    __syncwarp();
    h1[lane] = h3v[0];
    h1[lane + 32] = h3v[1];
    __syncwarp();
    float z = -INFINITY;
    if (lane < kOut) z = dense_unit(M->w4, M->b4, h1, kHidden, lane);
    if (logits && lane < kOut) logits[(size_t)g * kOut + lane] = z;
    // argmax, lowest index on ties
    float best = z;
    int bi = lane < kOut ? lane : kOut;
    for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
            best = ob;
            bi = oi;
        }
    }
    if (lane == 0) cls[g] = bi;
}

// ---------------------------------------------------------------------------
// MLP training: mini-batch Adam on softmax cross-entropy, all FP32
// ---------------------------------------------------------------------------

struct Params {  // fp32 master parameters, one contiguous buffer
    float* w[4];
    float* b[4];
};

constexpr int kIn[4] = {kFeat, kHidden, kHidden, kHidden};
constexpr int kOutDim[4] = {kHidden, kHidden, kHidden, kOut};
constexpr int kParams = kW1 + kW2 + kW3 + kW4 + 3 * kHidden + kOut;

// Z[s][o] = b[o] + sum_i W[o][i] X[s][i]; A = relu(Z) unless last
__global__ void dense_fwd_kernel(const float* W, const float* b, const float* X, int n_in, int n_out, int B,
                                 float* Z, float* A, int relu) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * n_out) return;
    const int s = idx / n_out, o = idx % n_out;
    float acc = b[o];
    for (int i = 0; i < n_in; ++i) acc += W[o * n_in + i] * X[s * n_in + i];
    Z[idx] = acc;
    if (A) A[idx] = relu ? fmaxf(acc, 0.f) : acc;
}

// dZ = (softmax(Z) - onehot(label)) / B ; loss accumulated (mean CE)
__global__ void softmax_ce_kernel(const float* Z, const int32_t* y, int B, float* dZ, float* loss) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B) return;
    const float* z = Z + s * kOut;
    float mx = z[0];
    for (int k = 1; k < kOut; ++k) mx = fmaxf(mx, z[k]);
    float sum = 0.f;
    for (int k = 0; k < kOut; ++k) sum += expf(z[k] - mx);
    const int lab = y[s];
    for (int k = 0; k < kOut; ++k) {
        const float p = expf(z[k] - mx) / sum;
        dZ[s * kOut + k] = (p - (k == lab ? 1.f : 0.f)) / (float)B;
    }
    atomicAdd(loss, (logf(sum) + mx - z[lab]) / (float)B);
}

// dW[o][i] = sum_s dZ[s][o] X[s][i]; db[o] = sum_s dZ[s][o]
__global__ void dense_grad_kernel(const float* dZ, const float* X, int n_in, int n_out, int B, float* dW,
                                  float* db) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n_out * n_in) {
        const int o = idx / n_in, i = idx % n_in;
        float acc = 0.f;
        for (int s = 0; s < B; ++s) acc += dZ[s * n_out + o] * X[s * n_in + i];
        dW[idx] = acc;
    }
    if (idx < n_out) {
        float acc = 0.f;
        for (int s = 0; s < B; ++s) acc += dZ[s * n_out + idx];
        db[idx] = acc;
    }
}

// dX[s][i] = (sum_o W[o][i] dZ[s][o]) * (Zprev[s][i] > 0)
__global__ void dense_bwd_input_kernel(const float* W, const float* dZ, const float* Zprev, int n_in, int n_out,
                                       int B, float* dX) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * n_in) return;
    const int s = idx / n_in, i = idx % n_in;
    float acc = 0.f;
    for (int o = 0; o < n_out; ++o) acc += W[o * n_in + i] * dZ[s * n_out + o];
    dX[idx] = Zprev[idx] > 0.f ? acc : 0.f;
}

// Adam (Kingma & Ba 2015) with bias correction; t is the 1-based step.
__global__ void adam_kernel(float* p, const float* g, float* m1, float* m2, int count, float lr, float b1,
                            float b2, float eps, int t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float c = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = c;
    const float ah = a / (1.f - powf(b1, (float)t));
    const float ch = c / (1.f - powf(b2, (float)t));
    p[i] -= lr * ah / (sqrtf(ch) + eps);
}

// per-feature mean and population std over N rows (one thread per feature)
__global__ void feat_stats_kernel(const float* X, int N, float* mean, float* std_) {
    const int f = threadIdx.x;
    if (f >= kFeat) return;
    double s = 0, q = 0;
    for (int r = 0; r < N; ++r) {
        const double v = X[(size_t)r * kFeat + f];
        s += v;
        q += v * v;
    }
    const double mu = N ? s / N : 0.0;
    double var = N ? q / N - mu * mu : 0.0;
    if (var < 0) var = 0;
    mean[f] = (float)mu;
    std_[f] = (float)(var > 1e-12 ? sqrt(var) : 1.0);
}

// Xn[r][f] = (X[perm[r]][f] - mean[f]) / std[f]
__global__ void normalize_rows_kernel(const float* X, const int32_t* perm, int N, const float* mean,
                                      const float* std_, float* Xn) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * kFeat) return;
    const int r = idx / kFeat, f = idx % kFeat;
    Xn[idx] = (X[(size_t)perm[r] * kFeat + f] - mean[f]) / std_[f];
}

__global__ void gather_labels_kernel(const int32_t* y, const int32_t* perm, int N, int32_t* out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < N) out[r] = y[perm[r]];
}

int nblk(long long items, int threads = 256) { return (int)((items + threads - 1) / threads); }

// host helpers for bf16 (round to nearest even) -- conversion is done with
// the CUDA host intrinsics so that device and host agree
__nv_bfloat16 to_bf16(float x) { return __float2bfloat16_rn(x); }

cc_status upload_blob(const unsigned char* blob, size_t bytes, Model** slot, std::vector<unsigned char>* store) {
    if (bytes != kBlobBytes) return cc::set_error(CC_EINVAL, "cc_sched_load: expected %zu bytes, got %zu", kBlobBytes, bytes);
    BlobHeader h;
    std::memcpy(&h, blob, sizeof h);
    if (std::memcmp(h.magic, "CCMLP01", 8) != 0 || h.n_in != kFeat || h.n_hidden != kHidden || h.n_layers != 3 ||
        h.n_out != kOut)
        return cc::set_error(CC_EINVAL, "cc_sched_load: not a CCMLP01 12-64x3-18 weight blob");
    Model m;
    for (int f = 0; f < kFeat; ++f) {
        if (!(h.std_[f] > 0.f)) return cc::set_error(CC_EINVAL, "cc_sched_load: feature std must be > 0");
        m.mean[f] = h.mean[f];
        m.inv_std[f] = 1.f / h.std_[f];
    }
    const unsigned char* p = blob + sizeof h;
    auto take = [&](void* dst, size_t nbytes) {
        std::memcpy(dst, p, nbytes);
        p += nbytes;
    };
    take(m.w1, sizeof m.w1);
    take(m.b1, sizeof m.b1);
    take(m.w2, sizeof m.w2);
    take(m.b2, sizeof m.b2);
    take(m.w3, sizeof m.w3);
    take(m.b3, sizeof m.b3);
    take(m.w4, sizeof m.w4);
    take(m.b4, sizeof m.b4);
    // a feature pass of another handle may still be reading the old weights
    // on its side stream
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cc::cuda_fail(e, "cc_sched_load", __FILE__, __LINE__);
    if (!*slot) {
        e = cudaMalloc(slot, sizeof(Model));
        if (e != cudaSuccess) return cc::cuda_fail(e, "cc_sched_load", __FILE__, __LINE__);
    }
    e = cudaMemcpy(*slot, &m, sizeof m, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cc::cuda_fail(e, "cc_sched_load", __FILE__, __LINE__);
    store->assign(blob, blob + bytes);
    return CC_OK;
}

#define SCUDA(expr)                                                                  \
    do {                                                                             \
        cudaError_t e_ = (expr);                                                     \
        if (e_ != cudaSuccess) return cc::cuda_fail(e_, #expr, __FILE__, __LINE__); \
    } while (0)

}  // namespace

namespace cc {

// Device buffers of the scheduler for one graph handle or batch plan, kept
// for the handle's lifetime: offsets, features, classes and the per-vertex
// scratch of the feature kernel (zeroed once; the kernel leaves it zero).
struct SchedCtx {
    int32_t G = 0;
    int64_t* d_off = nullptr;  // off_v[G+1] then off_e[G+1]
    float* d_feat = nullptr;   // G x kFeat
    int32_t* d_cls = nullptr;  // G
    std::vector<int32_t> h_cls;  // host copy of the classes
    std::vector<int64_t> h_off;  // offsets of a single graph, sent before each feature pass
    long long version = -1;    // model version h_cls was computed with
    // single graphs: the feature pass runs on a stream of its own while the
    // first CC_ORDER_AUTO call solves with the default schedule
    void* block = nullptr;     // d_off, d_feat and d_cls of a single graph in one allocation
    cudaStream_t side = nullptr;
    cudaEvent_t ready = nullptr, done = nullptr;
    long long pending = -1;    // model version of a feature pass enqueued on side
};

void sched_ctx_free(SchedCtx* c) {
    if (!c) return;
    if (c->side) {
        cudaStreamSynchronize(c->side);  // a feature pass may still read the edges
        cudaStreamDestroy(c->side);
    }
    if (c->ready) cudaEventDestroy(c->ready);
    if (c->done) cudaEventDestroy(c->done);
    if (c->block) {
        cc::dfree(c->block, nullptr);  // the side stream has finished
    } else {
        cudaFree(c->d_off);
        cudaFree(c->d_feat);
        cudaFree(c->d_cls);
    }
    delete c;
}

}  // namespace cc

namespace {

// Process-wide feature scratch for up to g_scratch_ctas CTAs (guarded by g_mu).
struct Scratch {
    int ctas = 0;
    int32_t* keys = nullptr;
    int32_t* deg = nullptr;
    uint32_t* word = nullptr;
    int32_t* su = nullptr;
    int32_t* sv = nullptr;
    int32_t* owned = nullptr;
} g_scratch;

cc_status scratch_get(int ctas, cudaStream_t s) {
    if (g_scratch.ctas >= ctas) return CC_OK;
    cudaFree(g_scratch.keys);
    cudaFree(g_scratch.deg);
    cudaFree(g_scratch.word);
    cudaFree(g_scratch.su);
    cudaFree(g_scratch.sv);
    cudaFree(g_scratch.owned);
    g_scratch = Scratch();
    const size_t T = (size_t)ctas * kSlots, S = (size_t)ctas * kSample;
    cudaError_t e = cudaMalloc(&g_scratch.keys, T * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&g_scratch.deg, T * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&g_scratch.word, T * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&g_scratch.su, S * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&g_scratch.sv, S * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&g_scratch.owned, 2 * S * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(g_scratch.keys, 0xff, T * sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(g_scratch.deg, 0, T * sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(g_scratch.word, 0, T * sizeof(uint32_t), s);
    if (e != cudaSuccess) return cc::cuda_fail(e, "scheduler scratch", __FILE__, __LINE__);
    g_scratch.ctas = ctas;
    return CC_OK;
}

cc_status ctx_get(cc::SchedCtx** slot, int32_t G, const int64_t* off_v, const int64_t* off_e, cudaStream_t s) {
    if (*slot) return CC_OK;
    cc::SchedCtx* c = new (std::nothrow) cc::SchedCtx();
    if (!c) return cc::set_error(CC_ENOMEM, "scheduler context");
    c->G = G;
    if (G == 1) {
        // a handle has one graph: 4 offsets, the features and the class in
        // one small block, and a stream for the background feature pass
        cudaError_t e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cc::dmalloc(&c->block, 4 * sizeof(int64_t) + 16 * sizeof(float) + 4 * sizeof(int32_t), c->side);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ready, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->done, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            cc::sched_ctx_free(c);
            return cc::cuda_fail(e, "scheduler buffers", __FILE__, __LINE__);
        }
        c->d_off = static_cast<int64_t*>(c->block);
        c->d_feat = reinterpret_cast<float*>(c->d_off + 4);
        c->d_cls = reinterpret_cast<int32_t*>(c->d_feat + 16);
        c->h_cls.assign(1, 0);
        c->h_off = {off_v[0], off_v[1], off_e[0], off_e[1]};
        *slot = c;
        return CC_OK;
    }
    cudaError_t e = cudaMalloc(&c->d_off, 2 * (size_t)(G + 1) * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_feat, (size_t)std::max(G, 1) * kFeat * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_cls, (size_t)std::max(G, 1) * sizeof(int32_t));
    c->h_cls.assign((size_t)std::max(G, 1), 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_off, off_v, (G + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_off + G + 1, off_e, (G + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host offsets may be temporaries
    if (e != cudaSuccess) {
        cc::sched_ctx_free(c);
        return cc::cuda_fail(e, "scheduler context", __FILE__, __LINE__);
    }
    *slot = c;
    return CC_OK;
}

// Features of every graph of the context into c->d_feat (caller holds g_mu).
cc_status run_features(cc::SchedCtx* c, const int32_t* src, const int32_t* dst, cudaStream_t s,
                       long long m_feat = -1) {
    if (c->G == 0) return CC_OK;
    if (c->G == 1) {  // one graph: a cluster of 8 CTAs
        SCUDA(cudaMemcpyAsync(c->d_off, c->h_off.data(), 4 * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        // per device and cheap: set before every launch
        SCUDA(cudaFuncSetAttribute(features_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)sizeof(ClusterSmem)));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(kCl, 1, 1);
        cfg.blockDim = dim3(kFeatThreads, 1, 1);
        cfg.dynamicSmemBytes = sizeof(ClusterSmem);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = kCl;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        SCUDA(cudaLaunchKernelEx(&cfg, features_cluster_kernel, (const int64_t*)c->d_off,
                                 (const int64_t*)(c->d_off + 2), src, dst, m_feat, c->d_feat));
        return CC_OK;
    }
    const int grid = std::max(1, std::min<int>(c->G, cc::device_sms() * 2));
    cc_status st = scratch_get(grid, s);
    if (st != CC_OK) return st;
    FeatArgs a{c->G, c->d_off, c->d_off + c->G + 1, src, dst, g_scratch.keys, g_scratch.deg, g_scratch.word,
               g_scratch.su, g_scratch.sv, g_scratch.owned, c->d_feat};
    features_kernel<<<grid, kFeatThreads, 0, s>>>(a);
    SCUDA(cudaGetLastError());
    return CC_OK;
}

void decode(int32_t k, int* order, int* mode, int* c) {
    static const int orders[3] = {2, 4, CC_ORDER_FULL};
    static const int cs[3] = {1, 2, 4};
    *order = orders[(k / 6) % 3];
    *mode = (k / 3) % 2 ? CC_ASYNC : CC_SYNC;
    *c = cs[k % 3];
}

// predict classes for G feature rows already on the device
cc_status predict_device(const Model* model, const float* d_feats, int32_t G, int32_t* d_cls, float* d_logits,
                         cudaStream_t s) {
    mlp_infer_kernel<<<(G + 7) / 8, 256, 0, s>>>(model, d_feats, G, d_cls, d_logits);
    SCUDA(cudaGetLastError());
    return CC_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// internal entry points
// ---------------------------------------------------------------------------

// The feature pass of one handle (caller holds g_mu).  A native CSR handle
// first gathers kSample entries as (row, column) pairs; for a symmetric input
// every undirected edge is stored twice, so its edge count is nnz / 2.
static cc_status handle_features(cc_graph* g, cudaStream_t s) {
    long long n = 0, m = 0;
    cc::graph_nm(g, &n, &m);
    cc::SchedCtx** slot = cc::graph_sched_slot(g);
    const int layout = cc::graph_layout(g);
    if (layout == CC_COO && cc::graph_hubs(g) != nullptr) {  // hub-encoded edges: decode a sample
        const long long S = m < kSample ? m : kSample;
        const int64_t ov[2] = {0, n}, oe[2] = {0, S};
        cc_status st = ctx_get(slot, 1, ov, oe, s);
        if (st != CC_OK) return st;
        (*slot)->h_off = {0, n, 0, S};  // the feature pass reads the S decoded pairs
        int32_t* pairs = nullptr;
        SCUDA(cc::dmalloc(reinterpret_cast<void**>(&pairs), (size_t)(2 * S + 1) * sizeof(int32_t), s));
        cc::hub_sample_kernel<<<(int)((S + 255) / 256), 256, 0, s>>>(
            static_cast<const int32_t*>(cc::graph_src(g)), static_cast<const int32_t*>(cc::graph_dst(g)), m, S,
            cc::graph_hubs(g), pairs, pairs + S);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            cc::dfree(pairs, s);
            return cc::cuda_fail(e, "hub_sample_kernel", __FILE__, __LINE__);
        }
        st = run_features(*slot, pairs, pairs + S, s, m);
        cc::dfree(pairs, s);
        return st;
    }
    if (layout == CC_COO) {
        const int64_t ov[2] = {0, n}, oe[2] = {0, m};
        cc_status st = ctx_get(slot, 1, ov, oe, s);
        if (st != CC_OK) return st;
        (*slot)->h_off = {0, n, 0, m};
        return run_features(*slot, static_cast<const int32_t*>(cc::graph_src(g)),
                            static_cast<const int32_t*>(cc::graph_dst(g)), s);
    }
    const long long S = m < kSample ? m : kSample;
    const int64_t ov[2] = {0, n}, oe[2] = {0, S};
    cc_status st = ctx_get(slot, 1, ov, oe, s);
    if (st != CC_OK) return st;
    (*slot)->h_off = {0, n, 0, S};  // the feature pass reads the S sampled entries
    int32_t* pairs = nullptr;
    SCUDA(cc::dmalloc(reinterpret_cast<void**>(&pairs), (size_t)(2 * S + 1) * sizeof(int32_t), s));
    if (S > 0) {
        cc::csr_sample_kernel<<<(int)((S + 255) / 256), 256, 0, s>>>(
            cc::graph_csr_off(g), static_cast<const int32_t*>(cc::graph_dst(g)), n, m, S, pairs, pairs + S);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            cc::dfree(pairs, s);
            return cc::cuda_fail(e, "csr_sample_kernel", __FILE__, __LINE__);
        }
    }
    st = run_features(*slot, pairs, pairs + S, s, layout == CC_CSR_NATIVE_SYM ? m / 2 : m);
    cc::dfree(pairs, s);
    return st;
}

namespace cc {

cc_status resolve_schedule(cc_graph* g, int* order, int* mode, int* c, bool* deferred) {
    std::lock_guard<std::mutex> lock(g_mu);
    const int want_c = *c;
    if (!g_model) {  // plain order-2 synchronous schedule
        *order = 2;
        *mode = CC_SYNC;
        *c = want_c < 1 ? 1 : want_c;
        return CC_OK;
    }
    if (graph_id_bits(g) != 32) {  // the feature kernel reads int32 ids
        *order = CC_ORDER_FULL;
        *mode = CC_ASYNC;
        *c = want_c < 1 ? 1 : want_c;
        return CC_OK;
    }
    // The edges of a handle never change: the choice is made once per model.
    // The first call does not wait for it: it solves with the paper's default
    // C-2 (order 2, asynchronous) and asks the caller to enqueue the feature
    // pass and the inference behind the solve (sched_defer_features); the
    // next call takes the predicted schedule.  Every schedule returns the
    // same labels.
    SchedCtx** slot = graph_sched_slot(g);
    SchedCtx* x = *slot;
    if (!x || (x->version != g_model_version && x->pending != g_model_version)) {
        *order = 2;
        *mode = CC_ASYNC;
        *c = want_c < 1 ? 1 : want_c;
        if (deferred) *deferred = true;
        return CC_OK;
    }
    if (x->version != g_model_version) {  // the feature pass enqueued by an earlier call
        cudaError_t e = cudaMemcpyAsync(x->h_cls.data(), x->d_cls, sizeof(int32_t), cudaMemcpyDeviceToHost, x->side);
        if (e == cudaSuccess) e = cudaStreamSynchronize(x->side);
        if (e != cudaSuccess) return cuda_fail(e, "sched", __FILE__, __LINE__);
        x->version = g_model_version;
    }
    int cc_ = 1;
    decode(x->h_cls[0], order, mode, &cc_);
    *c = want_c >= 1 ? want_c : cc_;
    return CC_OK;
}

// The feature pass and the inference of a handle, on the handle's own
// stream, ordered after everything the caller has enqueued on s so far (the
// solve of the first CC_ORDER_AUTO call): they run after that solve on the
// GPU, and the host returns without waiting for them.
cc_status sched_defer_features(cc_graph* g, cudaStream_t s) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_model) return CC_OK;
    SchedCtx** slot = graph_sched_slot(g);
    if (!*slot) {
        long long n = 0, m = 0;
        graph_nm(g, &n, &m);
        const int64_t ov[2] = {0, n}, oe[2] = {0, m};
        cc_status st = ctx_get(slot, 1, ov, oe, s);
        if (st != CC_OK) return st;
    }
    SchedCtx* x = *slot;
    if (x->pending == g_model_version || x->version == g_model_version) return CC_OK;
    cudaError_t e = cudaEventRecord(x->ready, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(x->side, x->ready, 0);
    if (e != cudaSuccess) return cuda_fail(e, "sched", __FILE__, __LINE__);
    cc_status st = handle_features(g, x->side);
    if (st == CC_OK) st = predict_device(g_model, x->d_feat, 1, x->d_cls, nullptr, x->side);
    if (st != CC_OK) return st;
    e = cudaEventRecord(x->done, x->side);
    if (e != cudaSuccess) return cuda_fail(e, "sched", __FILE__, __LINE__);
    x->pending = g_model_version;
    return CC_OK;
}

cc_status batch_resolve_schedule(cc_batch_plan* b, int mode, int c) {
    (void)mode;
    const int32_t G = batch_graph_count(b);
    std::vector<int32_t> h(G, 2), sync(G, 1), cv(G, c < 1 ? 1 : c);
    std::lock_guard<std::mutex> lock(g_mu);
    // weights trained for batched solves when loaded, else the single-graph ones
    const Model* model = g_model_batch ? g_model_batch : g_model;
    if (model && G > 0) {
        cudaStream_t s = batch_stream(b);
        SchedCtx** slot = batch_sched_slot(b);
        cc_status st = ctx_get(slot, G, batch_off_v(b), batch_off_e(b), s);
        if (st != CC_OK) return st;
        SchedCtx* x = *slot;
        if (x->version != g_model_version) {
            st = run_features(x, batch_src(b), batch_dst(b), s);
            if (st == CC_OK) st = predict_device(model, x->d_feat, G, x->d_cls, nullptr, s);
            if (st == CC_OK) {
                cudaError_t e = cudaMemcpyAsync(x->h_cls.data(), x->d_cls, G * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) st = cuda_fail(e, "batch sched", __FILE__, __LINE__);
            }
            if (st != CC_OK) return st;
            x->version = g_model_version;
        }
        for (int32_t g = 0; g < G; ++g) {
            int o, md, ci;
            decode(x->h_cls[g], &o, &md, &ci);
            h[g] = o == CC_ORDER_FULL ? CC_MAX_ORDER : o;
            sync[g] = md == CC_SYNC;
            // in a batch the convergence check is shared by all graphs of a
            // round (and free in the shared-memory path), so the interval the
            // model learned from single-graph runs -- where it saves check
            // launches -- would only add sweeps: check every sweep
            (void)ci;
            cv[g] = c >= 1 ? c : 1;
        }
    }
    batch_set_schedule(b, h.data(), sync.data(), cv.data());
    return CC_OK;
}

}  // namespace cc

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

static cc_status load_into(const void* weights, size_t bytes, Model** slot, std::vector<unsigned char>* store) {
    std::lock_guard<std::mutex> lock(g_mu);
    ++g_model_version;
    if (!weights) {
        if (*slot) cudaFree(*slot);  // waits for work that may still read it
        *slot = nullptr;
        store->clear();
        return CC_OK;
    }
    return upload_blob(static_cast<const unsigned char*>(weights), bytes, slot, store);
}

extern "C" cc_status cc_sched_load(const void* weights, size_t bytes) {
    return load_into(weights, bytes, &g_model, &g_blob);
}

extern "C" cc_status cc_sched_load_batch(const void* weights, size_t bytes) {
    return load_into(weights, bytes, &g_model_batch, &g_blob_batch);
}

extern "C" size_t cc_sched_blob_bytes(void) { return kBlobBytes; }

extern "C" cc_status cc_sched_decode(int32_t cls, int* order, int* mode, int* check_interval) {
    if (cls < 0 || cls >= kOut || !order || !mode || !check_interval)
        return cc::set_error(CC_EINVAL, "cc_sched_decode: class must be 0..%d", kOut - 1);
    decode(cls, order, mode, check_interval);
    return CC_OK;
}

extern "C" cc_status cc_graph_features(cc_graph* g, float* features_out) {
    if (!g || !features_out) return cc::set_error(CC_EINVAL, "cc_graph_features: NULL argument");
    if (cc::graph_id_bits(g) != 32) return cc::set_error(CC_EINVAL, "cc_graph_features: int32 ids only");
    // the feature scratch is shared: each use completes before the lock is released
    std::lock_guard<std::mutex> lock(g_mu);
    cudaStream_t s = cc::graph_stream(g);
    cc::SchedCtx** slot = cc::graph_sched_slot(g);
    if (*slot && (*slot)->side) {  // a background feature pass writes the same buffers
        cudaError_t e = cudaStreamSynchronize((*slot)->side);
        if (e != cudaSuccess) return cc::cuda_fail(e, "cc_graph_features", __FILE__, __LINE__);
    }
    cc_status st = handle_features(g, s);
    if (st != CC_OK) return st;
    cudaError_t e = cudaMemcpyAsync(features_out, (*slot)->d_feat, kFeat * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cc::cuda_fail(e, "cc_graph_features", __FILE__, __LINE__);
    return CC_OK;
}

extern "C" cc_status cc_batch_features(cc_batch_plan* b, float* features_out) {
    if (!b || !features_out) return cc::set_error(CC_EINVAL, "cc_batch_features: NULL argument");
    const int32_t G = cc::batch_graph_count(b);
    if (G == 0) return CC_OK;
    std::lock_guard<std::mutex> lock(g_mu);
    cudaStream_t s = cc::batch_stream(b);
    cc::SchedCtx** slot = cc::batch_sched_slot(b);
    cc_status st = ctx_get(slot, G, cc::batch_off_v(b), cc::batch_off_e(b), s);
    if (st != CC_OK) return st;
    st = run_features(*slot, cc::batch_src(b), cc::batch_dst(b), s);
    if (st != CC_OK) return st;
    cudaError_t e = cudaMemcpyAsync(features_out, (*slot)->d_feat, (size_t)G * kFeat * sizeof(float),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cc::cuda_fail(e, "cc_batch_features", __FILE__, __LINE__);
    return CC_OK;
}

static cc_status predict_host(const float* features, int32_t count, int32_t* cls_out, float* logits_out,
                              bool batch_model) {
    if (count < 0 || (count > 0 && (!features || !cls_out))) return cc::set_error(CC_EINVAL, "cc_sched_predict: bad arguments");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!(batch_model ? g_model_batch : g_model))
        return cc::set_error(CC_EINVAL, "cc_sched_predict: no scheduler weights loaded");
    if (count == 0) return CC_OK;
    float* d_f = nullptr;
    int32_t* d_c = nullptr;
    float* d_l = nullptr;
    SCUDA(cudaMalloc(&d_f, (size_t)count * kFeat * sizeof(float)));
    cudaError_t e = cudaMalloc(&d_c, (size_t)count * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&d_l, (size_t)count * kOut * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(d_f, features, (size_t)count * kFeat * sizeof(float), cudaMemcpyHostToDevice);
    cc_status st = e == cudaSuccess ? CC_OK : cc::cuda_fail(e, "cc_sched_predict", __FILE__, __LINE__);
    if (st == CC_OK) st = predict_device(batch_model ? g_model_batch : g_model, d_f, count, d_c, d_l, nullptr);
    if (st == CC_OK) {
        e = cudaMemcpy(cls_out, d_c, (size_t)count * sizeof(int32_t), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && logits_out)
            e = cudaMemcpy(logits_out, d_l, (size_t)count * kOut * sizeof(float), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = cc::cuda_fail(e, "cc_sched_predict", __FILE__, __LINE__);
    }
    cudaFree(d_f);
    cudaFree(d_c);
    cudaFree(d_l);
    return st;
}

extern "C" cc_status cc_sched_predict(const float* features, int32_t count, int32_t* cls_out, float* logits_out) {
    return predict_host(features, count, cls_out, logits_out, false);
}

extern "C" cc_status cc_sched_predict_batch(const float* features, int32_t count, int32_t* cls_out,
                                            float* logits_out) {
    return predict_host(features, count, cls_out, logits_out, true);
}

// Train the MLP from scratch (or from init_blob) on N labelled feature rows;
// writes a CCMLP01 blob (BF16 weights) of cc_sched_blob_bytes() bytes.
extern "C" cc_status cc_sched_train(const float* features, const int32_t* labels, int32_t N,
                                    const float* init_params, int32_t epochs, int32_t batch, float lr,
                                    uint64_t seed, void* blob_out, float* final_loss) {
    if (N <= 0 || !features || !labels || !blob_out || epochs < 1 || batch < 1)
        return cc::set_error(CC_EINVAL, "cc_sched_train: bad arguments");
    for (int32_t i = 0; i < N; ++i)
        if (labels[i] < 0 || labels[i] >= kOut) return cc::set_error(CC_EINVAL, "cc_sched_train: label %d out of range", i);
    const int B = std::min(batch, N);
    // fp32 master parameters: [W1 b1 W2 b2 W3 b3 W4 b4]
    std::vector<float> P(kParams);
    if (init_params) {
        std::copy(init_params, init_params + kParams, P.begin());
    } else {
        // He-uniform initialisation from SplitMix64 (Steele, Lea, Flood 2014)
        uint64_t st_ = seed;
        auto next = [&]() {
            st_ += 0x9E3779B97F4A7C15ull;
            uint64_t z = st_;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            return z ^ (z >> 31);
        };
        size_t off = 0;
        for (int l = 0; l < 4; ++l) {
            const int ni = kIn[l], no = kOutDim[l];
            const float lim = std::sqrt(6.f / (float)ni);
            for (int i = 0; i < no * ni; ++i) {
                const double u = (double)(next() >> 11) / (double)(1ull << 53);
                P[off + i] = (float)((2.0 * u - 1.0) * lim);
            }
            off += (size_t)no * ni;
            for (int i = 0; i < no; ++i) P[off + i] = 0.f;
            off += no;
        }
    }
    float *d_P, *d_G, *d_m1, *d_m2, *d_X, *d_Xn, *d_buf, *d_stats, *d_loss;
    int32_t *d_y, *d_yb, *d_perm;
    SCUDA(cudaMalloc(&d_P, 4 * (size_t)kParams * sizeof(float)));
    d_G = d_P + kParams;
    d_m1 = d_G + kParams;
    d_m2 = d_m1 + kParams;
    SCUDA(cudaMemset(d_m1, 0, 2 * (size_t)kParams * sizeof(float)));
    SCUDA(cudaMemcpy(d_P, P.data(), kParams * sizeof(float), cudaMemcpyHostToDevice));
    SCUDA(cudaMalloc(&d_X, 2 * (size_t)N * kFeat * sizeof(float)));
    d_Xn = d_X + (size_t)N * kFeat;
    SCUDA(cudaMemcpy(d_X, features, (size_t)N * kFeat * sizeof(float), cudaMemcpyHostToDevice));
    SCUDA(cudaMalloc(&d_y, 3 * (size_t)N * sizeof(int32_t)));
    d_yb = d_y + N;
    d_perm = d_yb + N;
    SCUDA(cudaMemcpy(d_y, labels, (size_t)N * sizeof(int32_t), cudaMemcpyHostToDevice));
    // activations: Z1 A1 Z2 A2 Z3 A3 Z4 dZ4 dA3 dA2 dA1 (B x 64 each, generous)
    const size_t act = (size_t)B * kHidden;
    SCUDA(cudaMalloc(&d_buf, 11 * act * sizeof(float)));
    SCUDA(cudaMalloc(&d_stats, (2 * kFeat + 1) * sizeof(float)));
    d_loss = d_stats + 2 * kFeat;
    feat_stats_kernel<<<1, 32>>>(d_X, N, d_stats, d_stats + kFeat);
    float* Z1 = d_buf;
    float* A1 = Z1 + act;
    float* Z2 = A1 + act;
    float* A2 = Z2 + act;
    float* Z3 = A2 + act;
    float* A3 = Z3 + act;
    float* Z4 = A3 + act;
    float* dZ4 = Z4 + act;
    float* dZ3 = dZ4 + act;
    float* dZ2 = dZ3 + act;
    float* dZ1 = dZ2 + act;
    float* w[4];
    float* bb[4];
    float* gw[4];
    float* gb[4];
    {
        size_t off = 0;
        for (int l = 0; l < 4; ++l) {
            w[l] = d_P + off;
            gw[l] = d_G + off;
            off += (size_t)kIn[l] * kOutDim[l];
            bb[l] = d_P + off;
            gb[l] = d_G + off;
            off += kOutDim[l];
        }
    }
    // epoch order: SplitMix64-keyed shuffle on the host (plumbing, not the model)
    std::vector<int32_t> perm(N);
    std::vector<uint64_t> key(N);
    int t = 0;
    float loss_h = 0.f;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int32_t i = 0; i < N; ++i) {
            uint64_t z = seed + 0x632BE59BD9B4E019ull * (uint64_t)(ep + 1) + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            key[i] = z ^ (z >> 31);
            perm[i] = i;
        }
        if (epochs > 1 || B < N)
            std::sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b2) { return key[a] < key[b2] || (key[a] == key[b2] && a < b2); });
        SCUDA(cudaMemcpy(d_perm, perm.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice));
        normalize_rows_kernel<<<nblk((long long)N * kFeat), 256>>>(d_X, d_perm, N, d_stats, d_stats + kFeat, d_Xn);
        gather_labels_kernel<<<nblk(N), 256>>>(d_y, d_perm, N, d_yb);
        SCUDA(cudaMemset(d_loss, 0, sizeof(float)));
        for (int32_t s0 = 0; s0 + B <= N; s0 += B) {
            const float* X = d_Xn + (size_t)s0 * kFeat;
            const int32_t* y = d_yb + s0;
            dense_fwd_kernel<<<nblk(B * kHidden), 256>>>(w[0], bb[0], X, kFeat, kHidden, B, Z1, A1, 1);
            dense_fwd_kernel<<<nblk(B * kHidden), 256>>>(w[1], bb[1], A1, kHidden, kHidden, B, Z2, A2, 1);
            dense_fwd_kernel<<<nblk(B * kHidden), 256>>>(w[2], bb[2], A2, kHidden, kHidden, B, Z3, A3, 1);
            dense_fwd_kernel<<<nblk(B * kOut), 256>>>(w[3], bb[3], A3, kHidden, kOut, B, Z4, nullptr, 0);
            softmax_ce_kernel<<<nblk(B), 256>>>(Z4, y, B, dZ4, d_loss);
            dense_grad_kernel<<<nblk(kOut * kHidden), 256>>>(dZ4, A3, kHidden, kOut, B, gw[3], gb[3]);
            dense_bwd_input_kernel<<<nblk(B * kHidden), 256>>>(w[3], dZ4, Z3, kHidden, kOut, B, dZ3);
            dense_grad_kernel<<<nblk(kHidden * kHidden), 256>>>(dZ3, A2, kHidden, kHidden, B, gw[2], gb[2]);
            dense_bwd_input_kernel<<<nblk(B * kHidden), 256>>>(w[2], dZ3, Z2, kHidden, kHidden, B, dZ2);
            dense_grad_kernel<<<nblk(kHidden * kHidden), 256>>>(dZ2, A1, kHidden, kHidden, B, gw[1], gb[1]);
            dense_bwd_input_kernel<<<nblk(B * kHidden), 256>>>(w[1], dZ2, Z1, kHidden, kHidden, B, dZ1);
            dense_grad_kernel<<<nblk(kHidden * kFeat), 256>>>(dZ1, X, kFeat, kHidden, B, gw[0], gb[0]);
            ++t;
            adam_kernel<<<nblk(kParams), 256>>>(d_P, d_G, d_m1, d_m2, kParams, lr, 0.9f, 0.999f, 1e-8f, t);
        }
        SCUDA(cudaGetLastError());
    }
    SCUDA(cudaMemcpy(&loss_h, d_loss, sizeof(float), cudaMemcpyDeviceToHost));
    SCUDA(cudaMemcpy(P.data(), d_P, kParams * sizeof(float), cudaMemcpyDeviceToHost));
    float stats[2 * kFeat];
    SCUDA(cudaMemcpy(stats, d_stats, sizeof stats, cudaMemcpyDeviceToHost));
    cudaFree(d_P);
    cudaFree(d_X);
    cudaFree(d_y);
    cudaFree(d_buf);
    cudaFree(d_stats);
    if (final_loss) *final_loss = loss_h / (float)std::max(1, N / B);
    // blob: header, then per layer bf16 weights and fp32 biases
    unsigned char* out = static_cast<unsigned char*>(blob_out);
    BlobHeader h = {};
    std::memcpy(h.magic, "CCMLP01", 8);
    h.n_in = kFeat;
    h.n_hidden = kHidden;
    h.n_layers = 3;
    h.n_out = kOut;
    std::memcpy(h.mean, stats, sizeof h.mean);
    std::memcpy(h.std_, stats + kFeat, sizeof h.std_);
    std::memcpy(out, &h, sizeof h);
    unsigned char* p = out + sizeof h;
    size_t off = 0;
    for (int l = 0; l < 4; ++l) {
        const int nw = kIn[l] * kOutDim[l];
        for (int i = 0; i < nw; ++i) {
            const __nv_bfloat16 v = to_bf16(P[off + i]);
            std::memcpy(p, &v, 2);
            p += 2;
        }
        off += nw;
        std::memcpy(p, P.data() + off, kOutDim[l] * sizeof(float));
        p += kOutDim[l] * sizeof(float);
        off += kOutDim[l];
    }
    return CC_OK;
}

// One optimiser step exposed for testing: returns the updated fp32 parameters.
extern "C" cc_status cc_sched_train_step(const float* features_norm, const int32_t* labels, int32_t B,
                                         float* params_inout, float lr, float* loss_out) {
    if (B <= 0 || !features_norm || !labels || !params_inout) return cc::set_error(CC_EINVAL, "cc_sched_train_step: bad arguments");
    float *d_P, *d_G, *d_m, *d_X, *d_buf, *d_loss;
    int32_t* d_y;
    SCUDA(cudaMalloc(&d_P, 4 * (size_t)kParams * sizeof(float)));
    d_G = d_P + kParams;
    d_m = d_G + kParams;
    SCUDA(cudaMemset(d_m, 0, 2 * (size_t)kParams * sizeof(float)));
    SCUDA(cudaMemcpy(d_P, params_inout, kParams * sizeof(float), cudaMemcpyHostToDevice));
    SCUDA(cudaMalloc(&d_X, (size_t)B * kFeat * sizeof(float)));
    SCUDA(cudaMemcpy(d_X, features_norm, (size_t)B * kFeat * sizeof(float), cudaMemcpyHostToDevice));
    SCUDA(cudaMalloc(&d_y, (size_t)B * sizeof(int32_t)));
    SCUDA(cudaMemcpy(d_y, labels, (size_t)B * sizeof(int32_t), cudaMemcpyHostToDevice));
    const size_t act = (size_t)B * kHidden;
    SCUDA(cudaMalloc(&d_buf, (11 * act + 1) * sizeof(float)));
    d_loss = d_buf + 11 * act;
    SCUDA(cudaMemset(d_loss, 0, sizeof(float)));
    float* Z1 = d_buf;
    float* A1 = Z1 + act;
    float* Z2 = A1 + act;
    float* A2 = Z2 + act;
    float* Z3 = A2 + act;
    float* A3 = Z3 + act;
    float* Z4 = A3 + act;
    float* dZ4 = Z4 + act;
    float* dZ3 = dZ4 + act;
    float* dZ2 = dZ3 + act;
    float* dZ1 = dZ2 + act;
    float *w[4], *bb[4], *gw[4], *gb[4];
    size_t off = 0;
    for (int l = 0; l < 4; ++l) {
        w[l] = d_P + off;
        gw[l] = d_G + off;
        off += (size_t)kIn[l] * kOutDim[l];
        bb[l] = d_P + off;
        gb[l] = d_G + off;
        off += kOutDim[l];
    }
    dense_fwd_kernel<<<nblk(B * kHidden), 256>>>(w[0], bb[0], d_X, kFeat, kHidden, B, Z1, A1, 1);
    dense_fwd_kernel<<<nblk(B * kHidden), 256>>>(w[1], bb[1], A1, kHidden, kHidden, B, Z2, A2, 1);
    dense_fwd_kernel<<<nblk(B * kHidden), 256>>>(w[2], bb[2], A2, kHidden, kHidden, B, Z3, A3, 1);
    dense_fwd_kernel<<<nblk(B * kOut), 256>>>(w[3], bb[3], A3, kHidden, kOut, B, Z4, nullptr, 0);
    softmax_ce_kernel<<<nblk(B), 256>>>(Z4, d_y, B, dZ4, d_loss);
    dense_grad_kernel<<<nblk(kOut * kHidden), 256>>>(dZ4, A3, kHidden, kOut, B, gw[3], gb[3]);
    dense_bwd_input_kernel<<<nblk(B * kHidden), 256>>>(w[3], dZ4, Z3, kHidden, kOut, B, dZ3);
    dense_grad_kernel<<<nblk(kHidden * kHidden), 256>>>(dZ3, A2, kHidden, kHidden, B, gw[2], gb[2]);
    dense_bwd_input_kernel<<<nblk(B * kHidden), 256>>>(w[2], dZ3, Z2, kHidden, kHidden, B, dZ2);
    dense_grad_kernel<<<nblk(kHidden * kHidden), 256>>>(dZ2, A1, kHidden, kHidden, B, gw[1], gb[1]);
    dense_bwd_input_kernel<<<nblk(B * kHidden), 256>>>(w[1], dZ2, Z1, kHidden, kHidden, B, dZ1);
    dense_grad_kernel<<<nblk(kHidden * kFeat), 256>>>(dZ1, d_X, kFeat, kHidden, B, gw[0], gb[0]);
    adam_kernel<<<nblk(kParams), 256>>>(d_P, d_G, d_m, d_m + kParams, kParams, lr, 0.9f, 0.999f, 1e-8f, 1);
    SCUDA(cudaGetLastError());
    SCUDA(cudaMemcpy(params_inout, d_P, kParams * sizeof(float), cudaMemcpyDeviceToHost));
    if (loss_out) SCUDA(cudaMemcpy(loss_out, d_loss, sizeof(float), cudaMemcpyDeviceToHost));
    cudaFree(d_P);
    cudaFree(d_X);
    cudaFree(d_y);
    cudaFree(d_buf);
    return CC_OK;
}

extern "C" int32_t cc_sched_param_count(void) { return kParams; }
