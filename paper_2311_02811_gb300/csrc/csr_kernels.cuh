// Sweep over a graph kept in CSR form (int32 ids): the rows are walked
// directly instead of being expanded into a per-entry row array.
//
// Entry k of row r (off[r] <= k < off[r+1]) is the edge <r, cols[k]>.  The
// entries are taken in groups of 4 (one 16-byte load of cols); seg[q] holds
// the row of entry 4q, computed once per handle, and the rows of the other
// three entries follow by stepping over off[] (rows are sorted, so the step
// reads the next offsets, which neighbouring threads read as well).  Each
// group is then four ordinary edges for the operator of mm_kernels.cuh.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mm_kernels.cuh"

namespace cc {

constexpr int kCsrGroup = 4;  // entries per 16-byte column load, one seg entry each

// seg[q] = the row r with off[r] <= 4q < off[r+1] (off non-decreasing, off[0] = 0,
// off[n] = nnz, validated before this runs).
static __global__ void csr_seg_rows_kernel(const int64_t* off, int64_t n, int64_t nnz, int32_t* seg) {
    const int64_t groups = (nnz + kCsrGroup - 1) / kCsrGroup;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < groups; q += stride) {
        const int64_t e = q * kCsrGroup;
        int64_t lo = 0, hi = n;  // largest r < n with off[r] <= e
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (off[mid] <= e) lo = mid; else hi = mid;
        }
        seg[q] = (int32_t)lo;
    }
}

// One sweep of MM^h (H > 0: fixed order; H = 0: run-time order h) over the
// CSR entries.  sym != 0: only entries with cols[k] < r are applied (a
// symmetric input then applies every undirected edge once).  Entries that are
// not applied become the self-loop <0, 0>, which never writes (L[0] == 0).
// first / gate / flag as in mm_sweep_kernel.
template <int H, bool SYNC>
__global__ void __launch_bounds__(256)
csr_sweep_kernel(const int64_t* __restrict__ off, const int32_t* __restrict__ cols,
                 const int32_t* __restrict__ seg, int64_t nnz, int32_t* L, int32_t* Lu, int h,
                 int32_t* flag, const Ctl* ctl, int first, int gate, int sym) {
    if (gate != 0 && ctl->sched_h != gate) return;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t groups = (nnz + kCsrGroup - 1) / kCsrGroup;
    const int64_t full = nnz / kCsrGroup;
    const bool ident = first == 2 || (first == 1 && ctl->sweeps == 0 && ctl->fresh != 0);
    int32_t* target = SYNC ? Lu : L;
    bool viol = false;
    for (int64_t q = tid; q < groups; q += stride) {
        int32_t c[kCsrGroup], r[kCsrGroup];
        const int64_t e0 = q * kCsrGroup;
        if (q < full) {
            load4(cols + e0, c);
        } else {
#pragma unroll
            for (int k = 0; k < kCsrGroup; ++k) c[k] = (e0 + k < nnz) ? __ldcs(cols + e0 + k) : 0;
        }
        int32_t row = __ldcs(seg + q);
        int64_t next = __ldg(off + row + 1);
#pragma unroll
        for (int k = 0; k < kCsrGroup; ++k) {
            const int64_t e = e0 + k;
            bool use = e < nnz;
            if (use) {
                while (e >= next) {  // ends at the entry's row: off[n] = nnz > e
                    ++row;
                    next = __ldg(off + row + 1);
                }
                use = !sym || c[k] < row;
            }
            r[k] = use ? row : 0;
            if (!use) c[k] = 0;
        }
        if (ident) {
#pragma unroll
            for (int k = 0; k < kCsrGroup; ++k) viol |= identity_pair(r[k], c[k], target);
        } else if constexpr (H > 0) {
            viol |= mm_fixed<H, SYNC, kCsrGroup>(r, c, L, Lu);
        } else {
            viol |= mm_runtime_ilp<SYNC, kCsrGroup>(r, c, h, L, Lu);
        }
    }
    if (flag != nullptr) {
        if (__syncthreads_or(viol) && threadIdx.x == 0) *flag = 1;
    }
}

// The (row, column) pairs of S entries spread evenly over the nnz entries
// (entry floor(j * nnz / S) for j < S), oriented so that the smaller id comes
// first, for the scheduler's feature pass.
static __global__ void csr_sample_kernel(const int64_t* off, const int32_t* cols, int64_t n, int64_t nnz,
                                         int64_t S, int32_t* su, int32_t* sv) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < S; j += stride) {
        const int64_t e = (nnz <= S) ? j : (j * nnz) / S;
        int64_t lo = 0, hi = n;
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (off[mid] <= e) lo = mid; else hi = mid;
        }
        const int32_t a = (int32_t)lo, b = cols[e];
        su[j] = a < b ? a : b;
        sv[j] = a < b ? b : a;
    }
}

}  // namespace cc
