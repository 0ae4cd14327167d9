// cc_run_noalloc: the Contour run for callers that must not allocate device
// memory (see include/contour.h).  Everything the run needs beyond the
// caller's edges and labels -- the control words (convergence flag,
// validation counters) and, for synchronous runs, the update array L_u --
// lives in one file-scope device array of fixed size.  No cudaMalloc,
// cudaFree, graph instantiation or other allocating call is made.
#include <cuda_runtime.h>

#include "../../include/contour.h"
#include "cc_internal.h"
#include "mm_kernels.cuh"

using cc::Ctl;

namespace {

constexpr size_t kCtlBytes = 256;  // control block, padded to keep L_u 256-byte aligned
static_assert(sizeof(Ctl) <= kCtlBytes, "control block does not fit its slot");

// Shared by every call in the process on a given device; holds the last
// call's contents.  The symbol named here is a host-side stand-in: host code
// obtains the device address with cudaGetSymbolAddress (scratch_for_device).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kCtlBytes + 4ull * CC_NOALLOC_MAX_N];

// Device address of the scratch array on the current device.  Looked up on
// every call (cudaGetSymbolAddress allocates nothing): a cached address would
// dangle after cudaDeviceReset or a new primary context reloads the module.
// The first lookup on a device loads the library's device code there.
cc_status scratch_for_device(unsigned char** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cc::cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
    *out = static_cast<unsigned char*>(p);
    return CC_OK;
}

// A kernel handed a host address faults (or, where the GPU can reach host
// memory, silently works on the wrong memory): accept only memory of the
// current device (device or managed allocations).  cudaPointerGetAttributes
// allocates nothing.
cc_status check_device_ptr(const void* p, const char* what) {
    if (!p) return CC_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cc::cuda_fail(e, "cudaGetDevice", __FILE__, __LINE__);
    cudaPointerAttributes a = {};
    e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cc::set_error(CC_EINVAL, "cc_run_noalloc: %s is not a CUDA pointer (%s)", what, cudaGetErrorString(e));
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return cc::set_error(CC_EINVAL, "cc_run_noalloc: %s is not device memory", what);
    if (a.type == cudaMemoryTypeDevice && a.device != dev)
        return cc::set_error(CC_EINVAL, "cc_run_noalloc: %s lives on device %d, the current device is %d", what,
                             a.device, dev);
    return CC_OK;
}

__global__ void noalloc_mark_converged(Ctl* ctl) {
    if (threadIdx.x == 0) ctl->converged = 1;
}

constexpr int kThreads = 256;

template <typename K>
int grid_for(K kernel, int64_t items) {
    const int cap = cc::persistent_blocks(reinterpret_cast<const void*>(kernel), kThreads, 0);
    int64_t need = (items + kThreads - 1) / kThreads;
    if (need < 1) need = 1;
    return (int)(need < cap ? need : cap);
}

template <int H, bool SYNC>
void sweep_t(const int32_t* src, const int32_t* dst, int64_t m, int32_t* L, int32_t* Lu, int h,
             int32_t* flag, int first, cudaStream_t s) {
    constexpr int G = (H == 1) ? 2 : 1;
    auto k = cc::mm_sweep_kernel<H, SYNC, G, int32_t>;
    k<<<grid_for(k, m / (4 * G) + 1), kThreads, 0, s>>>(src, dst, m, L, Lu, h, flag, nullptr, first, 0);
}

// first == 2 selects the identity sweep (the run's first sweep); 0 otherwise.
template <bool SYNC>
void sweep(int order, const int32_t* src, const int32_t* dst, int64_t m, int32_t* L, int32_t* Lu,
           int32_t* flag, int first, cudaStream_t s) {
    switch (order) {
        case 1: sweep_t<1, SYNC>(src, dst, m, L, Lu, 1, flag, first, s); break;
        case 2: sweep_t<2, SYNC>(src, dst, m, L, Lu, 2, flag, first, s); break;
        case 4: sweep_t<4, SYNC>(src, dst, m, L, Lu, 4, flag, first, s); break;
        case CC_ORDER_FULL: sweep_t<0, SYNC>(src, dst, m, L, Lu, cc::kFullChainHops, flag, first, s); break;
        default: sweep_t<0, SYNC>(src, dst, m, L, Lu, order, flag, first, s); break;
    }
}

#define NA_CUDA(expr)                                                           \
    do {                                                                        \
        cudaError_t e_ = (expr);                                                \
        if (e_ != cudaSuccess) return cc::cuda_fail(e_, #expr, __FILE__, __LINE__); \
    } while (0)

}  // namespace

extern "C" cc_status cc_run_noalloc(int64_t n, const int32_t* src, const int32_t* dst, int64_t m,
                                    int order, int mode, int check_interval, int32_t max_sweeps,
                                    int32_t* labels_out, int32_t* sweeps_out, void* cuda_stream) {
    if (n < 0 || m < 0) return cc::set_error(CC_EINVAL, "cc_run_noalloc: negative n or m");
    if (n > 0x7fffffffLL) return cc::set_error(CC_EINVAL, "cc_run_noalloc: n must be below 2^31 (int32 ids)");
    if (m > 0 && (!src || !dst)) return cc::set_error(CC_EINVAL, "cc_run_noalloc: edge arrays are NULL");
    if (n > 0 && !labels_out) return cc::set_error(CC_EINVAL, "cc_run_noalloc: labels_out is NULL");
    if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst) |
          reinterpret_cast<uintptr_t>(labels_out)) & 15) != 0)
        return cc::set_error(CC_EINVAL, "cc_run_noalloc: src, dst and labels_out must be 16-byte aligned device pointers");
    if (order < 0 || order > CC_MAX_ORDER) return cc::set_error(CC_EINVAL, "cc_run_noalloc: order must be 1..%d or CC_ORDER_FULL", CC_MAX_ORDER);
    if (mode != CC_SYNC && mode != CC_ASYNC) return cc::set_error(CC_EINVAL, "cc_run_noalloc: bad mode");
    if (check_interval < 1 || check_interval > 64) return cc::set_error(CC_EINVAL, "cc_run_noalloc: check_interval must be 1..64");
    if (max_sweeps < 1) return cc::set_error(CC_EINVAL, "cc_run_noalloc: max_sweeps must be >= 1");
    if (mode == CC_SYNC && n > CC_NOALLOC_MAX_N)
        return cc::set_error(CC_EINVAL,
                             "cc_run_noalloc: synchronous mode keeps L_u in a fixed scratch array of %d labels; n = %lld is larger",
                             CC_NOALLOC_MAX_N, (long long)n);
    if (sweeps_out) *sweeps_out = 0;
    if (n == 0) return CC_OK;

    cc_status st = check_device_ptr(labels_out, "labels_out");
    if (st == CC_OK && m > 0) st = check_device_ptr(src, "src");
    if (st == CC_OK && m > 0) st = check_device_ptr(dst, "dst");
    if (st != CC_OK) return st;
    unsigned char* scratch = nullptr;
    st = scratch_for_device(&scratch);
    if (st != CC_OK) return st;
    Ctl* ctl = reinterpret_cast<Ctl*>(scratch);
    int32_t* Lu = (mode == CC_SYNC) ? reinterpret_cast<int32_t*>(scratch + kCtlBytes) : nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    Ctl h;

    // the scratch keeps the previous call's contents: clear the control words
    cc::ctl_reset_kernel<<<1, 32, 0, s>>>(ctl, max_sweeps, 1);
    NA_CUDA(cudaGetLastError());
    if (m > 0) {
        auto kv = cc::validate_ids_kernel<int32_t>;
        kv<<<grid_for(kv, m / 4 + 1), kThreads, 0, s>>>(src, dst, m, n, ctl);
        NA_CUDA(cudaGetLastError());
        NA_CUDA(cudaMemcpyAsync(&h, ctl, sizeof h, cudaMemcpyDeviceToHost, s));
        NA_CUDA(cudaStreamSynchronize(s));
        if (h.bad_count)
            return cc::set_error(CC_EIDRANGE, "cc_run_noalloc: %llu edge endpoints outside [0, %lld)",
                                 h.bad_count, (long long)n);
    }
    auto ki = cc::iota_kernel<int32_t>;
    ki<<<grid_for(ki, n), kThreads, 0, s>>>(labels_out, Lu, n);
    NA_CUDA(cudaGetLastError());

    int32_t sweeps = 0;
    bool converged = false;
    while (true) {
        for (int j = 0; j < check_interval; ++j) {
            int32_t* flag = (j == check_interval - 1) ? &ctl->flag : nullptr;
            const int first = (sweeps == 0 && j == 0 && mode == CC_SYNC) ? 2 : 0;
            if (mode == CC_SYNC) {
                sweep<true>(order, src, dst, m, labels_out, Lu, flag, first, s);
                auto kc = cc::copy_kernel<int32_t>;
                kc<<<grid_for(kc, n / 4 + 1), kThreads, 0, s>>>(labels_out, Lu, n);
            } else {
                sweep<false>(order, src, dst, m, labels_out, nullptr, flag, first, s);
            }
        }
        NA_CUDA(cudaGetLastError());
        sweeps += check_interval;
        int32_t flag_h = 0;
        NA_CUDA(cudaMemcpyAsync(&flag_h, &ctl->flag, sizeof flag_h, cudaMemcpyDeviceToHost, s));
        NA_CUDA(cudaStreamSynchronize(s));
        if (flag_h == 0) {
            converged = true;
            break;
        }
        if (sweeps >= max_sweeps) break;
        NA_CUDA(cudaMemsetAsync(&ctl->flag, 0, sizeof(int32_t), s));
    }
    if (sweeps_out) *sweeps_out = sweeps;
    if (!converged)
        return cc::set_error(CC_ENOTCONVERGED, "cc_run_noalloc: not converged after %d sweeps", sweeps);
    noalloc_mark_converged<<<1, 32, 0, s>>>(ctl);
    auto kp = cc::compress_kernel<int32_t>;
    kp<<<grid_for(kp, n), kThreads, 0, s>>>(labels_out, n, ctl);
    NA_CUDA(cudaGetLastError());
    NA_CUDA(cudaMemcpyAsync(&h, ctl, sizeof h, cudaMemcpyDeviceToHost, s));
    NA_CUDA(cudaStreamSynchronize(s));
    if (h.compress_changes)
        return cc::set_error(CC_ECUDA, "cc_run_noalloc: converged state was not a set of stars (%llu labels moved)",
                             h.compress_changes);
    return CC_OK;
}
