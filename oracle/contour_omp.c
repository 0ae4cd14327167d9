/* Multicore CPU Contour -- a timed CPU baseline, TEST INFRASTRUCTURE ONLY.
 *
 * The asynchronous Contour variants as the paper runs them on a multicore
 * CPU (Section III-B): one parallel loop over the edge list per iteration,
 * labels updated in place (III-B1), the operator MM^h of Def. 3 with plain
 * stores instead of compare-and-swap (III-B3), and the loop ended by the
 * first iteration in which no edge changed a label (III-B2).  h = 2 is C-2,
 * h = 1 is C-1, h = 1024 is C-m (Section IV-C).
 *
 * The loads and stores of L are C11-style relaxed atomics: other threads
 * write L while it is read, and relaxed accesses are the defined form of the
 * paper's unsynchronised reads and plain stores.  A store may overwrite a
 * smaller label written by another thread in the meantime; every stored
 * value is still a label of the same component that is <= the vertex id, so
 * only iterations are lost, never the result (the fixed point is unique).
 *
 * Built into its own library with -fopenmp; the rest of the oracle does not
 * depend on it.
 */
#include <stdint.h>

#include <omp.h>

static inline int32_t ld(const int32_t* L, int64_t x) { return __atomic_load_n(L + x, __ATOMIC_RELAXED); }
static inline void st(int32_t* L, int64_t x, int32_t z) { __atomic_store_n(L + x, z, __ATOMIC_RELAXED); }

/* Last vertex of the order-h chain x, L[x], L[L[x]], ... (h steps, or fewer
 * when a root L[r] == r is reached: the chain only repeats r after that). */
static inline int32_t chain_end(const int32_t* L, int32_t x, int32_t h) {
    for (int32_t j = 0; j < h; ++j) {
        const int32_t y = ld(L, x);
        if (y == x) break;
        x = y;
    }
    return x;
}

/* Set every label on the chain from x that exceeds z to z (Def. 3); returns 1
 * when some label was written.  The chain is non-increasing, so the walk
 * stops at the first label <= z. */
static inline int write_chain(int32_t* L, int32_t x, int32_t z, int32_t h) {
    int wrote = 0;
    for (int32_t j = 0; j < h; ++j) {
        const int32_t y = ld(L, x);
        if (y <= z) break;
        st(L, x, z);
        wrote = 1;
        if (y == x) break;
        x = y;
    }
    return wrote;
}

/* Labels of the n vertices for the m edges (src[e], dst[e]) with asynchronous
 * order-h Contour on `threads` threads (<= 0: OpenMP's default).  Returns the
 * number of iterations (the last one changes nothing), or -1 when max_iter
 * iterations did not reach the fixed point.  *threads_used receives the team
 * size. */
int64_t omp_contour_async_i32(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, int32_t h,
                              int64_t max_iter, int32_t threads, int32_t* L, int32_t* threads_used) {
    if (threads > 0) omp_set_num_threads(threads);
    int32_t team = 1;
#pragma omp parallel
    {
#pragma omp single
        team = (int32_t)omp_get_num_threads();
    }
    if (threads_used) *threads_used = team;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) L[i] = (int32_t)i;
    for (int64_t it = 1; it <= max_iter; ++it) {
        int changed = 0;
#pragma omp parallel for schedule(static, 4096) reduction(| : changed)
        for (int64_t e = 0; e < m; ++e) {
            const int32_t w = src[e], v = dst[e];
            const int32_t ew = chain_end(L, w, h), ev = chain_end(L, v, h);
            const int32_t z = ew < ev ? ew : ev;
            changed |= write_chain(L, w, z, h);
            changed |= write_chain(L, v, z, h);
        }
        if (!changed) return it;
    }
    return -1;
}
