/*
 * Serial simulator of the synchronous Contour algorithm.  TEST INFRASTRUCTURE ONLY.
 *
 * Follows Alg. 1 ("Minimum-Mapping based Contour Algorithm") with the
 * h-order minimum-mapping operator MM^h of Def. 3 in place of MM^2:
 *
 *   for all i: L[i] = i, L_u[i] = i                     (Alg. 1, initialisation)
 *   do {
 *       for every edge <w, v>: MM^h(L_u, L, w, v)       (Alg. 1, edge loop)
 *       L = L_u                                          (Alg. 1, copy)
 *   } while (some label of L changed)
 *   return L
 *
 * MM^h(L_u, L, w, v) (Def. 3): with L^1[x] = L[x] and L^j[x] = L[L^{j-1}[x]],
 * z = min(L^h[w], L^h[v]); then the conditional vector assignment of Def. 1
 * (x_i = z if x_i > z) is applied to the 2h entries
 * L_u[w], L_u[L[w]], ..., L_u[L^{h-1}[w]] and the same h entries for v.
 *
 * Reads go to L and writes to L_u only, so the edge loop is order independent
 * and a plain serial loop gives exactly the per-iteration state that any
 * parallel execution of Alg. 1 with atomic (CAS, Eq. "cas") conditional
 * assignment gives.  The iteration count includes the final iteration that
 * observes no change, as the do-while of Alg. 1 does.
 *
 * The operator order h is taken literally (h = 1024 for the "C-m" variant of
 * Section III-B4 with m = 1024): the chain is walked h steps even after it has
 * reached a root, where it simply repeats the root.
 *
 * Arguments:
 *   n, m, src, dst   graph with ids 0..n-1, m undirected edges <src[e], dst[e]>
 *   h                operator order, h >= 1
 *   max_iters        stop after this many iterations even if not converged
 *   init             NULL, or a starting label array (resume from a snapshot)
 *   L                out: labels after the last iteration (n entries)
 *   states           NULL, or room for max_iters * n labels: the state of L
 *                    after each iteration k is stored at states[(k-1)*n ...]
 * Returns the number of iterations executed, negated when the loop stopped at
 * max_iters with a change still seen in the last iteration; -(2^62) if memory
 * for L_u could not be allocated.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

int64_t oracle_contour_sync_i32(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                                int32_t h, int64_t max_iters, const int32_t *init,
                                int32_t *L, int32_t *states)
{
    int32_t *Lu = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!Lu)
        return -((int64_t)1 << 62);
    for (int64_t i = 0; i < n; ++i) {
        L[i] = init ? init[i] : (int32_t)i;
        Lu[i] = L[i];
    }
    int64_t iter = 0;
    int changed = 0;
    do {
        for (int64_t e = 0; e < m; ++e) {
            int32_t w = src[e], v = dst[e];
            /* the chains end at L^h[w] and L^h[v] */
            int32_t cw = w, cv = v;
            for (int32_t j = 0; j < h; ++j) {
                cw = L[cw];
                cv = L[cv];
            }
            int32_t z = cw < cv ? cw : cv;
            /* conditional assignment to L_u[L^j[w]] and L_u[L^j[v]], j = 0..h-1 */
            int32_t xw = w, xv = v;
            for (int32_t j = 0; j < h; ++j) {
                if (Lu[xw] > z)
                    Lu[xw] = z;
                if (Lu[xv] > z)
                    Lu[xv] = z;
                xw = L[xw];
                xv = L[xv];
            }
        }
        changed = 0;
        for (int64_t i = 0; i < n; ++i)
            if (Lu[i] != L[i]) {
                changed = 1;
                break;
            }
        memcpy(L, Lu, (size_t)n * sizeof(int32_t));
        ++iter;
        if (states)
            memcpy(states + (iter - 1) * n, L, (size_t)n * sizeof(int32_t));
    } while (changed && iter < max_iters);
    free(Lu);
    return changed ? -iter : iter;
}
