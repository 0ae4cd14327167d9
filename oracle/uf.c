/*
 * Connected-components oracle: serial union-find.  TEST INFRASTRUCTURE ONLY.
 *
 * Computes, for every vertex v of an undirected graph with ids 0..n-1
 * (Section II-A), label[v] = min{ u : u is connected to v }, i.e. the smallest
 * vertex id in v's component.  That is the fixed point the Contour algorithm
 * returns (Alg. 1 returns L, whose stars are rooted at the component minimum:
 * Section II-A says the final pointer graph is S stars, and every label is
 * lowered to a minimum over its chain, Def. 1-3).
 *
 * Method: textbook disjoint sets.  union(a, b) hangs the root with the larger
 * id under the root with the smaller id, so every root is the minimum id of
 * its set; find() uses path halving.  After all edges are united,
 * label[v] = find(v).  This shares nothing with the CUDA path.
 *
 * Return value: 0 on success, or -(e + 1) where e is the index of the first
 * edge with an endpoint outside [0, n).
 */
#include <stdint.h>
#include <stdlib.h>

static int32_t find32(int32_t *parent, int32_t x)
{
    while (parent[x] != x) {
        parent[x] = parent[parent[x]];   /* path halving */
        x = parent[x];
    }
    return x;
}

static int64_t find64(int64_t *parent, int64_t x)
{
    while (parent[x] != x) {
        parent[x] = parent[parent[x]];
        x = parent[x];
    }
    return x;
}

int64_t oracle_uf_labels_i32(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                             int32_t *label)
{
    for (int64_t e = 0; e < m; ++e)
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n)
            return -(e + 1);
    int32_t *parent = label;              /* the output doubles as the forest */
    for (int64_t i = 0; i < n; ++i)
        parent[i] = (int32_t)i;
    for (int64_t e = 0; e < m; ++e) {
        int32_t a = find32(parent, src[e]);
        int32_t b = find32(parent, dst[e]);
        if (a < b)
            parent[b] = a;
        else if (b < a)
            parent[a] = b;
    }
    for (int64_t i = 0; i < n; ++i)
        label[i] = find32(parent, (int32_t)i);
    return 0;
}

int64_t oracle_uf_labels_i64(int64_t n, int64_t m, const int64_t *src, const int64_t *dst,
                             int64_t *label)
{
    for (int64_t e = 0; e < m; ++e)
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n)
            return -(e + 1);
    int64_t *parent = label;
    for (int64_t i = 0; i < n; ++i)
        parent[i] = i;
    for (int64_t e = 0; e < m; ++e) {
        int64_t a = find64(parent, src[e]);
        int64_t b = find64(parent, dst[e]);
        if (a < b)
            parent[b] = a;
        else if (b < a)
            parent[a] = b;
    }
    for (int64_t i = 0; i < n; ++i)
        label[i] = find64(parent, i);
    return 0;
}
