/*
 * PR-quadtree oracle -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Restates Section 4.1.1 (Index Creation) step by step:
 *   1. Morton code of every object at level L of the virtual full quadtree
 *      (a uniform 2^L x 2^L grid);
 *   2. sort the objects by that code, so every quadrant at any level l <= L
 *      owns one contiguous interval of the sorted order (the code of the level-l
 *      ancestor is z' = floor(z / 4^(L - l)));
 *   3. starting from the root interval, split every quadrant holding more than
 *      th objects into its four children, one level at a time, until nothing
 *      needs splitting or level L is reached, where the remaining quadrants
 *      become leaves.
 * Leaves are finally ordered by z'' = z * 4^(L - level), the Morton code of
 * the first level-L cell they cover (the paper prints the exponent as
 * l - l_deep; the leaf order it describes needs l_deep - l).
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>

static uint32_t cell_coord(float v, float v0, float scale, int L) {
    float t = (v - v0) * scale;
    float lim = (float)(1u << L);
    if (!(t >= 0.0f)) return 0u; /* below the domain, or NaN */
    if (t >= lim) return (1u << L) - 1u;
    return (uint32_t)t; /* t >= 0: truncation is floor */
}

uint32_t oracle_morton_key(float x, float y, float x0, float y0, float scale, int L) {
    uint32_t cx = cell_coord(x, x0, scale, L);
    uint32_t cy = cell_coord(y, y0, scale, L);
    uint32_t key = 0;
    for (int b = 0; b < L; ++b) {
        key |= ((cx >> b) & 1u) << (2 * b);
        key |= ((cy >> b) & 1u) << (2 * b + 1);
    }
    return key;
}

typedef struct {
    uint32_t key;
    int32_t id;
} pair_t;

static int cmp_pair(const void *a, const void *b) {
    const pair_t *pa = (const pair_t *)a, *pb = (const pair_t *)b;
    if (pa->key != pb->key) return pa->key < pb->key ? -1 : 1;
    return (pa->id > pb->id) - (pa->id < pb->id);
}

typedef struct {
    int32_t level;
    uint32_t z;
    int32_t start, count;
} quad_t_;

static int L_global_for_sort; /* set before qsort of the leaves */

static uint64_t zpp(const quad_t_ *q) {
    return (uint64_t)q->z << (2 * (L_global_for_sort - q->level));
}

static int cmp_leaf(const void *a, const void *b) {
    uint64_t za = zpp((const quad_t_ *)a), zb = zpp((const quad_t_ *)b);
    return (za > zb) - (za < zb);
}

int64_t oracle_pr_quadtree(int64_t n, const float *x, const float *y, float x0,
                           float y0, float scale, int L, int32_t th,
                           int min_level, int emit_empty, int64_t cap,
                           int32_t *level, uint32_t *z, int32_t *start,
                           int32_t *count, int32_t *sorted_ids) {
    pair_t *p = (pair_t *)malloc(sizeof(pair_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        p[i].key = oracle_morton_key(x[i], y[i], x0, y0, scale, L);
        p[i].id = (int32_t)i;
    }
    qsort(p, (size_t)n, sizeof(pair_t), cmp_pair);
    if (sorted_ids)
        for (int64_t i = 0; i < n; ++i) sorted_ids[i] = p[i].id;

    /* Level-by-level construction; "frontier" holds the quadrants of the
     * current level that still have to be examined. */
    size_t fcap = 16, lcap = 16;
    quad_t_ *frontier = (quad_t_ *)malloc(sizeof(quad_t_) * fcap);
    quad_t_ *leaves = (quad_t_ *)malloc(sizeof(quad_t_) * lcap);
    size_t nf = 0, nl = 0;
    frontier[nf++] = (quad_t_){0, 0u, 0, (int32_t)n};

    for (int l = 0; nf > 0; ++l) {
        size_t ncap = 16, nn = 0;
        quad_t_ *next = (quad_t_ *)malloc(sizeof(quad_t_) * ncap);
        for (size_t f = 0; f < nf; ++f) {
            quad_t_ q = frontier[f];
            int split = (q.count > th || l < min_level) && q.count > 0 && l < L;
            if (!split) {
                if (q.count > 0 || emit_empty) {
                    if (nl == lcap) {
                        lcap *= 2;
                        leaves = (quad_t_ *)realloc(leaves, sizeof(quad_t_) * lcap);
                    }
                    leaves[nl++] = q;
                }
                continue;
            }
            /* The four children partition q's interval; child c holds the keys
             * whose level-(l+1) ancestor code is 4 z + c. */
            int shift = 2 * (L - l - 1);
            int32_t s = q.start;
            for (uint32_t c = 0; c < 4; ++c) {
                int32_t e = s;
                while (e < q.start + q.count && ((p[e].key >> shift) & 3u) == c) ++e;
                if (nn == ncap) {
                    ncap *= 2;
                    next = (quad_t_ *)realloc(next, sizeof(quad_t_) * ncap);
                }
                next[nn++] = (quad_t_){l + 1, (q.z << 2) | c, s, e - s};
                s = e;
            }
        }
        free(frontier);
        frontier = next;
        nf = nn;
    }
    free(frontier);
    free(p);

    L_global_for_sort = L;
    qsort(leaves, nl, sizeof(quad_t_), cmp_leaf);
    if ((int64_t)nl > cap) {
        free(leaves);
        return -(int64_t)nl;
    }
    for (size_t i = 0; i < nl; ++i) {
        level[i] = leaves[i].level;
        z[i] = leaves[i].z;
        start[i] = leaves[i].start;
        count[i] = leaves[i].count;
    }
    free(leaves);
    return (int64_t)nl;
}
