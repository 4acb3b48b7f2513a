/*
 * CPU oracle for repeated k-NN over moving objects -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct restatement of what the per-tick hot path
 * computes (Lettich, Orlando, Silvestri, "Manycore processing of repeated k-NN
 * queries over massive moving objects observations").  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg use it; the library never
 * links it and shares no code with it.
 *
 * Arithmetic: binary32, round-to-nearest-even, each operation rounded on its
 * own.  This file must be compiled with -ffp-contract=off so that
 * dx*dx + dy*dy is never fused into an FMA.
 */
#ifndef KNN_ORACLE_H
#define KNN_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Batch semantics, Section 2.2: the updates of one tick are applied in array
 * order, so a later update of the same object overwrites an earlier one.
 * Entries whose id lies outside [0, n) or whose coordinates are not finite
 * are skipped.  Returns the number of skipped entries. */
int64_t oracle_apply_updates(int64_t n, float *x, float *y, int64_t n_upd,
                             const int32_t *upd_id, const float *upd_x,
                             const float *upd_y);

/* Squared Euclidean distance in binary32: dx = qx - px, dy = qy - py,
 * d = dx*dx + dy*dy with every operation rounded separately. */
float oracle_sqdist(float qx, float qy, float px, float py);

/* Def. 1 (k-NN query) with ties broken by (distance, object id).
 * For query i with issuer s = q_id[i] (or -1 for an anonymous query) and
 * centre (q_x[i], q_y[i]) -- or the issuer's position when q_x is NULL --
 * every object j != s is ranked by the key (d(q, o_j), j); the k smallest keys
 * are written to row i of out_ids / out_d2 (row-major, k per row), ascending.
 * Rows with fewer than k eligible objects are padded with (-1, +inf).
 * Invalid queries (issuer outside [-1, n), anonymous with q_x NULL, or a
 * non-finite centre) get a fully padded row and are counted in the return
 * value.  n_threads <= 0 uses every online CPU. */
int64_t oracle_knn(int64_t n, const float *x, const float *y, int64_t n_q,
                   const int32_t *q_id, const float *q_x, const float *q_y,
                   int32_t k, int32_t *out_ids, float *out_d2, int n_threads);

/* Section 4.1.1: index of the level-L quadrant holding (x, y) in the virtual
 * full quadtree over the square [x0, x0+side) x [y0, y0+side): the cell
 * coordinate is floor((x - x0) * scale), scale = 2^L / side rounded to
 * binary32, clamped to [0, 2^L - 1]; the Morton code interleaves the cell
 * coordinates, x in the even bits and y in the odd bits. */
uint32_t oracle_morton_key(float x, float y, float x0, float y0, float scale, int L);

/* Section 4.1.1: PR-quadtree construction.  Objects are sorted by Morton key
 * at level L (stable: equal keys keep ascending id).  Starting from the root
 * interval [0, n), every quadrant with more than th objects is split into its
 * four children, level by level, until no quadrant needs splitting or level L
 * is reached (leftover quadrants at L become leaves).  Quadrants above
 * min_level are split regardless of their count (min_level = 0 gives the
 * paper's tree).  Leaves are returned in Morton order (their code z'' at level
 * L, i.e. z * 4^(L - level)).
 *
 * Outputs (capacity cap each): level[], z[] (code at its own level), start[],
 * count[] (interval in the sorted order).  Empty leaves are emitted only when
 * emit_empty != 0 (they are never emitted below a split forced by min_level).
 * sorted_ids (n entries, may be NULL) receives the sorted object order.
 * Returns the number of leaves, or -(needed) when cap is too small. */
int64_t oracle_pr_quadtree(int64_t n, const float *x, const float *y, float x0,
                           float y0, float scale, int L, int32_t th,
                           int min_level, int emit_empty, int64_t cap,
                           int32_t *level, uint32_t *z, int32_t *start,
                           int32_t *count, int32_t *sorted_ids);

#ifdef __cplusplus
}
#endif
#endif
