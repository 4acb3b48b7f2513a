/*
 * Brute-force k-NN oracle -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Follows the paper's Section 2 directly:
 *   - Section 2.2 (batch processing): a tick's position updates are applied in
 *     order, the most recent one per object wins;
 *   - Def. 1 (k-NN query): the result of q issued by o_s holds the objects o_j,
 *     j != s, whose rank (number of objects strictly closer) is below k; ties
 *     that would give more than k are resolved here by the object id, i.e. the
 *     k smallest keys (d, j) in lexicographic order are returned, ascending.
 *
 * Compile with -ffp-contract=off (build.py does): each binary32 operation is
 * rounded on its own, there is no FMA in the distance.
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

int64_t oracle_apply_updates(int64_t n, float *x, float *y, int64_t n_upd,
                             const int32_t *upd_id, const float *upd_x,
                             const float *upd_y) {
    int64_t skipped = 0;
    for (int64_t i = 0; i < n_upd; ++i) {
        int32_t id = upd_id[i];
        if (id < 0 || (int64_t)id >= n || !isfinite(upd_x[i]) || !isfinite(upd_y[i])) {
            ++skipped;
            continue;
        }
        x[id] = upd_x[i];
        y[id] = upd_y[i];
    }
    return skipped;
}

float oracle_sqdist(float qx, float qy, float px, float py) {
    float dx = qx - px;
    float dy = qy - py;
    float dx2 = dx * dx;
    float dy2 = dy * dy;
    return dx2 + dy2;
}

typedef struct {
    float d;
    int32_t id;
} key_t_;

/* Lexicographic order on (distance, id). */
static int key_less(key_t_ a, key_t_ b) {
    if (a.d < b.d) return 1;
    if (a.d > b.d) return 0;
    return a.id < b.id;
}

/* Max-heap on key_less holding the best (smallest) keys seen so far. */
static void heap_sift_down(key_t_ *h, int32_t size, int32_t i) {
    for (;;) {
        int32_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < size && key_less(h[m], h[l])) m = l;
        if (r < size && key_less(h[m], h[r])) m = r;
        if (m == i) return;
        key_t_ t = h[i];
        h[i] = h[m];
        h[m] = t;
        i = m;
    }
}

static void heap_sift_up(key_t_ *h, int32_t i) {
    while (i > 0) {
        int32_t p = (i - 1) / 2;
        if (!key_less(h[p], h[i])) return;
        key_t_ t = h[i];
        h[i] = h[p];
        h[p] = t;
        i = p;
    }
}

static int cmp_key(const void *a, const void *b) {
    key_t_ ka = *(const key_t_ *)a, kb = *(const key_t_ *)b;
    if (key_less(ka, kb)) return -1;
    if (key_less(kb, ka)) return 1;
    return 0;
}

/* One query: keep the k smallest keys over all eligible objects. */
static void knn_one(int64_t n, const float *x, const float *y, float qx, float qy,
                    int32_t issuer, int32_t k, key_t_ *heap, int32_t *out_ids,
                    float *out_d2) {
    int32_t size = 0;
    for (int64_t j = 0; j < n; ++j) {
        if ((int32_t)j == issuer) continue;
        key_t_ c;
        c.d = oracle_sqdist(qx, qy, x[j], y[j]);
        c.id = (int32_t)j;
        if (size < k) {
            heap[size] = c;
            heap_sift_up(heap, size);
            ++size;
        } else if (key_less(c, heap[0])) {
            heap[0] = c;
            heap_sift_down(heap, size, 0);
        }
    }
    qsort(heap, (size_t)size, sizeof(key_t_), cmp_key);
    for (int32_t r = 0; r < k; ++r) {
        if (r < size) {
            out_ids[r] = heap[r].id;
            out_d2[r] = heap[r].d;
        } else {
            out_ids[r] = -1;
            out_d2[r] = INFINITY;
        }
    }
}

typedef struct {
    int64_t n, n_q;
    const float *x, *y;
    const int32_t *q_id;
    const float *q_x, *q_y;
    int32_t k;
    int32_t *out_ids;
    float *out_d2;
    int t, n_threads;
    int64_t invalid;
} job_t;

static void *worker(void *arg) {
    job_t *j = (job_t *)arg;
    key_t_ *heap = (key_t_ *)malloc(sizeof(key_t_) * (size_t)(j->k > 0 ? j->k : 1));
    j->invalid = 0;
    for (int64_t i = j->t; i < j->n_q; i += j->n_threads) {
        int32_t s = j->q_id[i];
        int32_t *oi = j->out_ids + i * j->k;
        float *od = j->out_d2 + i * j->k;
        int ok = (s >= -1 && (int64_t)s < j->n);
        float qx = 0.f, qy = 0.f;
        if (ok) {
            if (j->q_x) {
                qx = j->q_x[i];
                qy = j->q_y[i];
            } else if (s >= 0) {
                qx = j->x[s];
                qy = j->y[s];
            } else {
                ok = 0;
            }
        }
        if (ok && (!isfinite(qx) || !isfinite(qy))) ok = 0;
        if (!ok) {
            for (int32_t r = 0; r < j->k; ++r) {
                oi[r] = -1;
                od[r] = INFINITY;
            }
            ++j->invalid;
            continue;
        }
        knn_one(j->n, j->x, j->y, qx, qy, s, j->k, heap, oi, od);
    }
    free(heap);
    return NULL;
}

int64_t oracle_knn(int64_t n, const float *x, const float *y, int64_t n_q,
                   const int32_t *q_id, const float *q_x, const float *q_y,
                   int32_t k, int32_t *out_ids, float *out_d2, int n_threads) {
    if (k <= 0 || n_q < 0 || n < 0) return -1;
    if (n_threads <= 0) {
        long c = sysconf(_SC_NPROCESSORS_ONLN);
        n_threads = c > 0 ? (int)c : 1;
    }
    if ((int64_t)n_threads > n_q) n_threads = n_q > 0 ? (int)n_q : 1;
    job_t *jobs = (job_t *)calloc((size_t)n_threads, sizeof(job_t));
    pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    for (int t = 0; t < n_threads; ++t) {
        job_t *j = &jobs[t];
        j->n = n;
        j->n_q = n_q;
        j->x = x;
        j->y = y;
        j->q_id = q_id;
        j->q_x = q_x;
        j->q_y = q_y;
        j->k = k;
        j->out_ids = out_ids;
        j->out_d2 = out_d2;
        j->t = t;
        j->n_threads = n_threads;
        if (n_threads > 1)
            pthread_create(&th[t], NULL, worker, j);
        else
            worker(j);
    }
    int64_t invalid = 0;
    for (int t = 0; t < n_threads; ++t) {
        if (n_threads > 1) pthread_join(th[t], NULL);
        invalid += jobs[t].invalid;
    }
    free(th);
    free(jobs);
    return invalid;
}
