/*
 * knn.h -- C ABI of the GB300-native repeated k-NN library.
 *
 * Repeated k-NN queries over moving objects (Lettich, Orlando, Silvestri,
 * "Manycore processing of repeated k-NN queries over massive moving objects
 * observations", arXiv 1412.6170).  A "world" holds the last known positions
 * of n moving objects on one GPU.  Each tick applies a batch of position
 * updates and answers a batch of k-NN queries against the updated positions
 * (the paper's iterated batch processing, Section 2.3):
 *
 *   1. updates are applied in array order, the last one per object wins
 *      (Section 2.2, timeslice batching);
 *   2. a PR-quadtree over the positions is rebuilt on the device: Morton codes
 *      at level max_depth, a radix sort, and a leaf split at leaf_capacity
 *      (Section 4.1.1);
 *   3. every query expands over the quadtree leaves around it, keeping its k
 *      best objects, until the disc of its k-th distance is covered by the
 *      leaves already visited (Sections 4.2.1-4.2.2);
 *   4. results are written in the caller's query order, one row of k per query
 *      (Section 3.3.2, linear result layout).
 *
 * Result definition (Def. 1, Section 2.1): for query i issued by object s
 * (q_id[i] = s, or -1 for an anonymous query) and centred at c, every object
 * j != s is ranked by the key (d(c, o_j), j) where
 *     d = dx*dx + dy*dy,  dx = c.x - x_j,  dy = c.y - y_j,
 * evaluated in IEEE binary32 with every operation rounded to nearest-even and
 * no fused multiply-add.  Row i holds the k smallest keys, ascending, padded
 * with (id -1, d2 +inf) when fewer than k objects are eligible.  The output is
 * unique, so it is bit-exact against any correct implementation.
 *
 * Conventions
 *  - All sizes are int64_t.  Object ids are 0..n-1 (int32).  n <= 2^30.
 *  - Pointers named *_dev are device pointers of the world's GPU; the caller
 *    owns them and keeps inputs valid (and outputs unread) until the stream
 *    reaches the end of the call.  *_host are host pointers.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  knn_tick and knn_world_* calls on one world must be ordered on
 *    the device (one stream, or event-ordered streams): the world owns one set
 *    of scratch buffers.
 *  - Host-detectable errors return immediately and launch nothing.  Errors
 *    that only the device can see (an update id outside [0, n), a non-finite
 *    coordinate, an invalid query) never fault: the offending entry is
 *    skipped (an invalid query gets a padded row), an error bit is set in
 *    the world, and knn_tick_status reports it.
 *  - knn_last_error() returns a thread-local message for the last failure.
 *  - Every device-side wait is bounded; running out sets KNN_ERR_TIMEOUT.
 */
#ifndef KNN_H
#define KNN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct knn_world_s *knn_world;

typedef enum {
    KNN_OK = 0,
    KNN_ERR_INVALID = -1,      /* bad argument, detected on the host */
    KNN_ERR_OOM = -2,          /* device allocation failed */
    KNN_ERR_CUDA = -3,         /* a CUDA runtime call failed */
    KNN_ERR_TIMEOUT = -4,      /* a bounded device-side wait ran out */
    KNN_ERR_ADMISSION = -5,    /* reserved for request admission */
    KNN_ERR_DEVICE_INPUT = -6  /* the device skipped invalid input entries */
} knn_status;

/* World description.  The domain is the square [x0, x0+side) x [y0, y0+side)
 * that the virtual full quadtree covers (the paper's MBR G, Section 3.3).
 * Positions outside it are legal: they fall into the border cells for the
 * index, and distances always use the true coordinates. */
typedef struct {
    float x0, y0, side;      /* side > 0 and finite */
    int32_t leaf_capacity;   /* th_quad: max objects per leaf; 0 = automatic; <= 4096 */
    int32_t max_depth;       /* l_max in [1, 16]; 0 = automatic: 12 for n <= 2^20
                                objects (24-bit keys, a 3-pass sort), else 16 */
    int32_t k_max;           /* largest k a tick may ask for, in [1, 512] */
    int64_t max_queries;     /* largest n_q a tick may pass, >= 0 */
} knn_world_desc;

/* Create a world of n objects (ids 0..n-1) at the positions x_dev[i], y_dev[i]
 * (device arrays of n floats, copied; all must be finite): the set O of
 * moving objects with their last known positions (Section 2.1, the moving
 * object model, and Section 2.2: positions stay valid until an update
 * arrives).  No index is built here: the PR quadtree is rebuilt every tick
 * (Section 4.1.1), so a world is just positions plus scratch.  Allocates every
 * device buffer the ticks need (sized from n, k_max, max_queries), so ticks
 * never allocate.  May synchronize `stream`.  Returns KNN_ERR_INVALID for a
 * bad description, n outside [1, 2^30] or a non-finite position. */
knn_status knn_world_create(const knn_world_desc *desc, const float *x_dev,
                            const float *y_dev, int64_t n, void *stream,
                            knn_world *out);

/* One tick (Sections 2.2-2.3 and 4): apply n_upd updates (upd_id[i] moves to
 * (upd_x[i], upd_y[i]); later entries win; invalid entries are skipped), then
 * answer n_q k-NN queries.  Query i is issued by q_id[i] (-1 = anonymous) and
 * centred at (q_x[i], q_y[i]), or, when q_x and q_y are both NULL, at its
 * issuer's post-update position.  Writes out_ids_dev[i*k + r] and
 * out_d2_dev[i*k + r], r < k (row-major, caller order).  Asynchronous on
 * `stream`; performs no host synchronisation and no allocation.
 * KNN_ERR_INVALID for: k outside [1, k_max], n_q outside [0, max_queries],
 * n_upd outside [0, 2^31), a NULL array whose count is non-zero, or only one
 * of q_x / q_y given. */
knn_status knn_tick(knn_world w, const int32_t *upd_id_dev, const float *upd_x_dev,
                    const float *upd_y_dev, int64_t n_upd, const int32_t *q_id_dev,
                    const float *q_x_dev, const float *q_y_dev, int64_t n_q, int32_t k,
                    int32_t *out_ids_dev, float *out_d2_dev, void *stream);

/* Arguments of one world's tick, as for knn_tick (device pointers), plus
 * q_k_dev: NULL, or n_q per-query list sizes (Section 2.1: a query is
 * q = (x, y, k)).  Query i then gets the q_k_dev[i] nearest objects in the
 * first entries of its row (still k wide) and padding after them; 0 gives an
 * all-padding row, a value outside [0, k] a padded row and the invalid-query
 * bit of knn_tick_status. */
typedef struct {
    const int32_t *upd_id_dev;
    const float *upd_x_dev, *upd_y_dev;
    int64_t n_upd;
    const int32_t *q_id_dev;
    const float *q_x_dev, *q_y_dev;
    int64_t n_q;
    int32_t k;
    int32_t *out_ids_dev;
    float *out_d2_dev;
    const int32_t *q_k_dev;
} knn_tick_args;

/* knn_tick from an argument struct (which adds per-query list sizes). */
knn_status knn_tick_ex(knn_world w, const knn_tick_args *args, void *stream);

/* The same tick with every array in host memory (pageable or pinned): the
 * tick runs on `stream` and the call returns after the stream has finished.
 * Pageable arrays go through world-owned device staging buffers (inputs
 * copied in before the tick, rows copied out after it); the first call that
 * needs larger staging buffers allocates them (so that call is not
 * allocation-free).  Output arrays in pinned host memory (cudaHostAlloc,
 * cudaHostRegister) are written in place by the expansion kernel over the
 * CPU-GPU link, so the transfer overlaps the search; see
 * knn_world_set_host_io.  The rows are identical either way. */
knn_status knn_tick_host(knn_world w, const int32_t *upd_id_host, const float *upd_x_host,
                         const float *upd_y_host, int64_t n_upd, const int32_t *q_id_host,
                         const float *q_x_host, const float *q_y_host, int64_t n_q,
                         int32_t k, int32_t *out_ids_host, float *out_d2_host,
                         void *stream);

/* Pipelined host-buffer ticks: knn_tick_host_submit enqueues the tick that
 * knn_tick_host runs, with the same arguments, and returns without waiting.
 * The inputs are copied on a world-owned copy stream into one of two device
 * staging slots (used in turn), the tick runs on `stream` once they are in,
 * and the rows are copied back on a second copy stream once it is done; with
 * the arrays in pinned memory the copies of one tick overlap the search of
 * the next.  *ticket receives the tick's number.  Until knn_tick_host_wait
 * for that ticket returns, the caller must neither change its input arrays
 * nor read its output arrays; two ticks in flight need two sets of output
 * arrays.  Ticks of one world run in submission order.  Errors as knn_tick
 * (checked before anything is enqueued); a submission that needs larger
 * staging buffers waits for its slot's previous tick and allocates them. */
knn_status knn_tick_host_submit(knn_world w, const int32_t *upd_id_host,
                                const float *upd_x_host, const float *upd_y_host,
                                int64_t n_upd, const int32_t *q_id_host, const float *q_x_host,
                                const float *q_y_host, int64_t n_q, int32_t k,
                                int32_t *out_ids_host, float *out_d2_host, void *stream,
                                int64_t *ticket);

/* Blocks until the tick `ticket` (and possibly later ones) has finished and
 * its rows are in the output arrays.  A ticket never submitted: KNN_ERR_INVALID. */
knn_status knn_tick_host_wait(knn_world w, int64_t ticket);

/* How knn_tick_host treats pinned host arrays: bit 0 (on by default) lets the
 * kernels write the rows straight into pinned output arrays; bit 1 (off by
 * default) lets them read pinned input arrays in place instead of copying
 * them to the device first.  Arrays that are not pinned are always staged.
 * mode outside [0, 3]: KNN_ERR_INVALID. */
knn_status knn_world_set_host_io(knn_world w, int32_t mode);

/* Batch processing over many worlds (Section 2.3 per world): one tick of every
 * world in `worlds` (distinct handles on the current device), with args[i]
 * for worlds[i] exactly as knn_tick takes them; the rows are bit-identical to
 * separate knn_tick calls.  The batch is recorded into one CUDA graph: each
 * world's index stages (updates, sort, leaves, query order, packets) form an
 * independent chain, spread over internal streams between a fork and a join
 * on `stream`; then the expansion (Section 4.2) runs batched: per form and
 * list size (4, 8, 16, 32, 64) one persistent grid takes the packets of every
 * world of that class through a device-built prefix of the worlds' packet
 * counts, and one packet-walk grid per list size finishes the packets the
 * gathered form handed back.  Worlds on the tiled form (queries at their
 * issuers, k <= 32) run one batched tile grid per list size first, over the
 * tiles of all of them, and what the tiles pass on joins their packets for
 * the gathered grid.  Worlds whose expansion is one warp per query
 * (k > 32 by default) or the multi-pass ablation expand in their own chains.
 * While the same worlds, sizes and pointers come back, the recorded graph is
 * replayed without recording.  Asynchronous on `stream`; a call that has to
 * record the batch again does host work proportional to the number of worlds
 * and first waits for the last batch launched on this device to finish (its
 * expansion table is rewritten).  Not thread-safe with other batch calls on
 * the same device. */
knn_status knn_batch_tick(int32_t n_worlds, const knn_world *worlds, const knn_tick_args *args,
                          void *stream);

/* ---- serving ---------------------------------------------------------------
 * A request loop over many resident worlds (Sections 2.2-2.3: ticks of
 * updates and queries under a latency requirement).  A request is one world's
 * tick; its latency runs from knn_server_submit to the moment the dispatcher
 * sees the tick complete on the device.  The server keeps every world's
 * positions resident and gives a world its tick scratch only while it has
 * work: a dispatcher thread admits the oldest request of any idle world as
 * soon as one of n_slots streams is free and the world's scratch fits in
 * hbm_budget_bytes, evicting idle worlds' scratch (least recently used first)
 * when needed.  Requests of different worlds overlap on the GPU; requests of
 * one world run in submission order.  Every request gives exactly the rows
 * knn_tick would. */
typedef struct knn_server_s *knn_server;

typedef struct {
    int32_t n_slots;            /* requests on the GPU at once (one stream each), 1..32 */
    int32_t reserved;
    int64_t hbm_budget_bytes;   /* device memory for worlds' tick scratch; 0 = no limit */
} knn_server_desc;

typedef struct {
    int32_t worlds, resident_worlds;  /* registered / holding scratch now */
    int64_t scratch_bytes;            /* scratch the server holds now */
    int64_t largest_world_scratch;    /* scratch the largest registered world needs */
    int64_t admitted, completed, evictions, pending;
} knn_server_counters;

/* Start a server on the current device (creates its streams and dispatcher). */
knn_status knn_server_create(const knn_server_desc *desc, knn_server *out);
/* Register a world exactly as knn_world_create describes it; only its
 * positions are allocated now.  KNN_ERR_ADMISSION when the world's tick
 * scratch could never fit in the budget.  *world_index receives its index. */
knn_status knn_server_add_world(knn_server s, const knn_world_desc *desc, const float *x_dev,
                                const float *y_dev, int64_t n, int32_t *world_index);
/* Queue one tick of a world (arguments as knn_tick; the arrays must stay
 * valid, and the outputs unread, until the request is done). */
knn_status knn_server_submit(knn_server s, int32_t world_index, const knn_tick_args *args,
                             int64_t *request_id);
/* State of a request (0 queued, 1 running, 2 done, 3 failed) and, once done,
 * its latency in milliseconds (else -1). */
knn_status knn_server_poll(knn_server s, int64_t request_id, int32_t *state,
                           double *latency_ms);
/* Block until a request is done; returns its latency. */
knn_status knn_server_wait(knn_server s, int64_t request_id, double *latency_ms);
knn_status knn_server_stats(knn_server s, knn_server_counters *out);
/* Wait for a world's queued requests and report its device-detected input
 * problems as knn_tick_status does. */
knn_status knn_server_world_status(knn_server s, int32_t world_index, uint32_t *bits_out);
/* Finish every queued request, stop the dispatcher and free everything. */
knn_status knn_server_destroy(knn_server s);

/* Waits for the world's last tick and reports device-detected problems since
 * the previous call: KNN_ERR_TIMEOUT, then KNN_ERR_DEVICE_INPUT (skipped
 * updates, non-finite coordinates, invalid queries), else KNN_OK.  Section
 * 2.2 keeps, per object, only the most recent valid update of a batch; an
 * update or query the device finds invalid is dropped from the batch (the
 * query's row is padding) and reported here instead of failing the tick.  Clears the
 * recorded bits.  If `bits_out` is non-NULL it receives the raw bit set
 * (1 = bad update id, 2 = non-finite update, 4 = invalid query, 8 = timeout,
 * 16 = a failed bounds check of a debug build: KNN_ERR_CUDA). */
knn_status knn_tick_status(knn_world w, uint32_t *bits_out);

/* Release every device buffer of the world (synchronizes its device): the end
 * of the iterated batch processing of Section 2.3 for this set of objects.
 * The handle is invalid afterwards; NULL returns KNN_ERR_INVALID. */
knn_status knn_world_destroy(knn_world w);

/* Thread-local description of the last error returned on this thread. */
const char *knn_last_error(void);

/* ---- GPU brute force (the paper's brute-force comparison, Section 5) ---- */

/* Every query against every object, with no index: the same rows as knn_tick
 * (Def. 1: the k smallest (d^2, id) over objects other than the issuer,
 * ascending, padded with (-1, +inf)), for objects given as device arrays
 * x_dev, y_dev of n floats (ids 0..n-1).  q_x_dev/q_y_dev NULL: each query is
 * centred at its issuer q_id_dev[i] (which must lie in [0, n)); else at the
 * given point, q_id_dev[i] = -1 meaning no issuer to exclude.  A query with
 * an issuer outside [-1, n), no centre or a non-finite centre gets a padded
 * row.  k in [1, 64].  Asynchronous on `stream`; nothing is allocated.
 * O(n * n_q) work: an in-house baseline for the index's speedup. */
knn_status knn_brute_force(const float *x_dev, const float *y_dev, int64_t n,
                           const int32_t *q_id_dev, const float *q_x_dev, const float *q_y_dev,
                           int64_t n_q, int32_t k, int32_t *out_ids_dev, float *out_d2_dev,
                           void *stream);

/* ---- tuning and introspection ------------------------------------------ */

/* Index and expansion parameters; none of them changes any result.
 * leaf_capacity: th_quad (Section 4.1.1), 1..4096.
 * grid_level: level G of the uniform cell map over the leaves (the paper's
 *   z_map, Section 4.1.1); leaves are never coarser than G.  1..gmax, where a
 *   world of n objects has gmax = min(10, max_depth, the smallest g with
 *   4^g >= 4n) (a finer map never pays off); larger values are rejected.
 * packet_level: queries are packed 32 to a warp within one cell of this
 *   level (<= grid_level).
 * expansion: the expansion kernel.  1 = packets of up to 32 queries per warp,
 *   each lane keeping its query's list in registers (k <= 64), each packet
 *   walking the quadtree leaf by leaf; 4 = gathered packets (k <= 32): each
 *   packet fixes its search box from the local density first, gathers the
 *   box's useful leaves and objects in one pass (Section 4.2.2) and tests
 *   them in one loop; a packet it cannot finish goes to the walk; 2 = one warp
 *   per query, the list in shared memory and the row written by the whole
 *   warp (any k; the paper's coalesced-writes variant, Section 3.3.2); 3 =
 *   the paper's multi-pass form (Section 4.2: first iteration on the query's
 *   own cell, then alternating left/right Morton sub-visits, one cell per
 *   iteration; k <= 64), an ablation with the same rows, never recorded in a
 *   tick graph; 5 = tiles (k <= 32, queries at their issuers; other ticks
 *   run form 4): one thread block per packet-level cell of the sorted
 *   queries stages the objects around the cell in shared memory once
 *   (counting-sorted into a fine grid) and each lane scans only its own
 *   query's search box, nearest rows first, shrinking it as its k-th
 *   distance tightens (Alg. 1's per-cell scan); packets it cannot finish
 *   exactly (equal distances, a cell too full to stage) go to form 4, which
 *   finishes them.  The automatic choice is 5 for k <= 32 and 2 above.
 * Any field set to 0 keeps (or restores) the automatic choice. */
typedef struct {
    int32_t leaf_capacity;
    int32_t grid_level;
    int32_t packet_level;
    int32_t expansion;
} knn_tuning;

knn_status knn_world_set_tuning(knn_world w, const knn_tuning *t);
/* Autotuner: runs `trials` ticks without updates for each of a small set of
 * leaf capacities, cell-map levels and packet levels around the automatic
 * choice, then for the fastest of those each expansion form (threads per
 * query: a lane in packets or a warp per query; candidates staged along the
 * walk, gathered at once per packet, or staged once per tile), with the given
 * queries (device arrays as for
 * knn_tick; the output arrays receive the rows, identical for every setting),
 * keeps the fastest in the world and writes it to *chosen (may be NULL).  Each
 * setting is timed as a recorded CUDA graph of `trials` ticks (device time),
 * and the automatic setting stays unless another is at least 3 % faster.
 * Synchronizes `stream`.  The world's positions are unchanged. */
knn_status knn_world_autotune(knn_world w, const int32_t *q_id_dev, const float *q_x_dev,
                              const float *q_y_dev, int64_t n_q, int32_t k,
                              int32_t *out_ids_dev, float *out_d2_dev, int32_t trials,
                              knn_tuning *chosen, void *stream);

/* Autotuner for a batch: chooses the settings of the batch's worlds by timing
 * whole batch ticks (knn_batch_tick with args[i] but without updates, so the
 * positions are unchanged; the output arrays receive the rows).  The worlds
 * are grouped by list size class (k <= 4, 8, 16, 32, 64); per class, largest
 * query count first, each expansion form (packet walk, one warp per query,
 * gathered packets) and then half and twice the leaf capacity are tried for
 * all worlds of the class at once, each as `trials` timed replays of the
 * recorded batch (device time), and a change is kept only if the batch gets
 * at least 3 % faster.  The chosen settings stay in the worlds and go to
 * chosen[i] (n_worlds entries; may be NULL).  Synchronizes `stream`.  On an
 * error every world keeps the setting it had. */
knn_status knn_batch_autotune(int32_t n_worlds, const knn_world *worlds,
                              const knn_tick_args *args, int32_t trials, knn_tuning *chosen,
                              void *stream);

/* The parameters the next tick with query count n_q and k will use. */
knn_status knn_world_get_tuning(knn_world w, int64_t n_q, int32_t k, knn_tuning *out);

/* Copy the leaves built by the last tick (non-empty PR-quadtree leaves in
 * Morton order, never coarser than grid_level) into caller device buffers of
 * `cap` entries: level, code z at that level, start and count in the sorted
 * object order; sorted_ids_dev (n entries, may be NULL) receives that order.
 * Synchronizes `stream`; *m_host receives the number of leaves. */
knn_status knn_world_leaves(knn_world w, int32_t *level_dev, uint32_t *z_dev,
                            int32_t *start_dev, int32_t *count_dev,
                            int32_t *sorted_ids_dev, int64_t cap, int64_t *m_host,
                            void *stream);

/* Copy the current positions (after the last tick's updates) into caller
 * device arrays of n floats; a world re-created from them answers every later
 * tick identically (checkpoint / resume). */
knn_status knn_world_positions(knn_world w, float *x_dev, float *y_dev, void *stream);

/* Failure detection without a fault: enqueues on `stream` one bounded device
 * wait that nothing will satisfy -- a look-back whose predecessor never
 * publishes, the wait every scan of a tick uses -- so that it gives up after
 * its poll limit (milliseconds) exactly as a stalled tick would.  The world's
 * timeout bit is raised: knn_tick_status then reports KNN_ERR_TIMEOUT (and
 * clears it), and the next tick runs normally.  Call between ticks of this
 * world.  NULL world: KNN_ERR_INVALID. */
knn_status knn_world_test_wait_timeout(knn_world w, void *stream);

/* Debug builds (the library compiled with -DKNN_DEBUG: paper_1412_6170_gb300/
 * build.py, build_debug()).  No passage of the paper corresponds; this is the
 * library's own bounds checking.  In a debug build the kernels check their
 * index arithmetic at the main array accesses (objects, leaves, the gathered
 * list, candidate buffers, row writes, radix scatters); an index out of range
 * raises error bit 16 and the access is skipped -- nothing traps -- and
 * knn_tick_status then returns KNN_ERR_CUDA.  knn_debug_build returns KNN_OK
 * in a debug build, else KNN_ERR_INVALID.  knn_world_test_bounds_check
 * enqueues one check that fails on purpose (an index one past the world's
 * objects; the access is skipped), so that knn_tick_status reports bit 16;
 * KNN_ERR_INVALID in a regular build. */
knn_status knn_debug_build(void);
knn_status knn_world_test_bounds_check(knn_world w, void *stream);

/* Number of CUDA kernels this world's ticks have launched so far (host-side
 * count; memsets and copies are not kernels and are not counted). */
knn_status knn_world_launches(knn_world w, int64_t *count);

/* Index reuse (Section 4, the processing pipeline: the index is rebuilt only
 * when needed).  With max_age > 0 a tick keeps the previous tick's leaves and
 * only puts every object into a leaf of its level-G cell (a counting sort by
 * leaf instead of the radix sort and the leaf split).  The leaves are rebuilt
 * instead when max_age ticks have passed since the tick that built them, when
 * their cost -- the sum over leaves of the squared object count -- grew past
 * `factor` times its value right after that build (factor <= 0: no such
 * test), when the plan changed, or when an object entered a level-G cell
 * without leaves; the decision is taken on the device, tick by tick.  Results
 * are identical either way; only the time changes.  max_age = 0 (the
 * default) rebuilds every tick. */
knn_status knn_world_set_index_reuse(knn_world w, int32_t max_age, float factor);

/* Index reuse state after the last tick (synchronizes the world's last stream):
 * *age = ticks since the tick that built the leaves (0: the last tick built
 * them), *rebuilt = 1 when the last tick built them.  Either may be NULL. */
knn_status knn_world_index_info(knn_world w, int32_t *age, int32_t *rebuilt);

/* Tick graphs.  knn_tick records a tick as a CUDA graph and replays it when a
 * later tick passes the same arguments (pointers and sizes), tuning and
 * profiling setting as one of the last 16 recorded ticks.  A replay runs the
 * same kernels, reads the inputs afresh and advances the world's device state
 * exactly like direct launches, so results are identical; it only saves the
 * launch overhead.  enable = 0 launches the kernels directly.  A stream that
 * is itself being recorded always gets direct launches.  On by default. */
knn_status knn_world_set_graphs(knn_world w, int32_t enable);

/* How the last tick's expansion was served (synchronizes the world's last
 * stream): *gathered = packets (of up to 32 queries) the gathered form
 * finished, *handed_back = packets it handed to the packet walk (no object
 * near the packet, a search box of more than 4096 cells, or queries still
 * short of k objects after two thresholds); both 0 unless the tick used the
 * gathered form.  After the tiled form the gathered form only sees the
 * packets the tiles passed on, so the two counts add up to those.  Either may
 * be NULL.  Rows are identical either way. */
knn_status knn_world_expand_info(knn_world w, int64_t *gathered, int64_t *handed_back);

/* Records the graph of a tick with these arguments without running it, so
 * that a later knn_tick with the same arguments (and the same tuning and
 * profiling setting) replays it from its first call; for a loop that cycles a
 * fixed set of input and output buffers.  At most 16 are kept per world.
 * KNN_ERR_INVALID when graphs are off or the arguments would be rejected by
 * knn_tick. */
knn_status knn_world_record_tick(knn_world w, const knn_tick_args *args);

/* Per-stage device times of ticks.  When enabled, each tick records CUDA
 * events around its stages on its stream; knn_world_stage_times synchronizes
 * and writes up to n_stages milliseconds for the last tick.  Stage names come
 * from knn_stage_name (NULL past the last stage): update, keys+sort, leaves,
 * query order, packets, expand (the tick's first expansion kernel) and
 * pass-on (the kernels that finish the packets it passed on: the gathered
 * form after the tiled one, the packet walk after the gathered one). */
knn_status knn_world_set_profiling(knn_world w, int32_t enable);
knn_status knn_world_stage_times(knn_world w, float *ms_host, int32_t n_stages);
const char *knn_stage_name(int32_t i);

/* ---- allocation-free one-shot call --------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that must not allocate device memory: latency-critical loops (cudaMalloc and
 * cudaFree can synchronize the device and take milliseconds), services whose
 * device memory belongs to another allocator or a fixed budget, and code that
 * must not fail half-way through a request because an allocation did.
 *
 * knn_query_static answers n_q k-NN queries over n objects at x_dev/y_dev
 * exactly as knn_world_create + one knn_tick without updates would (same
 * rows, bit for bit), but creates no world and allocates nothing: its scratch
 * is one static device array of 8 MiB that every GPU loading this library
 * holds until the process exits.  Limits: n in [1, 65536], n_q in [0, 65536],
 * k in [1, 512], cell-map level at most 8; larger sizes return
 * KNN_ERR_INVALID.  desc gives the domain, leaf_capacity and max_depth
 * (k_max and max_queries are ignored).  Positions are only read.
 *
 * The first call on each device looks the array's device address up (with
 * that device current); make that first call before any stream capture.
 * Every call reuses the same array and finds the previous call's contents in
 * it; each call clears what must start at zero (error words, scan status
 * words) before its first kernel.  Calls that overlap on the GPU (other
 * streams, other host threads without ordering) race and corrupt each other's
 * results.  Device-side input problems give padded rows, as in knn_tick, but
 * are not reported (there is no world to hold a status); a bounded device wait
 * that gave up turns every row of the call into padding (-1, +inf).
 * Asynchronous on `stream`. */
knn_status knn_query_static(const knn_world_desc *desc, const float *x_dev,
                            const float *y_dev, int64_t n, const int32_t *q_id_dev,
                            const float *q_x_dev, const float *q_y_dev, int64_t n_q,
                            int32_t k, int32_t *out_ids_dev, float *out_d2_dev,
                            void *stream);

#ifdef __cplusplus
}
#endif
#endif /* KNN_H */
