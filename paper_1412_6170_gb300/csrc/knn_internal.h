// Host-side internals: the world object and the kernel launchers.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "knn.h"

namespace knnq {

// A named range on the host timeline for profilers that read NVTX (a push at
// construction, a pop at destruction; without a profiler attached each is a
// test of one function pointer).  The library's ranges are named "knnq ...".
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

constexpr int kMaxK = 512;        // largest k of any tick
constexpr int kMaxPacketK = 64;   // largest k of the packet expansion kernel
constexpr int kMaxGridLevel = 10;
constexpr int kMaxLeafCapacity = 4096;
constexpr int kMaxStages = 12;
constexpr int kNumCounters = 32;

// Radix sort tile: 256 threads x 16 keys.
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;
// Leaf split tile.
constexpr int kLeafTile = 1024;
// Single-value scan tile.
constexpr int kScanTile = 2048;

// Device scalars written by kernels and read by later kernels.
// Index reuse state (scratch, so an evicted world rebuilds): the signature
// of the plan the leaves were built for, the index's age in ticks, this
// tick's rebuild flag, and the leaves' sum of squared counts (a cost proxy)
// right after the build and at the last tick (64-bit, two words each).
enum Scalar : int { kScalarLeaves = 0, kScalarValidQueries = 1, kScalarPackets = 2,
                    kScalarIndexSig = 3, kScalarIndexAge = 4, kScalarRebuild = 5,
                    kScalarCostBase = 6, kScalarCostNow = 8, kScalarPartialPackets = 10,
                    kScalarHandedBack = 11, kNumScalars = 16 };

// Ticket counters (one per single-pass launch site in a tick).
enum Counter : int { kCtrObjSort = 0, kCtrQuerySort = 4, kCtrLeaves = 8, kCtrQueryScan = 9,
                     kCtrExpand = 11, kCtrReuseScan = 12,
                     kCtrIterLeft = 13 /* and 14: iterative expansion */, kCtrGather = 15,
                     kCtrHandBack = 16, kCtrTile = 17 };

struct Plan {
    int L;           // max depth (key has 2L bits)
    int th;          // leaf capacity
    int G;           // cell-map level (min leaf level)
    int Gp;          // packet level
    int passes;      // radix passes over 2L bits
    bool wide;       // expansion by one warp per query (else packets)
    bool gather;     // packets gather their search box at once (the rest: packet walk)
    bool tile;       // queries at issuers: one block per level-Gp cell stages its margin once
                     // and each lane scans its own box (the rest: gathered packets)
    bool iterative;  // expansion in the paper's multi-pass form (an ablation)
    int reuse_age;   // index reuse: rebuild at least every reuse_age ticks (0: every tick)
    int reuse_f16;   // and when the cost proxy grows past reuse_f16 / 16 of its built value
    bool by_id;      // queries at issuers counted by issuer id (most objects query): the
                     // leaf split then writes no inverse order
};

// A whole tick recorded as a CUDA graph, with what it was recorded for.
struct TickGraph {
    knn_tick_args args{};
    Plan plan{};
    bool marks = false;
    cudaGraphExec_t exec = nullptr;
    uint64_t used = 0;      // recency stamp
    int64_t launches = 0;   // kernels in the graph
};
constexpr int kTickGraphs = 16;

struct World {
    // unique per world created in this process, and bumped whenever the tick
    // scratch moves: a recorded batch that holds the world's pointers is valid
    // only for the (uid, scratch_gen) it was recorded with
    uint64_t uid = 0;
    uint32_t scratch_gen = 0;
    int device = 0;
    knn_world_desc desc{};
    int64_t n = 0;
    int L = 16;
    int gmax = 10;         // deepest cell-map level this world sizes its arrays for
    float scale = 0.f;     // 2^L / side, binary32
    knn_tuning tuning{};   // user overrides (0 = auto)
    int reuse_age = 0;     // index reuse (knn_world_set_index_reuse)
    float reuse_factor = 0.f;
    uint32_t site = 0;     // look-back launch index within the current tick
    cudaStream_t last_stream = nullptr;
    Plan last_plan{};

    // device memory: the resident part (positions, update stamps, counters)
    // lives as long as the world; the tick scratch can be released and
    // allocated again (a serving loop evicts idle worlds' scratch)
    void *arena_res = nullptr;
    size_t res_bytes = 0;
    void *arena = nullptr;       // tick scratch (nullptr while evicted)
    size_t arena_bytes = 0;
    bool arena_async = false;    // scratch from cudaMallocAsync (freed with cudaFreeAsync)

    float *px = nullptr, *py = nullptr;
    unsigned long long *stamp = nullptr;
    uint32_t *key[2] = {nullptr, nullptr};
    int32_t *val[2] = {nullptr, nullptr};
    float *xs = nullptr, *ys = nullptr;
    int32_t *sid = nullptr, *inv = nullptr;
    uint32_t *skey = nullptr;  // sorted object keys (copy kept for queries)
    int32_t *bstart = nullptr;
    uint32_t *bcode = nullptr;
    uint8_t *blevel = nullptr;
    float4 *baabb = nullptr;
    int2 *brange = nullptr;      // leaf b holds sorted objects [x, y)
    int64_t leaf_cap = 0;        // room for leaves (objects' ones + empty level-G cells)
    int32_t *lcnt = nullptr;     // index reuse: objects per leaf
    int32_t *obj_leaf = nullptr; // leaf of every sorted object
    int32_t *cb = nullptr;
    int32_t *qcnt = nullptr, *qoff = nullptr;
    float *qs_x = nullptr, *qs_y = nullptr;
    int32_t *qs_id = nullptr, *qs_orig = nullptr;
    uint32_t *qs_key = nullptr;
    int32_t *qs_leaf = nullptr;  // a leaf at (or next to) each sorted query
    uint32_t *nav = nullptr;     // iterative expansion: per sorted query, left and right position
    int32_t *qcs = nullptr;
    int32_t *pk_start = nullptr, *pk_len = nullptr;
    int2 *hb = nullptr;          // packets handed from the gathered form to the walk
    uint64_t *status = nullptr;
    size_t status_words = 0;
    uint32_t *hist = nullptr;
    uint32_t *counters = nullptr;
    // [0] look-back epoch base, [1] update stamp tick; advanced on the device by
    // k_tick_begin so that a recorded tick can be replayed (CUDA graphs)
    uint32_t *tickinfo = nullptr;
    int32_t *scalars = nullptr;
    uint32_t *err = nullptr;

    // host-pointer tick staging (grown on demand)
    void *stage = nullptr;
    size_t stage_bytes = 0;

    // pipelined host-buffer ticks (knn_tick_host_submit): two staging slots
    // used in turn, one copy stream per direction, per-slot events (inputs in,
    // tick run, rows out)
    struct HostSlot {
        void *buf = nullptr;
        size_t bytes = 0;
        cudaEvent_t in = nullptr, ran = nullptr, done = nullptr;
    } hslot[2];
    cudaStream_t h2d = nullptr, d2h = nullptr;
    int64_t tickets = 0;

    // kernels launched by this world's ticks so far
    int64_t launches = 0;

    // profiling
    bool profiling = false;
    cudaEvent_t ev[kMaxStages + 1] = {};
    int n_stage_events = 0;

    // knn_tick replays a recorded graph when its arguments, plan and profiling
    // marks match one of the last kTickGraphs ticks (least recently used goes)
    bool graphs = true;
    int host_io = 1;  // knn_tick_host: bit 0 writes rows, bit 1 reads inputs in pinned host memory
    TickGraph tick_graph[kTickGraphs];
    uint64_t tick_clock = 0;
    cudaStream_t capture_stream = nullptr;

    int64_t max_rows() const { return n > desc.max_queries ? n : desc.max_queries; }
};

}  // namespace knnq

// The opaque handle of the C ABI.
struct knn_world_s {
    knnq::World w;
};

namespace knnq {

// Automatic leaf capacity th (the paper ties th_quad to k; a performance knob
// only).  Measured on 1M uniform objects, all querying: leaves of about 15
// objects (level-8 cells) serve k from 4 to 32 best, so th = k + 16 for the
// packet kernel (k = 8: 5 % and k = 32: 9 % faster than th = 2k); the warp
// per query (k > 32) keeps th = 2k.  Clamped to [8, 256].
inline int default_leaf_capacity(int k) {
    const int th = k <= 32 ? k + 16 : 2 * k;
    return th < 8 ? 8 : (th > 256 ? 256 : th);
}

// l_max when the world's descriptor leaves it to the library (Section 4.1.1
// fixes l_max without a value): 12 while a uniform world would hold at most
// one object per 16 level-12 cells (n <= 4^12 / 16), so that the Morton keys
// have 24 bits and the radix sort three 8-bit passes; 16 (32-bit keys, four
// passes) for larger worlds.  Rows do not depend on it: a leaf at l_max may
// hold more than th_quad objects and is searched like any other.
inline int default_max_depth(int64_t n) { return n <= (int64_t(1) << 20) ? 12 : 16; }

// Packets never exceed n_q/32 + (non-empty packet cells) <= n_q + n_q/32 + 1.
inline int64_t packet_capacity(const World &w) {
    return w.desc.max_queries + w.desc.max_queries / 32 + 2;
}



// ---- launchers (knn_index.cu) ----------------------------------------------
void launch_validate_positions(const float *x, const float *y, int64_t n, uint32_t *flag,
                               cudaStream_t s);
// Start of a tick: advance epoch base and stamp tick, clear tickets and the abort flag.
void launch_tick_begin(World &w, const Plan &p, cudaStream_t s);
void launch_index_reuse(World &w, const Plan &p, cudaStream_t s);
void launch_updates(World &w, const int32_t *id, const float *ux, const float *uy,
                    int64_t n_upd, cudaStream_t s);
void launch_object_sort(World &w, const Plan &p, cudaStream_t s);
void launch_leaves(World &w, const Plan &p, cudaStream_t s);
void launch_queries_at_issuers(World &w, const Plan &p, const int32_t *q_id, int64_t n_q,
                               int32_t k, int32_t *out_ids, float *out_d2, cudaStream_t s);
void launch_queries_explicit(World &w, const Plan &p, const int32_t *q_id, const float *q_x,
                             const float *q_y, int64_t n_q, int32_t k, int32_t *out_ids,
                             float *out_d2, cudaStream_t s);
void launch_packets(World &w, const Plan &p, int64_t n_q, cudaStream_t s);
// First sorted query of every level-Gp cell (qcs); also clears the packet
// counts.
void launch_query_cells(World &w, const Plan &p, int64_t n_q, cudaStream_t s);
// One bounded device wait that nothing satisfies (failure-detection check).
void launch_wait_runs_out(World &w, cudaStream_t s);
// One failing bounds check (debug builds only; the access is skipped).
void launch_bounds_check_probe(World &w, cudaStream_t s);
void launch_export_leaves(World &w, int64_t m, int32_t *level, uint32_t *z, int32_t *start,
                          int32_t *count, cudaStream_t s);

// ---- launcher (knn_expand.cu) -----------------------------------------------
void launch_expand(World &w, const Plan &p, int32_t k, int64_t n_q, int32_t *out_ids,
                   float *out_d2, const int32_t *q_k, cudaStream_t s);
void launch_expand_wide(World &w, const Plan &p, int32_t k, int64_t n_q, int32_t *out_ids,
                        float *out_d2, const int32_t *q_k, cudaStream_t s);
void launch_expand_iter(World &w, const Plan &p, int32_t k, int64_t n_q, int32_t *out_ids,
                        float *out_d2, const int32_t *q_k, cudaStream_t s);
// The packet walk over the packets the gathered form handed back.
void launch_expand_handed_back(World &w, const Plan &p, int32_t k, int64_t n_q,
                               int32_t *out_ids, float *out_d2, const int32_t *q_k,
                               cudaStream_t s);
// ---- launcher (knn_expand_tile.cu) -------------------------------------------
// The tiled form over the level-Gp cells of the sorted queries (queries at
// their issuers, packets not cut): what it cannot finish it appends to the
// packet list, for launch_expand_gather.
void launch_expand_tile(World &w, const Plan &p, int32_t k, int64_t n_q, int32_t *out_ids,
                        float *out_d2, const int32_t *q_k, cudaStream_t s);
// ---- launcher (knn_expand_gather.cu) -----------------------------------------
// The gathered form, then (then_walk) the packet walk over the packets it
// handed back.
void launch_expand_gather(World &w, const Plan &p, int32_t k, int64_t n_q, int32_t *out_ids,
                          float *out_d2, const int32_t *q_k, cudaStream_t s,
                          bool then_walk = true);

// ---- batched expansion over many worlds (knn_expand_gather.cu, knn_expand.cu)
// A batch table holds one entry per world (the world's expansion arguments,
// filled on the host and copied to the device once per recorded batch).  One
// launch per list size then expands the packets of every world of the table:
// a one-block prefix kernel counts each world's packets on the device (pfx,
// n + 1 entries) and resets the ticket counter, and a persistent grid takes
// tickets across all worlds.  The walk form does the same over the packets
// the gathered form handed back, or over the packets of the worlds that run
// the packet walk.  kc: the list size class (4, 8, 16, 32, 64).
size_t gather_batch_entry_bytes();
void gather_batch_entry(World &w, const Plan &p, const knn_tick_args &t, void *dst);
void launch_gather_batch(int kc, const void *table, int n, long long *pfx,
                         unsigned long long *counter, int device, cudaStream_t s);
// The tiled form over many worlds (queries at their issuers, k <= 32): the
// worlds' tile arguments, their tile counts as a prefix (pfx, n + 1 entries,
// filled on the host: a world's tile count follows from its plan), and one
// grid per list size that takes tiles of every world; what the tiles pass on
// goes to each world's packet list, for the batched gathered form.
size_t tile_batch_entry_bytes();
// Fills dst with the world's tile arguments; returns its tile count.
int64_t tile_batch_entry(World &w, const Plan &p, const knn_tick_args &t, void *dst);
void launch_tile_batch(int kc, const void *table, int n, const long long *pfx,
                       unsigned long long *counter, int device, cudaStream_t s);
size_t walk_batch_entry_bytes();
// handed_back: the entry covers the packets the gathered form handed back
// (else the world's own packet list, for worlds on the packet walk)
void walk_batch_entry(World &w, const Plan &p, const knn_tick_args &t, bool handed_back,
                      void *dst);
void launch_walk_batch(int kc, const void *table, int n, long long *pfx,
                       unsigned long long *counter, int device, cudaStream_t s);

int num_sms(int device);
// One-time kernel attributes and cached device queries (called outside any
// stream capture).
void prepare_kernels();
void prepare_expand(int device);
void prepare_expand_wide(int device);
void prepare_expand_gather(int device);
void prepare_expand_tile(int device);

// Device memory layout of a world (knn_capi.cu).  base == nullptr only sizes.
size_t carve_resident(World &w, char *base);
size_t carve_scratch(World &w, char *base);
// Creates the resident part of a world (positions copied and validated);
// the scratch is left unallocated.  Sets the error message on failure.
knn_status world_init_resident(World &w, const knn_world_desc *desc, const float *x_dev,
                               const float *y_dev, int64_t n, cudaStream_t s);
// Points the scratch fields into `base` (scratch_bytes) and clears what must
// start at zero, on stream s.
void world_attach_scratch(World &w, void *base, cudaStream_t s);

// Message returned by knn_last_error() on this thread (knn_capi.cu).
void set_last_error(const char *msg);
// Host-side argument checks of one tick (sets the error message).
knn_status check_tick_args(const World &w, const knn_tick_args &a, const char *who);
// Enqueue every stage of one tick on s; `marks` records stage events when
// the world's profiling is on.  expand == false stops after the packets are
// cut (a batch expands them), or, with batch_tiles, after the query cells of
// the tiled form (a batch runs its tiles).
void enqueue_tick(World &w, const knn_tick_args &a, cudaStream_t s, bool marks,
                  bool expand = true, bool batch_tiles = false);
// One tick through the world's graph cache when graphs are on (else direct).
knn_status tick_launch(World &w, const knn_tick_args &a, cudaStream_t s);
// The index / expansion parameters a tick with n_q queries and this k uses.
Plan plan_for(const World &w, int64_t n_q, int k);

}  // namespace knnq
