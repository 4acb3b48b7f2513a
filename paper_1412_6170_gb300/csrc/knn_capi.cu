// C ABI (include/knn.h): argument validation, the world's device arena, the
// order of the per-tick stages, host-buffer ticks, status and introspection.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "knn.h"
#include "knn_internal.h"

using knnq::Plan;
using knnq::World;

namespace {

thread_local char g_err[512] = "";

knn_status fail(knn_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

knn_status cuda_fail(cudaError_t e, const char *what) {
    return fail(KNN_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// "expand" is the tick's first expansion kernel; "pass-on" the kernels that
// finish what it passed on (the gathered form after the tiled one, the packet
// walk after the gathered one; empty for the other forms).
const char *kStageNames[] = {"update", "keys+sort", "leaves", "query order", "packets",
                             "expand", "pass-on"};
constexpr int kNumStages = 7;

int round_log4(double v) {
    if (v <= 1.0) return 0;
    return (int)std::floor(std::log(v) / std::log(4.0) + 0.5);
}

int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Automatic index parameters (none changes a result):
//  leaf capacity th = default_leaf_capacity(k);
//  grid level G with about th/2 objects per cell, so most leaves are cells;
//  packet level with about max(48, 12k) queries per cell.
Plan make_plan(const World &w, int64_t n_q, int k) {
    Plan p{};
    p.L = w.L;
    p.passes = (2 * p.L + 7) / 8;
    p.th = w.tuning.leaf_capacity > 0 ? w.tuning.leaf_capacity : knnq::default_leaf_capacity(k);
    p.th = clampi(p.th, 1, knnq::kMaxLeafCapacity);
    const int gmax = w.gmax;
    int G = w.tuning.grid_level > 0 ? w.tuning.grid_level
                                    : round_log4(2.0 * (double)w.n / (double)p.th);
    p.G = clampi(G, 1, gmax);
    // about max(48, 12 k) queries per packet cell (measured on 1M uniform
    // objects, all querying: k <= 8 best at ~61 per cell, k = 32 at ~244)
    int Gp = w.tuning.packet_level > 0
                 ? w.tuning.packet_level
                 : round_log4((double)(n_q > 0 ? n_q : 1) / (k > 4 ? 12.0 * k : 48.0));
    p.Gp = clampi(Gp, 0, p.G);
    // one warp per query pays off above k = 32 (measured on 1M uniform objects:
    // k = 64 takes 2.8 ms that way against 3.5 ms in packets)
    p.iterative = w.tuning.expansion == 3 && k <= knnq::kMaxPacketK;
    p.wide = !p.iterative && (w.tuning.expansion == 2 || (w.tuning.expansion == 0 && k > 32) ||
                              k > knnq::kMaxPacketK);
    // packets gather their search box at once (k <= 32) unless the packet walk
    // is asked for (measured on 1M uniform objects, all querying: k = 8 0.26
    // against 0.33 ms, k = 16 0.39 against 0.43 ms, k = 32 0.87 against 0.86
    // ms for the walk; 4M clustered objects, a quarter querying, k = 32: 1.53
    // against 1.58 ms)
    p.gather = !p.iterative && !p.wide && k <= knnq::kMaxPacketK &&
               (w.tuning.expansion == 4 || w.tuning.expansion == 5 ||
                (w.tuning.expansion == 0 && k <= 32));
    // the tiled form (queries at issuers; the gathered form finishes what it
    // passes on) for k <= 32 (measured on 1M uniform objects, all querying:
    // k = 8 0.17 against 0.26 ms, k = 16 0.23 against 0.39 ms, k = 32 0.45
    // against 0.85 ms for the gathered form)
    p.tile = p.gather && k <= 32 && (w.tuning.expansion == 5 || w.tuning.expansion == 0);
    if (p.tile && w.tuning.packet_level <= 0)
        p.Gp = clampi(round_log4((double)(n_q > 0 ? n_q : 1) / 200.0), 0, p.G);
    p.by_id = 2 * n_q >= w.n;
    p.reuse_age = w.reuse_age;
    p.reuse_f16 = w.reuse_factor > 0.f ? (int)std::lround(w.reuse_factor * 16.f) : 0;
    return p;
}

size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

struct Carve {
    char *base;
    size_t off = 0;
    template <class T>
    T *take(size_t count) {
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += align_up(sizeof(T) * (count ? count : 1));
        return p;
    }
};

}  // namespace

namespace knnq {

// Resident part: positions, update stamps, tick counters, error words.
size_t carve_resident(World &w, char *base) {
    const int64_t n = w.n;
    Carve c{base};
    w.px = c.take<float>(n);
    w.py = c.take<float>(n);
    w.stamp = c.take<unsigned long long>(n);
    w.tickinfo = c.take<uint32_t>(4);
    w.err = c.take<uint32_t>(4);
    return c.off;
}

// Tick scratch: sort buffers, leaf-ordered SoA, leaves, cell map, queries,
// packets, look-back status words, histograms and tickets.
size_t carve_scratch(World &w, char *base) {
    const int64_t n = w.n, R = w.max_rows(), Q = w.desc.max_queries;
    const int64_t ncell = (1ll << (2 * w.gmax)) + 2;
    const int64_t sort_tiles = (R + kSortTile - 1) / kSortTile;
    int64_t status = sort_tiles * 256;
    // leaves: at most one per object, plus (index reuse) one per empty level-G cell
    const int64_t lcap = n + (1ll << (2 * w.gmax)) + 1;
    const int64_t others[] = {(n + kLeafTile - 1) / kLeafTile,
                              (n + 1 + kScanTile - 1) / kScanTile,
                              (ncell + kScanTile - 1) / kScanTile,
                              (lcap + 1 + kScanTile - 1) / kScanTile};
    for (int64_t o : others) status = status > o ? status : o;
    Carve c{base};
    w.leaf_cap = lcap;
    w.key[0] = c.take<uint32_t>(R);
    w.key[1] = c.take<uint32_t>(R);
    w.val[0] = c.take<int32_t>(R);
    w.val[1] = c.take<int32_t>(R);
    w.xs = c.take<float>(n);
    w.ys = c.take<float>(n);
    w.sid = c.take<int32_t>(n);
    w.inv = c.take<int32_t>(n);
    w.bstart = c.take<int32_t>(lcap + 1);
    w.bcode = c.take<uint32_t>(lcap);
    w.blevel = c.take<uint8_t>(lcap);
    w.baabb = c.take<float4>(lcap);
    w.brange = c.take<int2>(lcap);
    w.lcnt = c.take<int32_t>(lcap + 1);
    w.obj_leaf = c.take<int32_t>(n);
    w.cb = c.take<int32_t>(ncell);
    w.qcnt = c.take<int32_t>(n + 1);
    w.qoff = c.take<int32_t>(n + 2);
    w.qs_x = c.take<float>(Q);
    w.qs_y = c.take<float>(Q);
    w.qs_id = c.take<int32_t>(Q);
    w.qs_orig = c.take<int32_t>(Q);
    w.qs_key = c.take<uint32_t>(Q);
    w.qs_leaf = c.take<int32_t>(Q);
    w.nav = c.take<uint32_t>(2 * Q);
    w.qcs = c.take<int32_t>(ncell);
    w.pk_start = c.take<int32_t>(Q + Q / 32 + 2);
    w.pk_len = c.take<int32_t>(Q + Q / 32 + 2);
    w.hb = c.take<int2>(Q + Q / 32 + 2);
    w.status = c.take<uint64_t>(status);
    w.status_words = (size_t)status;
    w.hist = c.take<uint32_t>(4 * 256);
    w.counters = c.take<uint32_t>(kNumCounters);
    w.scalars = c.take<int32_t>(kNumScalars);
    return c.off;
}

void world_attach_scratch(World &w, void *base, cudaStream_t s) {
    // recorded tick graphs point into the old scratch
    for (TickGraph &t : w.tick_graph) {
        if (t.exec) cudaGraphExecDestroy(t.exec);
        t.exec = nullptr;
    }
    w.arena = base;
    ++w.scratch_gen;
    carve_scratch(w, static_cast<char *>(base));
    cudaMemsetAsync(w.scalars, 0, sizeof(int32_t) * kNumScalars, s);
    // look-back status words must not hold anything that could match a live epoch
    cudaMemsetAsync(w.status, 0, sizeof(uint64_t) * w.status_words, s);
}

knn_status world_init_resident(World &w, const knn_world_desc *desc, const float *x_dev,
                               const float *y_dev, int64_t n, cudaStream_t s) {
    if (!desc) return fail(KNN_ERR_INVALID, "NULL world description");
    if (!(desc->side > 0.f) || !std::isfinite(desc->side) || !std::isfinite(desc->x0) ||
        !std::isfinite(desc->y0))
        return fail(KNN_ERR_INVALID, "world: domain must be finite with side > 0");
    if (n < 1 || n > (1ll << 30))
        return fail(KNN_ERR_INVALID, "world: n=%lld outside [1, 2^30]", (long long)n);
    if (desc->k_max < 1 || desc->k_max > kMaxK)
        return fail(KNN_ERR_INVALID, "world: k_max=%d outside [1, %d]", desc->k_max, kMaxK);
    if (desc->max_depth < 0 || desc->max_depth > 16)
        return fail(KNN_ERR_INVALID, "world: max_depth=%d outside [0, 16]", desc->max_depth);
    if (desc->leaf_capacity < 0 || desc->leaf_capacity > kMaxLeafCapacity)
        return fail(KNN_ERR_INVALID, "world: leaf_capacity=%d outside [0, 4096]",
                    desc->leaf_capacity);
    if (desc->max_queries < 0 || desc->max_queries > (1ll << 30))
        return fail(KNN_ERR_INVALID, "world: max_queries outside [0, 2^30]");
    if (!x_dev || !y_dev) return fail(KNN_ERR_INVALID, "world: NULL positions");
    cudaGetDevice(&w.device);
    static std::atomic<uint64_t> next_uid{0};
    w.uid = ++next_uid;
    w.desc = *desc;
    w.n = n;
    w.L = desc->max_depth > 0 ? desc->max_depth : knnq::default_max_depth(n);
    // a cell map with more than ~4 cells per object never pays off
    int g = 1;
    while (g < kMaxGridLevel && g < w.L && (1ll << (2 * g)) < 4 * n) ++g;
    w.gmax = g;
    w.scale = (float)(1u << w.L) / desc->side;
    w.tuning.leaf_capacity = desc->leaf_capacity;
    w.res_bytes = carve_resident(w, nullptr);
    w.arena_bytes = carve_scratch(w, nullptr);
    cudaError_t e = cudaMalloc(&w.arena_res, w.res_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        w.arena_res = nullptr;
        return fail(KNN_ERR_OOM, "world: cudaMalloc(%zu) failed: %s", w.res_bytes,
                    cudaGetErrorString(e));
    }
    carve_resident(w, static_cast<char *>(w.arena_res));
    prepare_kernels();
    cudaMemsetAsync(w.stamp, 0, sizeof(unsigned long long) * (size_t)n, s);
    cudaMemsetAsync(w.err, 0, 16, s);
    cudaMemsetAsync(w.tickinfo, 0, 16, s);
    cudaMemcpyAsync(w.px, x_dev, sizeof(float) * (size_t)n, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(w.py, y_dev, sizeof(float) * (size_t)n, cudaMemcpyDeviceToDevice, s);
    launch_validate_positions(w.px, w.py, n, w.err + 1, s);
    uint32_t bad = 0;
    cudaMemcpyAsync(&bad, w.err + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "world creation");
    if (bad) return fail(KNN_ERR_INVALID, "world: non-finite initial position");
    cudaMemsetAsync(w.err, 0, 16, s);
    w.last_stream = s;
    return KNN_OK;
}

}  // namespace knnq

namespace {

void release(World &w) {
    if (w.arena) {
        if (w.arena_async) cudaFreeAsync(w.arena, w.last_stream);
        else cudaFree(w.arena);
    }
    if (w.arena_res) cudaFree(w.arena_res);
    w.arena_res = nullptr;
    if (w.stage) cudaFree(w.stage);
    for (int i = 0; i <= knnq::kMaxStages; ++i)
        if (w.ev[i]) cudaEventDestroy(w.ev[i]);
    for (knnq::TickGraph &t : w.tick_graph) {
        if (t.exec) cudaGraphExecDestroy(t.exec);
        t.exec = nullptr;
    }
    if (w.capture_stream) cudaStreamDestroy(w.capture_stream);
    w.capture_stream = nullptr;
    for (World::HostSlot &hs : w.hslot) {
        if (hs.done) cudaEventSynchronize(hs.done);
        if (hs.buf) cudaFree(hs.buf);
        for (cudaEvent_t e : {hs.in, hs.ran, hs.done})
            if (e) cudaEventDestroy(e);
        hs = World::HostSlot{};
    }
    if (w.h2d) cudaStreamDestroy(w.h2d);
    if (w.d2h) cudaStreamDestroy(w.d2h);
    w.h2d = w.d2h = nullptr;
    w.arena = nullptr;
    w.stage = nullptr;
}

bool same_tick(const knnq::TickGraph &t, const knn_tick_args &a, const knnq::Plan &p,
               bool marks) {
    return t.exec && t.marks == marks && std::memcmp(&t.args, &a, sizeof(a)) == 0 &&
           std::memcmp(&t.plan, &p, sizeof(p)) == 0;
}

// The world's graph for a tick with these arguments: a cached one, else this
// tick recorded (on an internal stream: the caller's stream may be the legacy
// default stream, which cannot be recorded) into the least recently used slot
// (updated in place, or instantiated anew).  *recorded tells which.
knn_status tick_graph(World &w, const knn_tick_args &a, knnq::TickGraph **out, bool *recorded) {
    const knnq::Plan p = knnq::plan_for(w, a.n_q, a.k);
    const bool marks = w.profiling;
    *recorded = false;
    knnq::TickGraph *hit = nullptr, *victim = &w.tick_graph[0];
    for (knnq::TickGraph &t : w.tick_graph) {
        if (same_tick(t, a, p, marks)) {
            hit = &t;
            break;
        }
        if (!t.exec || (victim->exec && t.used < victim->used)) victim = &t;
    }
    if (!hit) {
        if (!w.capture_stream &&
            cudaStreamCreateWithFlags(&w.capture_stream, cudaStreamNonBlocking) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "knn_tick: stream creation");
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(w.capture_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "knn_tick: begin capture");
        const int64_t l0 = w.launches;
        const cudaStream_t last_stream = w.last_stream;
        const knnq::Plan last_plan = w.last_plan;
        knnq::enqueue_tick(w, a, w.capture_stream, marks);
        w.last_stream = last_stream;  // nothing ran yet
        w.last_plan = last_plan;
        const int64_t launches = w.launches - l0;
        e = cudaStreamEndCapture(w.capture_stream, &graph);
        if (e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(e, "knn_tick: end capture");
        }
        bool updated = false;
        if (victim->exec) {
            cudaGraphExecUpdateResultInfo info;
            updated = cudaGraphExecUpdate(victim->exec, graph, &info) == cudaSuccess;
            if (!updated) {
                cudaGetLastError();
                cudaGraphExecDestroy(victim->exec);
                victim->exec = nullptr;
            }
        }
        if (!updated) {
            e = cudaGraphInstantiate(&victim->exec, graph, 0);
            if (e != cudaSuccess) {
                victim->exec = nullptr;
                cudaGraphDestroy(graph);
                return cuda_fail(e, "knn_tick: instantiate");
            }
        }
        cudaGraphDestroy(graph);
        victim->args = a;
        victim->plan = p;
        victim->marks = marks;
        victim->launches = launches;
        w.launches -= launches;  // counted when the graph runs
        hit = victim;
        *recorded = true;
    }
    hit->used = ++w.tick_clock;
    *out = hit;
    return KNN_OK;
}

// One tick through the world's graph cache.
knn_status tick_via_graph(World &w, const knn_tick_args &a, cudaStream_t s) {
    knnq::TickGraph *g = nullptr;
    bool recorded = false;
    const knn_status st = tick_graph(w, a, &g, &recorded);
    if (st != KNN_OK) return st;
    const cudaError_t e = cudaGraphLaunch(g->exec, s);
    if (e != cudaSuccess) return cuda_fail(e, "knn_tick: graph launch");
    w.launches += g->launches;
    w.last_stream = s;
    w.last_plan = g->plan;
    return KNN_OK;
}

void mark(World &w, int i, cudaStream_t s) {
    if (w.profiling && i <= knnq::kMaxStages) {
        // while a tick is being recorded, an "external" record becomes an event
        // record node of the graph (a plain one would only mark a dependency)
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(s, &cs);
        if (cs == cudaStreamCaptureStatusActive)
            cudaEventRecordWithFlags(w.ev[i], s, cudaEventRecordExternal);
        else
            cudaEventRecord(w.ev[i], s);
        w.n_stage_events = i + 1;
    }
}

}  // namespace

namespace knnq {
knn_status tick_launch(World &w, const knn_tick_args &a, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    // a stream the caller is recording gets the kernels themselves; the
    // iterative ablation (a cooperative launch) is never recorded
    if (w.graphs && !plan_for(w, a.n_q, a.k).iterative &&
        cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone)
        return tick_via_graph(w, a, s);
    cudaGetLastError();
    enqueue_tick(w, a, s, w.profiling);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "tick launch");
    return KNN_OK;
}

// Lets other translation units of the library report through knn_last_error.
void set_last_error(const char *msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

knn_status check_tick_args(const World &w, const knn_tick_args &a, const char *who) {
    if (a.k < 1 || a.k > w.desc.k_max)
        return fail(KNN_ERR_INVALID, "%s: k=%d outside [1, k_max=%d]", who, a.k, w.desc.k_max);
    if (a.n_q < 0 || a.n_q > w.desc.max_queries)
        return fail(KNN_ERR_INVALID, "%s: n_q=%lld outside [0, max_queries=%lld]", who,
                    (long long)a.n_q, (long long)w.desc.max_queries);
    if (a.n_upd < 0 || a.n_upd >= (1ll << 31))
        return fail(KNN_ERR_INVALID, "%s: n_upd=%lld outside [0, 2^31)", who,
                    (long long)a.n_upd);
    if (a.n_upd > 0 && (!a.upd_id_dev || !a.upd_x_dev || !a.upd_y_dev))
        return fail(KNN_ERR_INVALID, "%s: NULL update array with n_upd > 0", who);
    if ((a.q_x_dev == nullptr) != (a.q_y_dev == nullptr))
        return fail(KNN_ERR_INVALID, "%s: q_x and q_y must both be given or both NULL", who);
    if (a.n_q > 0 && (!a.q_id_dev || !a.out_ids_dev || !a.out_d2_dev))
        return fail(KNN_ERR_INVALID, "%s: NULL query or output array with n_q > 0", who);
    return KNN_OK;
}

// The stages of one tick, in order, on stream s (no synchronisation, no allocation).
void enqueue_tick(World &w, const knn_tick_args &a, cudaStream_t s, bool marks, bool expand,
                  bool batch_tiles) {
    const Plan p = make_plan(w, a.n_q, a.k);
    const bool m = marks && w.profiling;
    launch_tick_begin(w, p, s);
    if (m) mark(w, 0, s);
    {
        NvtxRange r("knnq a1 updates");
        launch_updates(w, a.upd_id_dev, a.upd_x_dev, a.upd_y_dev, a.n_upd, s);
    }
    if (m) mark(w, 1, s);
    {
        NvtxRange r("knnq a2-a3 keys + sort");
        if (p.reuse_age > 0) launch_index_reuse(w, p, s);  // on reuse ticks; else the sort runs
        launch_object_sort(w, p, s);
    }
    if (m) mark(w, 2, s);
    {
        NvtxRange r("knnq a4-a5 leaves");
        launch_leaves(w, p, s);
    }
    if (m) mark(w, 3, s);
    NvtxRange rq("knnq a6 query order, a7-a8 expansion");
    if (a.n_q > 0) {
        if (a.q_x_dev == nullptr)
            launch_queries_at_issuers(w, p, a.q_id_dev, a.n_q, a.k, a.out_ids_dev,
                                      a.out_d2_dev, s);
        else
            launch_queries_explicit(w, p, a.q_id_dev, a.q_x_dev, a.q_y_dev, a.n_q, a.k,
                                    a.out_ids_dev, a.out_d2_dev, s);
    }
    if (m) mark(w, 4, s);
    // the tiled form takes the level-Gp cells of the sorted queries directly
    // and cuts packets only for what it passes on
    const bool tile = p.tile && (expand || batch_tiles) && a.q_x_dev == nullptr;
    if (a.n_q > 0 && !p.wide && !p.iterative) {
        if (tile) launch_query_cells(w, p, a.n_q, s);
        else launch_packets(w, p, a.n_q, s);
    }
    if (m) mark(w, 5, s);
    if (a.n_q > 0 && expand) {
        if (p.gather) {
            if (tile)
                launch_expand_tile(w, p, a.k, a.n_q, a.out_ids_dev, a.out_d2_dev, a.q_k_dev, s);
            else
                launch_expand_gather(w, p, a.k, a.n_q, a.out_ids_dev, a.out_d2_dev, a.q_k_dev, s,
                                     false);
            if (m) mark(w, 6, s);
            if (tile)
                launch_expand_gather(w, p, a.k, a.n_q, a.out_ids_dev, a.out_d2_dev, a.q_k_dev, s,
                                     false);
            launch_expand_handed_back(w, p, a.k, a.n_q, a.out_ids_dev, a.out_d2_dev, a.q_k_dev,
                                      s);
        }
        else {
            if (p.iterative)
                launch_expand_iter(w, p, a.k, a.n_q, a.out_ids_dev, a.out_d2_dev, a.q_k_dev, s);
            else if (p.wide)
                launch_expand_wide(w, p, a.k, a.n_q, a.out_ids_dev, a.out_d2_dev, a.q_k_dev, s);
            else
                launch_expand(w, p, a.k, a.n_q, a.out_ids_dev, a.out_d2_dev, a.q_k_dev, s);
            if (m) mark(w, 6, s);
        }
    } else if (m) {
        mark(w, 6, s);
    }
    if (m) mark(w, 7, s);
    w.last_stream = s;
    w.last_plan = p;
}

Plan plan_for(const World &w, int64_t n_q, int k) { return make_plan(w, n_q, k); }
}  // namespace knnq

extern "C" {

const char *knn_last_error(void) { return g_err; }

const char *knn_stage_name(int32_t i) {
    return (i >= 0 && i < kNumStages) ? kStageNames[i] : nullptr;
}

knn_status knn_world_create(const knn_world_desc *desc, const float *x_dev, const float *y_dev,
                            int64_t n, void *stream, knn_world *out) {
    if (!desc || !out) return fail(KNN_ERR_INVALID, "knn_world_create: NULL desc or out");
    *out = nullptr;
    knn_world_s *h = new (std::nothrow) knn_world_s();
    if (!h) return fail(KNN_ERR_OOM, "knn_world_create: host allocation failed");
    World &w = h->w;
    cudaStream_t s = (cudaStream_t)stream;
    knn_status st = knnq::world_init_resident(w, desc, x_dev, y_dev, n, s);
    if (st != KNN_OK) {
        release(w);
        delete h;
        return st;
    }
    void *scratch = nullptr;
    cudaError_t e = cudaMalloc(&scratch, w.arena_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        release(w);
        delete h;
        return fail(KNN_ERR_OOM, "knn_world_create: cudaMalloc(%zu) failed: %s", w.arena_bytes,
                    cudaGetErrorString(e));
    }
    knnq::world_attach_scratch(w, scratch, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        release(w);
        delete h;
        return cuda_fail(e, "knn_world_create");
    }
    *out = h;
    return KNN_OK;
}

knn_status knn_world_destroy(knn_world h) {
    if (!h) return fail(KNN_ERR_INVALID, "knn_world_destroy: NULL world");
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(h->w.device);
    cudaDeviceSynchronize();
    release(h->w);
    cudaSetDevice(prev);
    delete h;
    return KNN_OK;
}

knn_status knn_world_set_tuning(knn_world h, const knn_tuning *t) {
    if (!h || !t) return fail(KNN_ERR_INVALID, "knn_world_set_tuning: NULL argument");
    if (t->leaf_capacity < 0 || t->leaf_capacity > knnq::kMaxLeafCapacity)
        return fail(KNN_ERR_INVALID, "leaf_capacity outside [0, 4096]");
    if (t->grid_level < 0 || t->grid_level > h->w.gmax)
        return fail(KNN_ERR_INVALID, "grid_level outside [0, %d] for this world", h->w.gmax);
    if (t->packet_level < 0 || t->packet_level > knnq::kMaxGridLevel)
        return fail(KNN_ERR_INVALID, "packet_level outside [0, 10]");
    if (t->expansion < 0 || t->expansion > 5)
        return fail(KNN_ERR_INVALID, "expansion outside [0, 5]");
    h->w.tuning = *t;
    return KNN_OK;
}

knn_status knn_world_get_tuning(knn_world h, int64_t n_q, int32_t k, knn_tuning *out) {
    if (!h || !out) return fail(KNN_ERR_INVALID, "knn_world_get_tuning: NULL argument");
    Plan p = make_plan(h->w, n_q, k);
    out->leaf_capacity = p.th;
    out->grid_level = p.G;
    out->packet_level = p.Gp;
    out->expansion = p.iterative ? 3 : (p.wide ? 2 : (p.tile ? 5 : (p.gather ? 4 : 1)));
    return KNN_OK;
}

knn_status knn_tick(knn_world h, const int32_t *upd_id, const float *upd_x, const float *upd_y,
                    int64_t n_upd, const int32_t *q_id, const float *q_x, const float *q_y,
                    int64_t n_q, int32_t k, int32_t *out_ids, float *out_d2, void *stream) {
    if (!h) return fail(KNN_ERR_INVALID, "knn_tick: NULL world");
    knnq::NvtxRange range("knnq tick");
    knn_tick_args a{upd_id, upd_x, upd_y, n_upd, q_id, q_x, q_y, n_q, k, out_ids, out_d2,
                    nullptr};
    const knn_status st = knnq::check_tick_args(h->w, a, "knn_tick");
    if (st != KNN_OK) return st;
    World &w = h->w;
    cudaSetDevice(w.device);
    return knnq::tick_launch(w, a, (cudaStream_t)stream);
}

knn_status knn_tick_ex(knn_world h, const knn_tick_args *args, void *stream) {
    if (!h || !args) return fail(KNN_ERR_INVALID, "knn_tick_ex: NULL argument");
    knnq::NvtxRange range("knnq tick");
    const knn_status st = knnq::check_tick_args(h->w, *args, "knn_tick_ex");
    if (st != KNN_OK) return st;
    World &w = h->w;
    cudaSetDevice(w.device);
    return knnq::tick_launch(w, *args, (cudaStream_t)stream);
}

// The device-side address of a host array that the runtime has pinned
// (cudaHostAlloc, cudaHostRegister), or NULL (pageable memory, or a device
// array).  Kernels can read and write pinned host memory through it over the
// CPU-GPU link, so the rows can go straight to the caller's buffer while the
// expansion runs instead of being copied after it.
static void *pinned_alias(const void *p) {
    if (!p) return nullptr;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    return a.devicePointer;
}

knn_status knn_tick_host(knn_world h, const int32_t *upd_id, const float *upd_x,
                         const float *upd_y, int64_t n_upd, const int32_t *q_id,
                         const float *q_x, const float *q_y, int64_t n_q, int32_t k,
                         int32_t *out_ids, float *out_d2, void *stream) {
    if (!h) return fail(KNN_ERR_INVALID, "knn_tick_host: NULL world");
    World &w = h->w;
    if (n_upd < 0 || n_q < 0 || k < 1 || k > w.desc.k_max)
        return fail(KNN_ERR_INVALID, "knn_tick_host: bad sizes");
    if (n_upd > 0 && (!upd_id || !upd_x || !upd_y))
        return fail(KNN_ERR_INVALID, "knn_tick_host: NULL update array with n_upd > 0");
    const bool explicit_q = q_x != nullptr;
    if (n_q > 0 && (!q_id || !out_ids || !out_d2 || (explicit_q && !q_y)))
        return fail(KNN_ERR_INVALID, "knn_tick_host: NULL query or output array");
    cudaSetDevice(w.device);
    cudaStream_t s = (cudaStream_t)stream;

    // pinned arrays are used in place (outputs: bit 0 of host_io; inputs: bit 1)
    int32_t *a_oid = nullptr;
    float *a_od = nullptr;
    if ((w.host_io & 1) && n_q > 0) {
        a_oid = static_cast<int32_t *>(pinned_alias(out_ids));
        a_od = static_cast<float *>(pinned_alias(out_d2));
        if (!a_oid || !a_od) a_oid = nullptr, a_od = nullptr;
    }
    const int32_t *a_uid = nullptr, *a_qid = nullptr;
    const float *a_ux = nullptr, *a_uy = nullptr, *a_qx = nullptr, *a_qy = nullptr;
    if (w.host_io & 2) {
        if (n_upd > 0) {
            a_uid = static_cast<const int32_t *>(pinned_alias(upd_id));
            a_ux = static_cast<const float *>(pinned_alias(upd_x));
            a_uy = static_cast<const float *>(pinned_alias(upd_y));
            if (!a_uid || !a_ux || !a_uy) a_uid = nullptr, a_ux = a_uy = nullptr;
        }
        if (n_q > 0) {
            a_qid = static_cast<const int32_t *>(pinned_alias(q_id));
            if (explicit_q) {
                a_qx = static_cast<const float *>(pinned_alias(q_x));
                a_qy = static_cast<const float *>(pinned_alias(q_y));
                if (!a_qx || !a_qy) a_qid = nullptr, a_qx = a_qy = nullptr;
            }
        }
    }
    const bool stage_upd = n_upd > 0 && !a_uid, stage_q = n_q > 0 && !a_qid;
    const bool stage_out = n_q > 0 && !a_oid;

    const size_t b_upd = stage_upd ? align_up(sizeof(int32_t) * (size_t)n_upd) +
                                         2 * align_up(sizeof(float) * (size_t)n_upd)
                                   : 0;
    const size_t b_q = stage_q ? align_up(sizeof(int32_t) * (size_t)n_q) +
                                     (explicit_q ? 2 * align_up(sizeof(float) * (size_t)n_q) : 0)
                               : 0;
    const size_t b_out = stage_out ? align_up(sizeof(int32_t) * (size_t)n_q * k) +
                                         align_up(sizeof(float) * (size_t)n_q * k)
                                   : 0;
    const size_t need = b_upd + b_q + b_out;
    if (need > w.stage_bytes) {
        cudaStreamSynchronize(s);
        if (w.stage) cudaFree(w.stage);
        w.stage = nullptr;
        w.stage_bytes = 0;
        if (cudaMalloc(&w.stage, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(KNN_ERR_OOM, "knn_tick_host: staging allocation of %zu bytes failed",
                        need);
        }
        w.stage_bytes = need;
    }
    Carve c{static_cast<char *>(w.stage)};
    if (stage_upd) {
        int32_t *d_uid = c.take<int32_t>((size_t)n_upd);
        float *d_ux = c.take<float>((size_t)n_upd);
        float *d_uy = c.take<float>((size_t)n_upd);
        cudaMemcpyAsync(d_uid, upd_id, sizeof(int32_t) * n_upd, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_ux, upd_x, sizeof(float) * n_upd, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_uy, upd_y, sizeof(float) * n_upd, cudaMemcpyHostToDevice, s);
        a_uid = d_uid, a_ux = d_ux, a_uy = d_uy;
    }
    if (stage_q) {
        int32_t *d_qid = c.take<int32_t>((size_t)n_q);
        cudaMemcpyAsync(d_qid, q_id, sizeof(int32_t) * n_q, cudaMemcpyHostToDevice, s);
        a_qid = d_qid;
        if (explicit_q) {
            float *d_qx = c.take<float>((size_t)n_q);
            float *d_qy = c.take<float>((size_t)n_q);
            cudaMemcpyAsync(d_qx, q_x, sizeof(float) * n_q, cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(d_qy, q_y, sizeof(float) * n_q, cudaMemcpyHostToDevice, s);
            a_qx = d_qx, a_qy = d_qy;
        }
    }
    int32_t *d_oid = a_oid;
    float *d_od = a_od;
    if (stage_out) {
        d_oid = c.take<int32_t>((size_t)n_q * k);
        d_od = c.take<float>((size_t)n_q * k);
    }
    knn_status st = knn_tick(h, a_uid, a_ux, a_uy, n_upd, a_qid, a_qx, a_qy, n_q, k, d_oid, d_od,
                             stream);
    if (st != KNN_OK) return st;
    if (stage_out) {
        cudaMemcpyAsync(out_ids, d_oid, sizeof(int32_t) * n_q * k, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(out_d2, d_od, sizeof(float) * n_q * k, cudaMemcpyDeviceToHost, s);
    }
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "knn_tick_host");
    return KNN_OK;
}

knn_status knn_tick_host_submit(knn_world h, const int32_t *upd_id, const float *upd_x,
                                const float *upd_y, int64_t n_upd, const int32_t *q_id,
                                const float *q_x, const float *q_y, int64_t n_q, int32_t k,
                                int32_t *out_ids, float *out_d2, void *stream,
                                int64_t *ticket) {
    if (!h || !ticket) return fail(KNN_ERR_INVALID, "knn_tick_host_submit: NULL argument");
    knnq::NvtxRange range("knnq tick_host_submit");
    World &w = h->w;
    const bool explicit_q = q_x != nullptr;
    if (n_upd > 0 && (!upd_id || !upd_x || !upd_y))
        return fail(KNN_ERR_INVALID, "knn_tick_host_submit: NULL update array with n_upd > 0");
    if (n_q > 0 && (!q_id || !out_ids || !out_d2 || (explicit_q && !q_y)))
        return fail(KNN_ERR_INVALID, "knn_tick_host_submit: NULL query or output array");
    if (explicit_q != (q_y != nullptr))
        return fail(KNN_ERR_INVALID, "knn_tick_host_submit: q_x and q_y must both be given");
    {
        // the checks of knn_tick, before anything is enqueued
        knn_tick_args a{};
        a.upd_id_dev = upd_id, a.upd_x_dev = upd_x, a.upd_y_dev = upd_y, a.n_upd = n_upd;
        a.q_id_dev = q_id, a.q_x_dev = q_x, a.q_y_dev = q_y, a.n_q = n_q, a.k = k;
        a.out_ids_dev = out_ids, a.out_d2_dev = out_d2;
        const knn_status st = knnq::check_tick_args(w, a, "knn_tick_host_submit");
        if (st != KNN_OK) return st;
    }
    cudaSetDevice(w.device);
    cudaStream_t s = (cudaStream_t)stream;
    if (!w.h2d || !w.d2h) {
        if ((!w.h2d && cudaStreamCreateWithFlags(&w.h2d, cudaStreamNonBlocking) != cudaSuccess) ||
            (!w.d2h && cudaStreamCreateWithFlags(&w.d2h, cudaStreamNonBlocking) != cudaSuccess))
            return cuda_fail(cudaGetLastError(), "knn_tick_host_submit: copy streams");
    }
    for (World::HostSlot &slot : w.hslot)
        for (cudaEvent_t *e : {&slot.in, &slot.ran, &slot.done})
            if (!*e && cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) {
                *e = nullptr;
                return cuda_fail(cudaGetLastError(), "knn_tick_host_submit: events");
            }
    World::HostSlot &hs = w.hslot[w.tickets & 1];
    const size_t b_upd = align_up(sizeof(int32_t) * (size_t)n_upd) +
                         2 * align_up(sizeof(float) * (size_t)n_upd);
    const size_t b_q = align_up(sizeof(int32_t) * (size_t)n_q) +
                       (explicit_q ? 2 * align_up(sizeof(float) * (size_t)n_q) : 0);
    const size_t b_out = align_up(sizeof(int32_t) * (size_t)n_q * k) +
                         align_up(sizeof(float) * (size_t)n_q * k);
    const size_t need = b_upd + b_q + b_out;
    if (need > hs.bytes) {
        cudaEventSynchronize(hs.done);  // the slot's last ticket is finished
        if (hs.buf) cudaFree(hs.buf);
        hs.buf = nullptr;
        hs.bytes = 0;
        if (cudaMalloc(&hs.buf, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(KNN_ERR_OOM, "knn_tick_host_submit: staging allocation of %zu bytes failed",
                        need);
        }
        hs.bytes = need;
    }
    Carve c{static_cast<char *>(hs.buf)};
    int32_t *d_uid = c.take<int32_t>((size_t)n_upd);
    float *d_ux = c.take<float>((size_t)n_upd);
    float *d_uy = c.take<float>((size_t)n_upd);
    int32_t *d_qid = c.take<int32_t>((size_t)n_q);
    float *d_qx = explicit_q ? c.take<float>((size_t)n_q) : nullptr;
    float *d_qy = explicit_q ? c.take<float>((size_t)n_q) : nullptr;
    int32_t *d_oid = c.take<int32_t>((size_t)n_q * k);
    float *d_od = c.take<float>((size_t)n_q * k);

    // inputs: once the slot's previous rows have left (its buffers are free)
    cudaStreamWaitEvent(w.h2d, hs.done, 0);
    if (n_upd > 0) {
        cudaMemcpyAsync(d_uid, upd_id, sizeof(int32_t) * n_upd, cudaMemcpyHostToDevice, w.h2d);
        cudaMemcpyAsync(d_ux, upd_x, sizeof(float) * n_upd, cudaMemcpyHostToDevice, w.h2d);
        cudaMemcpyAsync(d_uy, upd_y, sizeof(float) * n_upd, cudaMemcpyHostToDevice, w.h2d);
    }
    if (n_q > 0) {
        cudaMemcpyAsync(d_qid, q_id, sizeof(int32_t) * n_q, cudaMemcpyHostToDevice, w.h2d);
        if (explicit_q) {
            cudaMemcpyAsync(d_qx, q_x, sizeof(float) * n_q, cudaMemcpyHostToDevice, w.h2d);
            cudaMemcpyAsync(d_qy, q_y, sizeof(float) * n_q, cudaMemcpyHostToDevice, w.h2d);
        }
    }
    cudaEventRecord(hs.in, w.h2d);
    // the tick, on the caller's stream, after its inputs
    cudaStreamWaitEvent(s, hs.in, 0);
    const knn_status st = knn_tick(h, n_upd ? d_uid : nullptr, n_upd ? d_ux : nullptr,
                                   n_upd ? d_uy : nullptr, n_upd, n_q ? d_qid : nullptr, d_qx,
                                   d_qy, n_q, k, n_q ? d_oid : nullptr, n_q ? d_od : nullptr,
                                   stream);
    if (st != KNN_OK) return st;
    cudaEventRecord(hs.ran, s);
    // rows: after the tick
    cudaStreamWaitEvent(w.d2h, hs.ran, 0);
    if (n_q > 0) {
        cudaMemcpyAsync(out_ids, d_oid, sizeof(int32_t) * n_q * k, cudaMemcpyDeviceToHost, w.d2h);
        cudaMemcpyAsync(out_d2, d_od, sizeof(float) * n_q * k, cudaMemcpyDeviceToHost, w.d2h);
    }
    cudaEventRecord(hs.done, w.d2h);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "knn_tick_host_submit");
    *ticket = w.tickets++;
    return KNN_OK;
}

knn_status knn_tick_host_wait(knn_world h, int64_t ticket) {
    if (!h) return fail(KNN_ERR_INVALID, "knn_tick_host_wait: NULL world");
    World &w = h->w;
    if (ticket < 0 || ticket >= w.tickets)
        return fail(KNN_ERR_INVALID, "knn_tick_host_wait: ticket %lld was not submitted",
                    (long long)ticket);
    cudaSetDevice(w.device);
    // the slot's last rows-out event belongs to this ticket or a later one of
    // the same slot; the copy stream runs them in order
    const cudaError_t e = cudaEventSynchronize(w.hslot[ticket & 1].done);
    if (e != cudaSuccess) return cuda_fail(e, "knn_tick_host_wait");
    return KNN_OK;
}

knn_status knn_world_set_host_io(knn_world h, int32_t mode) {
    if (!h || mode < 0 || mode > 3) return fail(KNN_ERR_INVALID, "knn_world_set_host_io: bad argument");
    h->w.host_io = mode;
    return KNN_OK;
}

knn_status knn_tick_status(knn_world h, uint32_t *bits_out) {
    if (!h) return fail(KNN_ERR_INVALID, "knn_tick_status: NULL world");
    World &w = h->w;
    cudaSetDevice(w.device);
    uint32_t bits = 0;
    cudaError_t e = cudaStreamSynchronize(w.last_stream);
    if (e == cudaSuccess) e = cudaMemcpy(&bits, w.err, sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(w.err, 0, sizeof(uint32_t));
    if (e != cudaSuccess) return cuda_fail(e, "knn_tick_status");
    if (bits_out) *bits_out = bits;
    if (bits & 8u) return fail(KNN_ERR_TIMEOUT, "a bounded device wait ran out");
    if (bits & 16u)
        return fail(KNN_ERR_CUDA, "a device bounds check of the debug build failed (bits 0x%x)",
                    bits);
    if (bits) return fail(KNN_ERR_DEVICE_INPUT, "device skipped invalid input (bits 0x%x)", bits);
    return KNN_OK;
}

knn_status knn_world_leaves(knn_world h, int32_t *level, uint32_t *z, int32_t *start,
                            int32_t *count, int32_t *sorted_ids, int64_t cap, int64_t *m_host,
                            void *stream) {
    if (!h || !m_host) return fail(KNN_ERR_INVALID, "knn_world_leaves: NULL argument");
    World &w = h->w;
    cudaSetDevice(w.device);
    cudaStream_t s = (cudaStream_t)stream;
    int32_t m = 0;
    cudaMemcpyAsync(&m, w.scalars + knnq::kScalarLeaves, sizeof(int32_t), cudaMemcpyDeviceToHost,
                    s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "knn_world_leaves");
    *m_host = m;
    const int64_t c = m < cap ? m : cap;
    if (c > 0 && level && z && start && count)
        knnq::launch_export_leaves(w, c, level, z, start, count, s);
    if (sorted_ids)
        cudaMemcpyAsync(sorted_ids, w.sid, sizeof(int32_t) * (size_t)w.n,
                        cudaMemcpyDeviceToDevice, s);
    e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "knn_world_leaves");
    return KNN_OK;
}

knn_status knn_world_positions(knn_world h, float *x_dev, float *y_dev, void *stream) {
    if (!h || !x_dev || !y_dev) return fail(KNN_ERR_INVALID, "knn_world_positions: NULL argument");
    World &w = h->w;
    cudaSetDevice(w.device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemcpyAsync(x_dev, w.px, sizeof(float) * (size_t)w.n, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(y_dev, w.py, sizeof(float) * (size_t)w.n, cudaMemcpyDeviceToDevice, s);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "knn_world_positions");
    return KNN_OK;
}

knn_status knn_debug_build(void) {
#ifdef KNN_DEBUG
    return KNN_OK;
#else
    return fail(KNN_ERR_INVALID, "not a debug build (compiled without KNN_DEBUG)");
#endif
}

knn_status knn_world_test_bounds_check(knn_world h, void *stream) {
    if (!h) return fail(KNN_ERR_INVALID, "knn_world_test_bounds_check: NULL world");
#ifndef KNN_DEBUG
    return fail(KNN_ERR_INVALID, "knn_world_test_bounds_check: not a debug build");
#else
    World &w = h->w;
    cudaSetDevice(w.device);
    cudaStream_t s = (cudaStream_t)stream;
    knnq::launch_bounds_check_probe(w, s);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "knn_world_test_bounds_check");
    w.last_stream = s;
    return KNN_OK;
#endif
}

knn_status knn_world_test_wait_timeout(knn_world h, void *stream) {
    if (!h) return fail(KNN_ERR_INVALID, "knn_world_test_wait_timeout: NULL world");
    World &w = h->w;
    cudaSetDevice(w.device);
    cudaStream_t s = (cudaStream_t)stream;
    knnq::launch_wait_runs_out(w, s);
    w.last_stream = s;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "knn_world_test_wait_timeout");
    return KNN_OK;
}

knn_status knn_world_launches(knn_world h, int64_t *count) {
    if (!h || !count) return fail(KNN_ERR_INVALID, "knn_world_launches: NULL argument");
    *count = h->w.launches;
    return KNN_OK;
}

knn_status knn_world_set_profiling(knn_world h, int32_t enable) {
    if (!h) return fail(KNN_ERR_INVALID, "knn_world_set_profiling: NULL world");
    World &w = h->w;
    cudaSetDevice(w.device);
    if (enable && !w.ev[0]) {
        for (int i = 0; i <= knnq::kMaxStages; ++i) {
            if (cudaEventCreate(&w.ev[i]) != cudaSuccess)
                return cuda_fail(cudaGetLastError(), "knn_world_set_profiling");
        }
    }
    w.profiling = enable != 0;
    w.n_stage_events = 0;
    return KNN_OK;
}

knn_status knn_world_record_tick(knn_world h, const knn_tick_args *args) {
    if (!h || !args) return fail(KNN_ERR_INVALID, "knn_world_record_tick: NULL argument");
    World &w = h->w;
    const knn_status st = knnq::check_tick_args(w, *args, "knn_world_record_tick");
    if (st != KNN_OK) return st;
    if (!w.graphs) return fail(KNN_ERR_INVALID, "knn_world_record_tick: graphs are off");
    cudaSetDevice(w.device);
    knnq::TickGraph *g = nullptr;
    bool recorded = false;
    knn_status st2 = tick_graph(w, *args, &g, &recorded);
    if (st2 != KNN_OK) return st2;
    // move the graph to the device now rather than at its first launch
    cudaError_t e = cudaGraphUpload(g->exec, w.capture_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w.capture_stream);
    if (e != cudaSuccess) return cuda_fail(e, "knn_world_record_tick: upload");
    return KNN_OK;
}

knn_status knn_world_set_index_reuse(knn_world h, int32_t max_age, float factor) {
    if (!h) return fail(KNN_ERR_INVALID, "knn_world_set_index_reuse: NULL world");
    if (max_age < 0 || !std::isfinite(factor) || factor > 1e6f)
        return fail(KNN_ERR_INVALID, "knn_world_set_index_reuse: bad max_age or factor");
    h->w.reuse_age = max_age;
    h->w.reuse_factor = factor > 0.f ? factor : 0.f;
    return KNN_OK;
}

knn_status knn_world_index_info(knn_world h, int32_t *age, int32_t *rebuilt) {
    if (!h) return fail(KNN_ERR_INVALID, "knn_world_index_info: NULL world");
    World &w = h->w;
    if (!w.arena) return fail(KNN_ERR_INVALID, "knn_world_index_info: world scratch released");
    cudaSetDevice(w.device);
    int32_t v[knnq::kNumScalars];
    cudaError_t e = cudaMemcpyAsync(v, w.scalars, sizeof(v), cudaMemcpyDeviceToHost,
                                    w.last_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w.last_stream);
    if (e != cudaSuccess) return cuda_fail(e, "knn_world_index_info");
    if (age) *age = v[knnq::kScalarRebuild] ? 0 : v[knnq::kScalarIndexAge];
    if (rebuilt) *rebuilt = v[knnq::kScalarRebuild];
    return KNN_OK;
}

knn_status knn_world_expand_info(knn_world h, int64_t *gathered, int64_t *handed_back) {
    if (!h) return fail(KNN_ERR_INVALID, "knn_world_expand_info: NULL world");
    World &w = h->w;
    if (!w.arena) return fail(KNN_ERR_INVALID, "knn_world_expand_info: world scratch released");
    cudaSetDevice(w.device);
    int32_t v[knnq::kNumScalars];
    cudaError_t e = cudaMemcpyAsync(v, w.scalars, sizeof(v), cudaMemcpyDeviceToHost,
                                    w.last_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w.last_stream);
    if (e != cudaSuccess) return cuda_fail(e, "knn_world_expand_info");
    const bool on = w.last_plan.gather;
    const int64_t packets = (int64_t)v[knnq::kScalarPackets] + v[knnq::kScalarPartialPackets];
    const int64_t back = on ? v[knnq::kScalarHandedBack] : 0;
    if (gathered) *gathered = on ? packets - back : 0;
    if (handed_back) *handed_back = back;
    return KNN_OK;
}

knn_status knn_world_set_graphs(knn_world h, int32_t enable) {
    if (!h) return fail(KNN_ERR_INVALID, "knn_world_set_graphs: NULL world");
    h->w.graphs = enable != 0;
    return KNN_OK;
}

knn_status knn_world_stage_times(knn_world h, float *ms, int32_t n_stages) {
    if (!h || !ms) return fail(KNN_ERR_INVALID, "knn_world_stage_times: NULL argument");
    World &w = h->w;
    if (!w.profiling || w.n_stage_events < 2)
        return fail(KNN_ERR_INVALID, "knn_world_stage_times: profiling is off or no tick ran");
    cudaSetDevice(w.device);
    cudaError_t e = cudaEventSynchronize(w.ev[w.n_stage_events - 1]);
    if (e != cudaSuccess) return cuda_fail(e, "knn_world_stage_times");
    for (int i = 0; i < n_stages; ++i) {
        ms[i] = 0.f;
        if (i + 1 < w.n_stage_events) cudaEventElapsedTime(&ms[i], w.ev[i], w.ev[i + 1]);
    }
    return KNN_OK;
}

}  // extern "C"
