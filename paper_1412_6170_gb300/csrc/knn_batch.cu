// Batched ticks over many worlds, and the per-world autotuner.
//
// knn_batch_tick records the tick of every world of a batch into one CUDA
// graph: each world's index stages form an independent chain, the chains are
// spread over internal streams between a fork and a join on the caller's
// stream, so the GPU runs small worlds side by side and the whole batch costs
// one graph launch.  The expansion runs batched: per form and list size one
// persistent grid over the packets of all the class's worlds, started as soon
// as that class's chains are done.  The executable graph is kept and replayed while the batch keeps the
// same worlds, sizes and pointers (a steady serving or simulation loop); any
// change records the batch again and updates the graph in place.  Every tick
// takes its look-back epochs and update stamps from device counters, so a
// replay is a genuine new tick.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "knn.h"
#include "knn_internal.h"

using knnq::World;

namespace {

constexpr int kMaxStreams = 16;

struct BatchGraph {
    int device = -1;
    std::vector<knn_world> worlds;
    std::vector<knn_tick_args> args;
    std::vector<int> shape;  // per world: plan and which stages run
    cudaGraphExec_t exec = nullptr;
    // the batch is recorded on internal non-blocking streams (the caller's
    // stream may be the legacy default stream, which cannot be recorded);
    // streams[0] is the origin of the fork and the target of the join
    cudaStream_t streams[kMaxStreams] = {};
    cudaEvent_t fork = nullptr, join[kMaxStreams] = {};
    int64_t nodes = 0;
    // The batched expansion: the worlds' expansion arguments by list size
    // class (device table, written when the batch is recorded, after the last
    // replay that read it has finished), the prefix arrays and the tickets.
    void *table = nullptr;
    size_t table_bytes = 0;
    std::vector<char> host;
    // one stream per expansion class; cls_done[c][i]: stream i has finished
    // the index chains of class c's worlds (and of every world before them)
    cudaStream_t cstreams[10] = {};
    cudaEvent_t cls_done[10][kMaxStreams] = {};
    cudaEvent_t cjoin[10] = {};
    cudaEvent_t done = nullptr;  // after the last launch of the graph
    bool pending = false;
};

// One list size class of the batched expansion, and where its parts sit in
// the table.
struct ExpandClass {
    int kc = 0;
    bool walk = false;             // worlds on the packet walk (else the gathered form)
    std::vector<int32_t> members;  // world indices
    std::vector<int32_t> tiled;    // the members whose tiles run first (a gathered class)
    size_t gather_off = 0, walk_off = 0, pfx_g_off = 0, pfx_w_off = 0, ctr_off = 0;
    size_t tile_off = 0, pfx_t_off = 0, ctr_t_off = 0;
};

constexpr int kClasses[5] = {4, 8, 16, 32, 64};

int class_of(int32_t k) {
    for (int c = 0; c < 5; ++c)
        if (k <= kClasses[c]) return c;
    return 4;
}

size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

std::mutex g_mu;
BatchGraph g_batch[64];

knn_status bad(knn_status st, const char *msg) {
    knnq::set_last_error(msg);
    return st;
}

bool same_args(const knn_tick_args &a, const knn_tick_args &b) {
    return std::memcmp(&a, &b, sizeof(knn_tick_args)) == 0;
}

knn_status ensure_streams(BatchGraph &g) {
    if (g.fork) return KNN_OK;
    if (cudaEventCreateWithFlags(&g.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming) != cudaSuccess)
        return bad(KNN_ERR_CUDA, "knn_batch_tick: event creation failed");
    for (int i = 0; i < kMaxStreams; ++i) {
        if (cudaStreamCreateWithFlags(&g.streams[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&g.join[i], cudaEventDisableTiming) != cudaSuccess)
            return bad(KNN_ERR_CUDA, "knn_batch_tick: stream creation failed");
    }
    for (int c = 0; c < 10; ++c) {
        if (cudaStreamCreateWithFlags(&g.cstreams[c], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&g.cjoin[c], cudaEventDisableTiming) != cudaSuccess)
            return bad(KNN_ERR_CUDA, "knn_batch_tick: stream creation failed");
        for (int i = 0; i < kMaxStreams; ++i)
            if (cudaEventCreateWithFlags(&g.cls_done[c][i], cudaEventDisableTiming) != cudaSuccess)
                return bad(KNN_ERR_CUDA, "knn_batch_tick: event creation failed");
    }
    return KNN_OK;
}

// Lays out the batched-expansion table of the worlds whose plan is the
// gathered form (and, for the tiled ones among them, their tile arguments and
// tile-count prefix), fills its host copy and copies it to the device
// (growing the device buffer), after the graph's last replay has finished
// with it.
knn_status build_expand_table(BatchGraph &g, int32_t n_worlds, const knn_world *worlds,
                              const knn_tick_args *args, const std::vector<knnq::Plan> &plans,
                              std::vector<ExpandClass> &classes, std::vector<char> &batched,
                              std::vector<char> &tiled) {
    classes.clear();
    batched.assign(n_worlds, 0);
    tiled.assign(n_worlds, 0);
    ExpandClass by[10];  // gathered form by list size, then the packet walk by list size
    for (int32_t i = 0; i < n_worlds; ++i) {
        const knnq::Plan &p = plans[i];
        if (p.wide || p.iterative || args[i].n_q <= 0) continue;
        batched[i] = 1;
        ExpandClass &e = by[(p.gather ? 0 : 5) + class_of(args[i].k)];
        e.members.push_back(i);
        if (p.gather && p.tile && args[i].q_x_dev == nullptr) {
            tiled[i] = 1;
            e.tiled.push_back(i);
        }
    }
    const size_t gsz = knnq::gather_batch_entry_bytes(), wsz = knnq::walk_batch_entry_bytes();
    const size_t tsz = knnq::tile_batch_entry_bytes();
    size_t off = 0;
    for (int c = 0; c < 10; ++c) {
        ExpandClass &e = by[c];
        if (e.members.empty()) continue;
        const size_t n = e.members.size();
        e.kc = kClasses[c % 5];
        e.walk = c >= 5;
        e.gather_off = off;
        if (!e.walk) off = align16(off + n * gsz);
        e.walk_off = off;
        off = align16(off + n * wsz);
        e.pfx_g_off = off;
        off = align16(off + (n + 1) * sizeof(long long));
        e.pfx_w_off = off;
        off = align16(off + (n + 1) * sizeof(long long));
        e.ctr_off = off;
        off = align16(off + 2 * sizeof(unsigned long long));
        if (!e.tiled.empty()) {
            const size_t nt = e.tiled.size();
            e.tile_off = off;
            off = align16(off + nt * tsz);
            e.pfx_t_off = off;
            off = align16(off + (nt + 1) * sizeof(long long));
            e.ctr_t_off = off;
            off = align16(off + sizeof(unsigned long long));
        }
        classes.push_back(e);
    }
    if (classes.empty()) return KNN_OK;
    g.host.assign(off, 0);
    for (const ExpandClass &e : classes) {
        for (size_t j = 0; j < e.members.size(); ++j) {
            const int32_t i = e.members[j];
            knnq::World &w = worlds[i]->w;
            if (!e.walk)
                knnq::gather_batch_entry(w, plans[i], args[i],
                                         g.host.data() + e.gather_off + j * gsz);
            knnq::walk_batch_entry(w, plans[i], args[i], !e.walk,
                                   g.host.data() + e.walk_off + j * wsz);
        }
        long long *pfx = reinterpret_cast<long long *>(g.host.data() + e.pfx_t_off);
        long long acc = 0;
        for (size_t j = 0; j < e.tiled.size(); ++j) {
            const int32_t i = e.tiled[j];
            pfx[j] = acc;
            acc += knnq::tile_batch_entry(worlds[i]->w, plans[i], args[i],
                                          g.host.data() + e.tile_off + j * tsz);
        }
        if (!e.tiled.empty()) pfx[e.tiled.size()] = acc;
    }
    if (g.pending && cudaEventSynchronize(g.done) != cudaSuccess)
        return bad(KNN_ERR_CUDA, "knn_batch_tick: waiting for the last batch failed");
    g.pending = false;
    if (off > g.table_bytes) {
        if (g.table) cudaFree(g.table);
        g.table = nullptr;
        g.table_bytes = 0;
        if (cudaMalloc(&g.table, off) != cudaSuccess) {
            cudaGetLastError();
            return bad(KNN_ERR_OOM, "knn_batch_tick: no device memory for the expansion table");
        }
        g.table_bytes = off;
    }
    if (cudaMemcpy(g.table, g.host.data(), off, cudaMemcpyHostToDevice) != cudaSuccess)
        return bad(KNN_ERR_CUDA, "knn_batch_tick: copying the expansion table failed");
    return KNN_OK;
}

}  // namespace

extern "C" knn_status knn_batch_tick(int32_t n_worlds, const knn_world *worlds,
                                     const knn_tick_args *args, void *stream) {
    if (n_worlds < 0 || (n_worlds > 0 && (!worlds || !args)))
        return bad(KNN_ERR_INVALID, "knn_batch_tick: bad world list");
    if (n_worlds == 0) return KNN_OK;
    knnq::NvtxRange range("knnq batch_tick");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return bad(KNN_ERR_CUDA, "knn_batch_tick: bad device");
    for (int32_t i = 0; i < n_worlds; ++i) {
        if (!worlds[i]) return bad(KNN_ERR_INVALID, "knn_batch_tick: NULL world");
        if (worlds[i]->w.device != dev)
            return bad(KNN_ERR_INVALID, "knn_batch_tick: world on another device");
        for (int32_t j = 0; j < i; ++j)
            if (worlds[j] == worlds[i])
                return bad(KNN_ERR_INVALID, "knn_batch_tick: a world appears twice");
        const knn_status st = knnq::check_tick_args(worlds[i]->w, args[i], "knn_batch_tick");
        if (st != KNN_OK) return st;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    BatchGraph &g = g_batch[dev];
    g.device = dev;
    knn_status st = ensure_streams(g);
    if (st != KNN_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;

    // Shape: the plan of every world (and whether updates run) fixes the graph's
    // nodes; the world's uid and scratch generation pin the pointers recorded
    // in it (a world destroyed and created again at the same handle address,
    // or whose scratch moved, is recorded again).
    std::vector<int> shape;
    std::vector<knnq::Plan> plans;
    shape.reserve(11 * n_worlds);
    plans.reserve(n_worlds);
    for (int32_t i = 0; i < n_worlds; ++i) {
        const knnq::Plan p = knnq::plan_for(worlds[i]->w, args[i].n_q, args[i].k);
        plans.push_back(p);
        const knnq::World &wi = worlds[i]->w;
        shape.insert(shape.end(), {p.th, p.G, p.Gp, (int)p.wide, (int)p.gather, (int)p.tile,
                                   args[i].n_upd > 0, args[i].q_x_dev != nullptr,
                                   args[i].n_q > 0, (int)(wi.uid & 0x7fffffffu),
                                   (int)(wi.uid >> 31), (int)wi.scratch_gen});
    }
    bool reuse = g.exec && (int32_t)g.worlds.size() == n_worlds && g.shape == shape;
    for (int32_t i = 0; reuse && i < n_worlds; ++i)
        reuse = g.worlds[i] == worlds[i] && same_args(g.args[i], args[i]);

    if (!reuse) {
        knnq::NvtxRange rec("knnq batch record");
        // a failed record below must not leave an older recording replayable
        g.worlds.clear();
        g.shape.clear();
        std::vector<ExpandClass> classes;
        std::vector<char> batched, tiled;
        st = build_expand_table(g, n_worlds, worlds, args, plans, classes, batched, tiled);
        if (st != KNN_OK) return st;
        cudaGraph_t graph = nullptr;
        cudaStream_t origin = g.streams[0];
        cudaError_t e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return bad(KNN_ERR_CUDA, cudaGetErrorString(e));
        const int ns = n_worlds < kMaxStreams ? n_worlds : kMaxStreams;
        cudaEventRecord(g.fork, origin);
        for (int i = 1; i < ns; ++i) cudaStreamWaitEvent(g.streams[i], g.fork, 0);
        int64_t launches0 = 0, launches1 = 0, batch_launches = 0;
        for (int32_t i = 0; i < n_worlds; ++i) launches0 += worlds[i]->w.launches;
        // Every world's index stages (and the expansion of the worlds that are
        // not batched) as independent chains, round robin over the streams,
        // class by class with the costliest expansion class first (query
        // count x list size).  Once a class's chains are done on every
        // stream, its own stream runs one gathered-expansion grid over the
        // packets of all its worlds and one packet-walk grid over what they
        // handed back (a walk class: one walk grid), so the expansion of the
        // first classes overlaps the index stages of the later ones.
        std::vector<size_t> corder(classes.size());
        for (size_t c = 0; c < classes.size(); ++c) corder[c] = c;
        auto cost = [&](size_t c) {
            double q = 0.0;
            for (int32_t i : classes[c].members) q += (double)args[i].n_q;
            return q * classes[c].kc;
        };
        std::sort(corder.begin(), corder.end(),
                  [&](size_t a0, size_t b0) { return cost(a0) > cost(b0); });
        char *tb = static_cast<char *>(g.table);
        int32_t pos = 0;
        for (size_t r = 0; r < corder.size(); ++r) {
            const size_t c = corder[r];
            const ExpandClass &x = classes[c];
            for (int32_t i : x.members)
                knnq::enqueue_tick(worlds[i]->w, args[i], g.streams[pos++ % ns], false, false,
                                   tiled[i] != 0);
            cudaStream_t cs = g.cstreams[r];
            for (int i = 0; i < ns; ++i) {
                cudaEventRecord(g.cls_done[r][i], g.streams[i]);
                cudaStreamWaitEvent(cs, g.cls_done[r][i], 0);
            }
            const int n = (int)x.members.size();
            unsigned long long *ctr = reinterpret_cast<unsigned long long *>(tb + x.ctr_off);
            if (!x.tiled.empty()) {
                // the tiles of the class's tiled worlds; what they pass on joins
                // those worlds' packet lists for the gathered grid
                knnq::launch_tile_batch(
                    x.kc, tb + x.tile_off, (int)x.tiled.size(),
                    reinterpret_cast<const long long *>(tb + x.pfx_t_off),
                    reinterpret_cast<unsigned long long *>(tb + x.ctr_t_off), dev, cs);
                batch_launches += 1;
            }
            if (!x.walk) {
                knnq::launch_gather_batch(x.kc, tb + x.gather_off, n,
                                          reinterpret_cast<long long *>(tb + x.pfx_g_off), ctr,
                                          dev, cs);
                batch_launches += 2;
            }
            knnq::launch_walk_batch(x.kc, tb + x.walk_off, n,
                                    reinterpret_cast<long long *>(tb + x.pfx_w_off), ctr + 1, dev,
                                    cs);
            batch_launches += 2;
            cudaEventRecord(g.cjoin[r], cs);
        }
        for (int32_t i = 0; i < n_worlds; ++i)
            if (!batched[i])
                knnq::enqueue_tick(worlds[i]->w, args[i], g.streams[pos++ % ns], false, true);
        for (int32_t i = 0; i < n_worlds; ++i) launches1 += worlds[i]->w.launches;
        launches1 += batch_launches;
        for (int i = 1; i < ns; ++i) {
            cudaEventRecord(g.join[i], g.streams[i]);
            cudaStreamWaitEvent(origin, g.join[i], 0);
        }
        for (size_t r = 0; r < corder.size(); ++r) cudaStreamWaitEvent(origin, g.cjoin[r], 0);
        e = cudaStreamEndCapture(origin, &graph);
        if (e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return bad(KNN_ERR_CUDA, cudaGetErrorString(e));
        }
        bool updated = false;
        if (g.exec) {
            cudaGraphExecUpdateResultInfo info;
            updated = cudaGraphExecUpdate(g.exec, graph, &info) == cudaSuccess;
            if (!updated) {
                cudaGetLastError();
                cudaGraphExecDestroy(g.exec);
                g.exec = nullptr;
            }
        }
        if (!updated) {
            e = cudaGraphInstantiate(&g.exec, graph, 0);
            if (e != cudaSuccess) {
                cudaGraphDestroy(graph);
                g.exec = nullptr;
                return bad(KNN_ERR_CUDA, cudaGetErrorString(e));
            }
        }
        cudaGraphDestroy(graph);
        g.worlds.assign(worlds, worlds + n_worlds);
        g.args.assign(args, args + n_worlds);
        g.shape = shape;
        g.nodes = launches1 - launches0;
    }
    const cudaError_t e = cudaGraphLaunch(g.exec, s);
    if (e != cudaSuccess) return bad(KNN_ERR_CUDA, cudaGetErrorString(e));
    if (cudaEventRecord(g.done, s) == cudaSuccess) g.pending = true;
    int64_t per_world = g.nodes / (n_worlds ? n_worlds : 1);
    for (int32_t i = 0; i < n_worlds; ++i) {
        worlds[i]->w.last_stream = s;
        if (reuse) worlds[i]->w.launches += per_world;
    }
    return KNN_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: time a few index/expansion settings on the world's own data (ticks
// without updates, so the world's state is unchanged; every setting gives the
// same rows) and keep the fastest.

extern "C" knn_status knn_world_autotune(knn_world h, const int32_t *q_id_dev,
                                         const float *q_x_dev, const float *q_y_dev,
                                         int64_t n_q, int32_t k, int32_t *out_ids_dev,
                                         float *out_d2_dev, int32_t trials, knn_tuning *chosen,
                                         void *stream) {
    if (!h) return bad(KNN_ERR_INVALID, "knn_world_autotune: NULL world");
    knnq::NvtxRange range("knnq world_autotune");
    World &w = h->w;
    knn_tick_args a{nullptr, nullptr, nullptr, 0, q_id_dev, q_x_dev, q_y_dev, n_q, k,
                    out_ids_dev, out_d2_dev, nullptr};
    knn_status st = knnq::check_tick_args(w, a, "knn_world_autotune");
    if (st != KNN_OK) return st;
    if (trials < 1) trials = 1;
    cudaSetDevice(w.device);
    cudaStream_t s = (cudaStream_t)stream;
    const knn_tuning saved = w.tuning;
    knn_tuning automatic{};
    automatic.leaf_capacity = saved.leaf_capacity;  // a capacity fixed at creation stays
    w.tuning = automatic;
    const knnq::Plan p0 = knnq::plan_for(w, n_q, k);
    const int gmax = w.gmax;

    // candidates: leaf capacity x cell-map level x packet level around the automatic plan
    std::vector<knn_tuning> cand;
    const int ths[3] = {p0.th / 2 > 4 ? p0.th / 2 : 4, p0.th, p0.th * 2 < 4096 ? p0.th * 2 : 4096};
    for (int ti = 0; ti < 3; ++ti) {
        const int th = ths[ti];
        const int gauto = (int)std::floor(std::log(2.0 * (double)w.n / th) / std::log(4.0) + 0.5);
        for (int dg = -1; dg <= 1; ++dg) {
            const int G = gauto + dg;
            if (G < 1 || G > gmax) continue;
            for (int dp = 1; dp <= 2; ++dp) {
                const int Gp = G - dp;
                if (Gp < 0) continue;
                cand.push_back(knn_tuning{th, G, Gp, 0});
            }
        }
    }
    // Each setting is timed as a recorded graph of `trials` ticks (device time,
    // as the ticks run inside a batch or a replayed tick graph; direct launches
    // would time the host's launch gaps of small worlds instead).
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        w.tuning = saved;
        return bad(KNN_ERR_CUDA, "knn_world_autotune: stream creation failed");
    }
    auto time_setting = [&](const knn_tuning &t, float *ms) -> bool {
        w.tuning = t;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return false;
        for (int r = 0; r < trials; ++r) knnq::enqueue_tick(w, a, cs, false);
        if (cudaStreamEndCapture(cs, &graph) != cudaSuccess) return false;
        bool ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
        cudaGraphDestroy(graph);
        ok = ok && cudaGraphLaunch(exec, s) == cudaSuccess;  // warm
        ok = ok && cudaEventRecord(e0, s) == cudaSuccess;
        ok = ok && cudaGraphLaunch(exec, s) == cudaSuccess;
        ok = ok && cudaEventRecord(e1, s) == cudaSuccess;
        ok = ok && cudaEventSynchronize(e1) == cudaSuccess;
        if (ok) cudaEventElapsedTime(ms, e0, e1);
        if (exec) cudaGraphExecDestroy(exec);
        return ok;
    };
    auto finish = [&](knn_status st) {
        cudaStreamDestroy(cs);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        // the timed graphs ran on s, the last one with the last plan captured
        w.last_stream = s;
        return st;
    };
    float auto_ms = 0.f;
    if (!time_setting(automatic, &auto_ms)) {
        w.tuning = saved;
        cudaGetLastError();
        return finish(bad(KNN_ERR_CUDA, "knn_world_autotune: a trial tick failed"));
    }
    float best = auto_ms;
    knn_tuning best_t = automatic;
    for (const knn_tuning &t : cand) {
        float ms = 0.f;
        if (!time_setting(t, &ms)) {
            w.tuning = saved;
            cudaGetLastError();
            return finish(bad(KNN_ERR_CUDA, "knn_world_autotune: a trial tick failed"));
        }
        if (ms < best) {
            best = ms;
            best_t = t;
        }
    }
    // then the expansion form on the best index setting: threads per query (one
    // lane in packets, or a whole warp) and how candidates are staged (leaf by
    // leaf along the walk, gathered for the whole search box at once, or
    // staged once per tile of queries)
    std::vector<int> forms = {1, 2};
    if (k <= 32) {
        forms.push_back(4);
        forms.push_back(5);
    }
    const knn_tuning base_t = best_t;
    for (int f : forms) {
        knn_tuning t = base_t;
        t.expansion = f;
        float ms = 0.f;
        if (!time_setting(t, &ms)) {
            w.tuning = saved;
            cudaGetLastError();
            return finish(bad(KNN_ERR_CUDA, "knn_world_autotune: a trial tick failed"));
        }
        if (ms < best) {
            best = ms;
            best_t = t;
        }
    }
    // keep the automatic setting unless another one is clearly (3 %) faster
    if (!(best < 0.97f * auto_ms)) best_t = automatic;
    w.tuning = best_t;
    if (chosen) *chosen = best_t;
    return finish(KNN_OK);
}

// ---------------------------------------------------------------------------
// Batch autotuner: the settings of a batch's worlds chosen by timing the whole
// batch (a world's best setting alone is not its best inside a batch, where
// the batched expansion already fills the GPU with many worlds' packets).
// Worlds are grouped by list size class; per class (largest query count
// first) the expansion form is tried (gathered packets, packet walk, one warp
// per query), then half and twice the leaf capacity; a change is kept only if
// the batch gets clearly (3 %) faster.  Ticks run without updates, so the
// worlds' positions are unchanged.

extern "C" knn_status knn_batch_autotune(int32_t n_worlds, const knn_world *worlds,
                                         const knn_tick_args *args, int32_t trials,
                                         knn_tuning *chosen, void *stream) {
    if (n_worlds < 0 || (n_worlds > 0 && (!worlds || !args)))
        return bad(KNN_ERR_INVALID, "knn_batch_autotune: bad world list");
    if (n_worlds == 0) return KNN_OK;
    for (int32_t i = 0; i < n_worlds; ++i)
        if (!worlds[i]) return bad(KNN_ERR_INVALID, "knn_batch_autotune: NULL world");
    knnq::NvtxRange range("knnq batch_autotune");
    if (trials < 1) trials = 1;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<knn_tick_args> a(args, args + n_worlds);
    for (knn_tick_args &x : a) {
        x.upd_id_dev = nullptr;
        x.upd_x_dev = nullptr;
        x.upd_y_dev = nullptr;
        x.n_upd = 0;
    }
    std::vector<knn_tuning> saved(n_worlds), cur(n_worlds);
    for (int32_t i = 0; i < n_worlds; ++i) {
        saved[i] = worlds[i]->w.tuning;
        cur[i] = knn_tuning{saved[i].leaf_capacity, 0, 0, 0};  // a capacity fixed at creation stays
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto restore = [&](knn_status st) {
        for (int32_t i = 0; i < n_worlds; ++i) worlds[i]->w.tuning = saved[i];
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return st;
    };
    // device time of one batch tick with the settings t (recorded, one warm
    // replay, then `trials` timed replays)
    auto time_batch = [&](const std::vector<knn_tuning> &t, float *ms) -> knn_status {
        for (int32_t i = 0; i < n_worlds; ++i) worlds[i]->w.tuning = t[i];
        for (int r = 0; r < 2; ++r) {
            const knn_status st = knn_batch_tick(n_worlds, worlds, a.data(), stream);
            if (st != KNN_OK) return st;
        }
        if (cudaEventRecord(e0, s) != cudaSuccess)
            return bad(KNN_ERR_CUDA, "knn_batch_autotune: event record failed");
        for (int r = 0; r < trials; ++r) {
            const knn_status st = knn_batch_tick(n_worlds, worlds, a.data(), stream);
            if (st != KNN_OK) return st;
        }
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
            return bad(KNN_ERR_CUDA, "knn_batch_autotune: a timed batch failed");
        cudaEventElapsedTime(ms, e0, e1);
        *ms /= (float)trials;
        return KNN_OK;
    };
    float best = 0.f;
    knn_status st = time_batch(cur, &best);
    if (st != KNN_OK) return restore(st);

    // classes: the packet list sizes, then the lists above them (one warp per query only)
    std::vector<std::vector<int32_t>> members(6);
    std::vector<int64_t> queries(6, 0);
    for (int32_t i = 0; i < n_worlds; ++i) {
        const int c = a[i].k > knnq::kMaxPacketK ? 5 : class_of(a[i].k);
        members[c].push_back(i);
        queries[c] += a[i].n_q;
    }
    std::vector<int> order;
    for (int c = 0; c < 5; ++c)
        if (!members[c].empty() && queries[c] > 0) order.push_back(c);
    std::sort(order.begin(), order.end(), [&](int x, int y) { return queries[x] > queries[y]; });
    auto try_setting = [&](const std::vector<knn_tuning> &t) -> knn_status {
        float ms = 0.f;
        const knn_status r = time_batch(t, &ms);
        if (r != KNN_OK) return r;
        if (ms < 0.97f * best) {
            best = ms;
            cur = t;
        }
        return KNN_OK;
    };
    for (int c : order) {
        // the expansion form
        for (int form : {1, 2, 4}) {
            std::vector<knn_tuning> t = cur;
            for (int32_t i : members[c]) t[i].expansion = form;
            if ((st = try_setting(t)) != KNN_OK) return restore(st);
        }
        // the leaf capacity (with the cell-map and packet levels that follow from it)
        for (int scale : {-1, 1}) {
            std::vector<knn_tuning> t = cur;
            for (int32_t i : members[c]) {
                worlds[i]->w.tuning = cur[i];
                const int th = knnq::plan_for(worlds[i]->w, a[i].n_q, a[i].k).th;
                const int th2 = scale < 0 ? th / 2 : th * 2;
                t[i].leaf_capacity = th2 < 4 ? 4 : (th2 > 4096 ? 4096 : th2);
                t[i].grid_level = 0;
                t[i].packet_level = 0;
            }
            if ((st = try_setting(t)) != KNN_OK) return restore(st);
        }
    }
    for (int32_t i = 0; i < n_worlds; ++i) {
        worlds[i]->w.tuning = cur[i];
        if (chosen) chosen[i] = cur[i];
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return KNN_OK;
}
