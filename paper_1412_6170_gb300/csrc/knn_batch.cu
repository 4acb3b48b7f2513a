// Batched ticks over many worlds, and the per-world autotuner.
//
// knn_batch_tick records the tick of every world of a batch into one CUDA
// graph: each world's stages form an independent chain, the chains are spread
// over internal streams between a fork and a join on the caller's stream, so
// the GPU runs small worlds side by side and the whole batch costs one graph
// launch.  The executable graph is kept and replayed while the batch keeps the
// same worlds, sizes and pointers (a steady serving or simulation loop); any
// change records the batch again and updates the graph in place.  Every tick
// takes its look-back epochs and update stamps from device counters, so a
// replay is a genuine new tick.
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
};

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
    if (cudaEventCreateWithFlags(&g.fork, cudaEventDisableTiming) != cudaSuccess)
        return bad(KNN_ERR_CUDA, "knn_batch_tick: event creation failed");
    for (int i = 0; i < kMaxStreams; ++i) {
        if (cudaStreamCreateWithFlags(&g.streams[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&g.join[i], cudaEventDisableTiming) != cudaSuccess)
            return bad(KNN_ERR_CUDA, "knn_batch_tick: stream creation failed");
    }
    return KNN_OK;
}

}  // namespace

extern "C" knn_status knn_batch_tick(int32_t n_worlds, const knn_world *worlds,
                                     const knn_tick_args *args, void *stream) {
    if (n_worlds < 0 || (n_worlds > 0 && (!worlds || !args)))
        return bad(KNN_ERR_INVALID, "knn_batch_tick: bad world list");
    if (n_worlds == 0) return KNN_OK;
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

    // Shape: the plan of every world (and whether updates run) fixes the graph's nodes.
    std::vector<int> shape;
    shape.reserve(8 * n_worlds);
    for (int32_t i = 0; i < n_worlds; ++i) {
        const knnq::Plan p = knnq::plan_for(worlds[i]->w, args[i].n_q, args[i].k);
        shape.insert(shape.end(), {p.th, p.G, p.Gp, (int)p.wide, (int)p.gather,
                                   args[i].n_upd > 0, args[i].q_x_dev != nullptr,
                                   args[i].n_q > 0});
    }
    bool reuse = g.exec && (int32_t)g.worlds.size() == n_worlds && g.shape == shape;
    for (int32_t i = 0; reuse && i < n_worlds; ++i)
        reuse = g.worlds[i] == worlds[i] && same_args(g.args[i], args[i]);

    if (!reuse) {
        cudaGraph_t graph = nullptr;
        cudaStream_t origin = g.streams[0];
        cudaError_t e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return bad(KNN_ERR_CUDA, cudaGetErrorString(e));
        const int ns = n_worlds < kMaxStreams ? n_worlds : kMaxStreams;
        cudaEventRecord(g.fork, origin);
        for (int i = 1; i < ns; ++i) cudaStreamWaitEvent(g.streams[i], g.fork, 0);
        int64_t launches0 = 0, launches1 = 0;
        for (int32_t i = 0; i < n_worlds; ++i) launches0 += worlds[i]->w.launches;
        for (int32_t i = 0; i < n_worlds; ++i)
            knnq::enqueue_tick(worlds[i]->w, args[i], g.streams[i % ns], false);
        for (int32_t i = 0; i < n_worlds; ++i) launches1 += worlds[i]->w.launches;
        for (int i = 1; i < ns; ++i) {
            cudaEventRecord(g.join[i], g.streams[i]);
            cudaStreamWaitEvent(origin, g.join[i], 0);
        }
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
    // leaf along the walk, or gathered for the whole search box at once)
    std::vector<int> forms = {1, 2};
    if (k <= 32) forms.push_back(4);
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
