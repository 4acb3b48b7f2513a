// Serving loop: tick requests from many resident worlds, admitted as GPU
// slots and device memory free up, run concurrently on separate streams.
//
// The paper's setting is a stream of position updates and queries processed
// tick by tick under a latency requirement (Sections 2.2-2.3): a request is
// one world's tick, its latency the time from submission to the moment its
// results are complete on the device (the tick latency of the paper's
// batch-processing model).  The server keeps every world's positions
// resident and gives a world its tick scratch only while it has work: a
// dispatcher thread admits the oldest request of any idle world as soon as a
// slot (stream) is free and the world's scratch fits in the device-memory
// budget, evicting the scratch of idle worlds (least recently used first)
// when it has to.  Requests of different worlds overlap on the GPU; the
// requests of one world run one after another in submission order.  Results
// are the same rows knn_tick gives: every request runs the same kernels.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "knn.h"
#include "knn_internal.h"

using knnq::World;

namespace {

using Clock = std::chrono::steady_clock;

enum : int32_t { kQueued = 0, kRunning = 1, kDone = 2, kFailed = 3 };

struct Request {
    int32_t world = 0;
    knn_tick_args args{};
    Clock::time_point t_submit, t_done;
    int32_t state = kQueued;
    int slot = -1;
};

struct ServerWorld {
    knn_world_s h;              // the world (resident part always allocated)
    std::deque<int64_t> queue;  // its requests, oldest first
    bool busy = false;
    uint64_t last_used = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    int64_t request = -1;
};

knn_status bad(knn_status st, const char *msg) {
    knnq::set_last_error(msg);
    return st;
}

}  // namespace

struct knn_server_s {
    int device = 0;
    int64_t budget = 0;  // bytes of tick scratch the server may hold (0: no limit)
    int64_t used = 0;
    int64_t evictions = 0, admitted = 0, completed = 0;
    uint64_t clock = 0;
    std::vector<ServerWorld *> worlds;
    std::unordered_map<int64_t, Request> requests;
    int64_t next_id = 0;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_done, cv_work;
    std::thread thread;
    bool stop = false;
    bool failed = false;

    // Make world w's scratch resident (evicting idle worlds if needed).
    bool ensure_scratch(ServerWorld &sw, cudaStream_t s) {
        World &w = sw.h.w;
        if (w.arena) return true;
        const int64_t need = (int64_t)w.arena_bytes;
        if (budget > 0) {
            while (used + need > budget) {
                ServerWorld *victim = nullptr;
                for (ServerWorld *o : worlds)
                    if (o->h.w.arena && !o->busy &&
                        (!victim || o->last_used < victim->last_used))
                        victim = o;
                if (!victim) return false;  // everything resident is running
                World &v = victim->h.w;
                cudaFreeAsync(v.arena, v.last_stream);
                v.arena = nullptr;
                used -= (int64_t)v.arena_bytes;
                ++evictions;
            }
        }
        void *p = nullptr;
        if (cudaMallocAsync(&p, (size_t)need, s) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        w.arena_async = true;
        knnq::world_attach_scratch(w, p, s);
        used += need;
        return true;
    }

    void loop() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        while (!stop) {
            bool progress = false;
            // completions
            for (Slot &sl : slots) {
                if (sl.request < 0) continue;
                const cudaError_t q = cudaEventQuery(sl.done);
                if (q == cudaErrorNotReady) continue;
                Request &r = requests[sl.request];
                r.t_done = Clock::now();
                r.state = q == cudaSuccess ? kDone : kFailed;
                if (q != cudaSuccess) failed = true;
                ServerWorld &sw = *worlds[r.world];
                sw.busy = false;
                sw.queue.pop_front();
                sl.request = -1;
                ++completed;
                progress = true;
            }
            if (progress) cv_done.notify_all();
            // admissions: the oldest waiting request of any idle world first
            for (;;) {
                int free_slot = -1;
                for (int i = 0; i < (int)slots.size(); ++i)
                    if (slots[i].request < 0) {
                        free_slot = i;
                        break;
                    }
                if (free_slot < 0) break;
                ServerWorld *pick = nullptr;
                int64_t pick_id = -1;
                for (ServerWorld *sw : worlds) {
                    if (sw->busy || sw->queue.empty()) continue;
                    const int64_t id = sw->queue.front();
                    if (pick_id < 0 || id < pick_id) {
                        pick = sw;
                        pick_id = id;
                    }
                }
                if (!pick) break;
                Slot &sl = slots[free_slot];
                if (!ensure_scratch(*pick, sl.stream)) break;  // wait for memory
                Request &r = requests[pick_id];
                knnq::NvtxRange range("knnq serve tick");
                knnq::tick_launch(pick->h.w, r.args, sl.stream);  // replays a recorded tick
                cudaEventRecord(sl.done, sl.stream);
                sl.request = pick_id;
                r.state = kRunning;
                r.slot = free_slot;
                pick->busy = true;
                pick->last_used = ++clock;
                ++admitted;
                progress = true;
            }
            if (!progress) {
                bool running = false;
                for (const Slot &sl : slots) running |= sl.request >= 0;
                if (running) {
                    lk.unlock();
                    std::this_thread::sleep_for(std::chrono::microseconds(5));
                    lk.lock();
                } else {
                    cv_work.wait_for(lk, std::chrono::milliseconds(5));
                }
            }
        }
    }
};

extern "C" {

knn_status knn_server_create(const knn_server_desc *desc, knn_server *out) {
    if (!desc || !out) return bad(KNN_ERR_INVALID, "knn_server_create: NULL argument");
    if (desc->n_slots < 1 || desc->n_slots > 32)
        return bad(KNN_ERR_INVALID, "knn_server_create: n_slots outside [1, 32]");
    if (desc->hbm_budget_bytes < 0)
        return bad(KNN_ERR_INVALID, "knn_server_create: negative budget");
    knn_server_s *s = new knn_server_s();
    cudaGetDevice(&s->device);
    s->budget = desc->hbm_budget_bytes;
    s->slots.resize(desc->n_slots);
    for (Slot &sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            delete s;
            return bad(KNN_ERR_CUDA, "knn_server_create: stream creation failed");
        }
    }
    knnq::prepare_kernels();
    s->thread = std::thread([s] { s->loop(); });
    *out = s;
    return KNN_OK;
}

knn_status knn_server_add_world(knn_server s, const knn_world_desc *desc, const float *x_dev,
                                const float *y_dev, int64_t n, int32_t *world_index) {
    if (!s || !world_index) return bad(KNN_ERR_INVALID, "knn_server_add_world: NULL argument");
    ServerWorld *sw = new ServerWorld();
    cudaSetDevice(s->device);
    const knn_status st =
        knnq::world_init_resident(sw->h.w, desc, x_dev, y_dev, n, s->slots[0].stream);
    if (st != KNN_OK) {
        if (sw->h.w.arena_res) cudaFree(sw->h.w.arena_res);
        delete sw;
        return st;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->budget > 0 && (int64_t)sw->h.w.arena_bytes > s->budget) {
        cudaFree(sw->h.w.arena_res);
        delete sw;
        return bad(KNN_ERR_ADMISSION,
                   "knn_server_add_world: the world's tick scratch exceeds the memory budget");
    }
    *world_index = (int32_t)s->worlds.size();
    s->worlds.push_back(sw);
    return KNN_OK;
}

knn_status knn_server_submit(knn_server s, int32_t world_index, const knn_tick_args *args,
                             int64_t *request_id) {
    if (!s || !args || !request_id) return bad(KNN_ERR_INVALID, "knn_server_submit: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    if (world_index < 0 || world_index >= (int32_t)s->worlds.size())
        return bad(KNN_ERR_INVALID, "knn_server_submit: no such world");
    ServerWorld &sw = *s->worlds[world_index];
    const knn_status st = knnq::check_tick_args(sw.h.w, *args, "knn_server_submit");
    if (st != KNN_OK) return st;
    const int64_t id = s->next_id++;
    Request &r = s->requests[id];
    r.world = world_index;
    r.args = *args;
    r.t_submit = Clock::now();
    sw.queue.push_back(id);
    *request_id = id;
    s->cv_work.notify_one();
    return KNN_OK;
}

knn_status knn_server_poll(knn_server s, int64_t request_id, int32_t *state, double *latency_ms) {
    if (!s) return bad(KNN_ERR_INVALID, "knn_server_poll: NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->requests.find(request_id);
    if (it == s->requests.end()) return bad(KNN_ERR_INVALID, "knn_server_poll: no such request");
    if (state) *state = it->second.state;
    if (latency_ms)
        *latency_ms = it->second.state >= kDone
                          ? std::chrono::duration<double, std::milli>(it->second.t_done -
                                                                      it->second.t_submit)
                                .count()
                          : -1.0;
    if (it->second.state == kFailed) return bad(KNN_ERR_CUDA, "the request's tick failed");
    return KNN_OK;
}

knn_status knn_server_wait(knn_server s, int64_t request_id, double *latency_ms) {
    if (!s) return bad(KNN_ERR_INVALID, "knn_server_wait: NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->requests.find(request_id);
    if (it == s->requests.end()) return bad(KNN_ERR_INVALID, "knn_server_wait: no such request");
    // element references stay valid while the map grows (iterators do not)
    Request *r = &it->second;
    s->cv_done.wait(lk, [&] { return r->state >= kDone; });
    if (latency_ms)
        *latency_ms =
            std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    if (r->state == kFailed) return bad(KNN_ERR_CUDA, "the request's tick failed");
    return KNN_OK;
}

knn_status knn_server_stats(knn_server s, knn_server_counters *out) {
    if (!s || !out) return bad(KNN_ERR_INVALID, "knn_server_stats: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    out->worlds = (int32_t)s->worlds.size();
    int32_t resident = 0;
    for (ServerWorld *w : s->worlds) resident += w->h.w.arena != nullptr;
    out->resident_worlds = resident;
    out->scratch_bytes = s->used;
    int64_t largest = 0;
    for (ServerWorld *w : s->worlds)
        largest = (int64_t)w->h.w.arena_bytes > largest ? (int64_t)w->h.w.arena_bytes : largest;
    out->largest_world_scratch = largest;
    out->admitted = s->admitted;
    out->completed = s->completed;
    out->evictions = s->evictions;
    int64_t queued = 0;
    for (ServerWorld *w : s->worlds) queued += (int64_t)w->queue.size();
    out->pending = queued;
    return KNN_OK;
}

knn_status knn_server_world_status(knn_server s, int32_t world_index, uint32_t *bits_out) {
    if (!s) return bad(KNN_ERR_INVALID, "knn_server_world_status: NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    if (world_index < 0 || world_index >= (int32_t)s->worlds.size())
        return bad(KNN_ERR_INVALID, "knn_server_world_status: no such world");
    ServerWorld &sw = *s->worlds[world_index];
    s->cv_done.wait(lk, [&] { return sw.queue.empty(); });
    return knn_tick_status(&sw.h, bits_out);
}

knn_status knn_server_destroy(knn_server s) {
    if (!s) return bad(KNN_ERR_INVALID, "knn_server_destroy: NULL server");
    {
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv_done.wait(lk, [&] {
            for (ServerWorld *w : s->worlds)
                if (!w->queue.empty()) return false;
            return true;
        });
        s->stop = true;
        s->cv_work.notify_all();
    }
    s->thread.join();
    cudaSetDevice(s->device);
    cudaDeviceSynchronize();
    for (ServerWorld *w : s->worlds) {
        if (w->h.w.arena) cudaFreeAsync(w->h.w.arena, w->h.w.last_stream);
        if (w->h.w.arena_res) cudaFree(w->h.w.arena_res);
        delete w;
    }
    cudaDeviceSynchronize();
    for (Slot &sl : s->slots) {
        cudaEventDestroy(sl.done);
        cudaStreamDestroy(sl.stream);
    }
    delete s;
    return KNN_OK;
}

}  // extern "C"
