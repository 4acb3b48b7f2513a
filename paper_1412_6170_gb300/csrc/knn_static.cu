// knn_query_static: a one-shot k-NN call that allocates nothing.
//
// Some callers cannot call cudaMalloc: latency-critical loops (cudaMalloc and
// cudaFree can synchronize the device and take milliseconds), services whose
// device memory is owned by another allocator or fixed budget, and code that
// must not fail half-way through a request because an allocation did.  For
// them this entry point runs the same per-tick pipeline as knn_tick (without
// updates) with every scratch buffer carved from one file-scope device array
// of kStaticScratchBytes, so the caller provides only inputs and outputs.
//
// The array exists once per GPU that loads the library and stays resident
// until the process exits.  All calls share it and it keeps the last call's
// contents, so calls whose work overlaps on the GPU (different streams, or
// different host threads without ordering) race and corrupt each other.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "knn.h"
#include "knn_device.cuh"
#include "knn_internal.h"

namespace {

constexpr size_t kStaticScratchBytes = size_t(8) << 20;  // 8 MiB per GPU
constexpr int64_t kStaticMaxN = 65536;
constexpr int64_t kStaticMaxQ = 65536;
constexpr int kStaticMaxGridLevel = 8;

static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

// Host-side state per device: the scratch array's device address, looked up
// once with cudaGetSymbolAddress with that device current.  The look-back
// epoch base lives in the scratch too.  Its place moves with n and n_q, so it
// may hold any leftover value; that is harmless because every call clears its
// look-back status words first, and within one call every launch that scans
// uses its own epoch (base + launch index).
struct Slot {
    unsigned char *base = nullptr;
};
Slot g_slots[64];
std::mutex g_mu;

knn_status bad(knn_status st, const char *msg) {
    char buf[256];
    snprintf(buf, sizeof(buf), "knn_query_static: %s", msg);
    knnq::set_last_error(buf);  // reported by knn_last_error()
    return st;
}

size_t up256(size_t v) { return (v + 255) & ~size_t(255); }

struct Cut {
    unsigned char *base;
    size_t off = 0;
    template <class T>
    T *take(size_t count) {
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += up256(sizeof(T) * (count ? count : 1));
        return p;
    }
};

// Scratch layout for n objects and n_q queries (base == nullptr: size only).
size_t cut_scratch(knnq::World &w, unsigned char *base, int64_t n_q) {
    const int64_t n = w.n, R = n > n_q ? n : n_q;
    const int64_t ncell = (1ll << (2 * kStaticMaxGridLevel)) + 2;
    int64_t status = ((R + knnq::kSortTile - 1) / knnq::kSortTile) * 256;
    const int64_t others[] = {(n + knnq::kLeafTile - 1) / knnq::kLeafTile,
                              (n + 1 + knnq::kScanTile - 1) / knnq::kScanTile,
                              (ncell + knnq::kScanTile - 1) / knnq::kScanTile};
    for (int64_t o : others) status = status > o ? status : o;
    Cut c{base};
    w.key[0] = c.take<uint32_t>(R);
    w.key[1] = c.take<uint32_t>(R);
    w.val[0] = c.take<int32_t>(R);
    w.val[1] = c.take<int32_t>(R);
    w.xs = c.take<float>(n);
    w.ys = c.take<float>(n);
    w.sid = c.take<int32_t>(n);
    w.inv = c.take<int32_t>(n);
    w.leaf_cap = n;  // no index reuse here, so no empty leaves
    w.bstart = c.take<int32_t>(n + 1);
    w.bcode = c.take<uint32_t>(n);
    w.blevel = c.take<uint8_t>(n);
    w.baabb = c.take<float4>(n);
    w.brange = c.take<int2>(n);
    w.obj_leaf = c.take<int32_t>(n);
    w.cb = c.take<int32_t>(ncell);
    w.qcnt = c.take<int32_t>(n + 1);
    w.qoff = c.take<int32_t>(n + 2);
    w.qs_x = c.take<float>(n_q);
    w.qs_y = c.take<float>(n_q);
    w.qs_id = c.take<int32_t>(n_q);
    w.qs_orig = c.take<int32_t>(n_q);
    w.qs_key = c.take<uint32_t>(n_q);
    w.qs_leaf = c.take<int32_t>(n_q);
    w.qcs = c.take<int32_t>(ncell);
    w.pk_start = c.take<int32_t>(n_q + n_q / 32 + 2);
    w.pk_len = c.take<int32_t>(n_q + n_q / 32 + 2);
    w.status = c.take<uint64_t>(status);
    w.status_words = (size_t)status;
    w.hist = c.take<uint32_t>(4 * 256);
    w.counters = c.take<uint32_t>(knnq::kNumCounters);
    w.tickinfo = c.take<uint32_t>(4);
    w.scalars = c.take<int32_t>(knnq::kNumScalars);
    w.err = c.take<uint32_t>(4);
    return c.off;
}

// A bounded look-back wait that gave up (error bit kErrTimeout) leaves the
// scans' offsets unreliable.  This call has no world to hold a status, so the
// rows say it instead: every row becomes padding (-1, +inf).
__global__ void k_pad_rows_on_timeout(const uint32_t *err, int32_t *ids, float *d2,
                                      int64_t total) {
    if ((*reinterpret_cast<const volatile uint32_t *>(err) & knnq::kErrTimeout) == 0u) return;
    const float inf = __int_as_float(0x7f800000);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        ids[i] = -1;
        d2[i] = inf;
    }
}

int round_log4(double v) {
    if (v <= 1.0) return 0;
    return (int)std::floor(std::log(v) / std::log(4.0) + 0.5);
}

int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

}  // namespace

extern "C" knn_status knn_query_static(const knn_world_desc *desc, const float *x_dev,
                                       const float *y_dev, int64_t n, const int32_t *q_id_dev,
                                       const float *q_x_dev, const float *q_y_dev, int64_t n_q,
                                       int32_t k, int32_t *out_ids_dev, float *out_d2_dev,
                                       void *stream) {
    knnq::NvtxRange range("knnq query_static");
    if (!desc) return bad(KNN_ERR_INVALID, "NULL desc");
    if (!(desc->side > 0.f) || !std::isfinite(desc->side) || !std::isfinite(desc->x0) ||
        !std::isfinite(desc->y0))
        return bad(KNN_ERR_INVALID, "domain must be finite with side > 0");
    if (desc->max_depth < 0 || desc->max_depth > 16)
        return bad(KNN_ERR_INVALID, "max_depth outside [0, 16]");
    if (desc->leaf_capacity < 0 || desc->leaf_capacity > knnq::kMaxLeafCapacity)
        return bad(KNN_ERR_INVALID, "leaf_capacity outside [0, 4096]");
    if (n < 1 || n > kStaticMaxN)
        return bad(KNN_ERR_INVALID, "n outside [1, 65536] (the static scratch limit)");
    if (n_q < 0 || n_q > kStaticMaxQ)
        return bad(KNN_ERR_INVALID, "n_q outside [0, 65536] (the static scratch limit)");
    if (k < 1 || k > knnq::kMaxK) return bad(KNN_ERR_INVALID, "k outside [1, 512]");
    if (!x_dev || !y_dev) return bad(KNN_ERR_INVALID, "NULL positions");
    if ((q_x_dev == nullptr) != (q_y_dev == nullptr))
        return bad(KNN_ERR_INVALID, "q_x and q_y must both be given or both NULL");
    if (n_q > 0 && (!q_id_dev || !out_ids_dev || !out_d2_dev))
        return bad(KNN_ERR_INVALID, "NULL query or output array with n_q > 0");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return bad(KNN_ERR_CUDA, "cudaGetDevice failed");
    std::lock_guard<std::mutex> lock(g_mu);
    Slot &slot = g_slots[dev];
    if (!slot.base) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return bad(KNN_ERR_CUDA, cudaGetErrorString(e));
        slot.base = static_cast<unsigned char *>(p);
    }

    knnq::World w;  // host-side view; every device pointer lands in the scratch
    w.device = dev;
    w.desc = *desc;
    w.desc.k_max = knnq::kMaxK;
    w.desc.max_queries = n_q;
    w.n = n;
    w.L = desc->max_depth > 0 ? desc->max_depth : knnq::default_max_depth(n);
    w.gmax = w.L < kStaticMaxGridLevel ? w.L : kStaticMaxGridLevel;
    w.scale = (float)(1u << w.L) / desc->side;
    w.tuning.leaf_capacity = desc->leaf_capacity;
    if (cut_scratch(w, nullptr, n_q) > kStaticScratchBytes)
        return bad(KNN_ERR_INVALID, "n and n_q together exceed the 8 MiB static scratch");
    cut_scratch(w, slot.base, n_q);
    // positions are only read (no updates in a one-shot call)
    w.px = const_cast<float *>(x_dev);
    w.py = const_cast<float *>(y_dev);

    knnq::Plan p{};
    p.L = w.L;
    p.passes = (2 * p.L + 7) / 8;
    p.th = w.tuning.leaf_capacity > 0 ? w.tuning.leaf_capacity : knnq::default_leaf_capacity(k);
    const int gmax = p.L < kStaticMaxGridLevel ? p.L : kStaticMaxGridLevel;
    p.G = clampi(round_log4(2.0 * (double)n / (double)p.th), 1, gmax);
    p.Gp = clampi(round_log4((double)(n_q > 0 ? n_q : 1) / (k > 4 ? 12.0 * k : 48.0)), 0, p.G);
    p.wide = k > 32;
    p.by_id = 2 * n_q >= n;

    cudaStream_t s = (cudaStream_t)stream;
    // what must start at zero: error words, device scalars and the look-back
    // status words (their place moves with n and n_q, so they may hold another
    // call's ids or offsets, which could read as a ready status); tile tickets
    // are cleared (and the epoch advanced) by the tick-begin kernel
    cudaMemsetAsync(w.err, 0, sizeof(uint32_t) * 4, s);
    cudaMemsetAsync(w.scalars, 0, sizeof(int32_t) * knnq::kNumScalars, s);
    cudaMemsetAsync(w.status, 0, sizeof(uint64_t) * w.status_words, s);
    knnq::launch_tick_begin(w, p, s);
    knnq::launch_object_sort(w, p, s);
    knnq::launch_leaves(w, p, s);
    if (n_q > 0) {
        if (q_x_dev == nullptr)
            knnq::launch_queries_at_issuers(w, p, q_id_dev, n_q, k, out_ids_dev, out_d2_dev, s);
        else
            knnq::launch_queries_explicit(w, p, q_id_dev, q_x_dev, q_y_dev, n_q, k, out_ids_dev,
                                          out_d2_dev, s);
        if (p.wide) {
            knnq::launch_expand_wide(w, p, k, n_q, out_ids_dev, out_d2_dev, nullptr, s);
        } else {
            knnq::launch_packets(w, p, n_q, s);
            knnq::launch_expand(w, p, k, n_q, out_ids_dev, out_d2_dev, nullptr, s);
        }
        k_pad_rows_on_timeout<<<64, 256, 0, s>>>(w.err, out_ids_dev, out_d2_dev,
                                                 n_q * (int64_t)k);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bad(KNN_ERR_CUDA, cudaGetErrorString(e));
    return KNN_OK;
}
