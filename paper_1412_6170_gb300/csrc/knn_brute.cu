// GPU brute force: every query against every object, no index (the paper's
// GPU brute-force comparison, Section 5; the same result definition as the
// indexed path, Def. 1).  An in-house baseline for the index's speedup.
//
// A block of kBruteWarps warps serves 32 queries per warp, one per lane, each
// lane keeping its query's sorted top-k of packed (d^2, id + 1) keys in
// registers.  The objects stream through shared memory in tiles of
// kBruteTile, loaded once per block and read by every warp (broadcast reads);
// a candidate within the lane's k-th distance is pushed on a per-lane
// shared-memory stack and merged kBatch at a time by sorting networks, as in
// the packet expansion kernel.
#include <cmath>
#include <cstdio>

#include "knn.h"
#include "knn_device.cuh"
#include "knn_internal.h"

namespace knnq {
namespace {

constexpr int kBruteWarps = 4;   // 16 KB of objects + 32 KB of stacks: 48 KB per block
constexpr int kBruteTile = 1024;              // objects per shared-memory tile
constexpr int kBruteBuf = 32;                 // candidate slots per lane
constexpr int kBruteFlushAt = kBruteBuf - kBatch;

struct BruteArgs {
    const float *x, *y;
    const int32_t *q_id;
    const float *q_x, *q_y;
    int32_t *out_ids;
    float *out_d2;
    int64_t n, n_q;
    int k;
};

template <int KC>
__global__ void __launch_bounds__(kBruteWarps * 32) k_brute(const BruteArgs g) {
    __shared__ float4 s_obj[kBruteTile];
    __shared__ unsigned long long s_buf[kBruteWarps][kBruteBuf][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long (*buf)[32] = s_buf[wid];
    const int k = g.k;
    const float kInf = __int_as_float(0x7f800000);
    const int64_t groups = (g.n_q + 32 * kBruteWarps - 1) / (32 * kBruteWarps);

    for (int64_t grp = blockIdx.x; grp < groups; grp += gridDim.x) {
        // this lane's query
        const int64_t qi = grp * (32 * kBruteWarps) + threadIdx.x;
        bool active = false;
        float qx = 0.f, qy = 0.f;
        int32_t self = 0;  // id + 1 of the issuer; 0 excludes nothing
        if (qi < g.n_q) {
            const int32_t s = g.q_id[qi];
            if (s >= -1 && s < g.n) {
                if (g.q_x) {
                    qx = g.q_x[qi];
                    qy = g.q_y[qi];
                } else if (s >= 0) {
                    qx = g.x[s];
                    qy = g.y[s];
                }
                active = (g.q_x != nullptr || s >= 0) && isfinite(qx) && isfinite(qy);
                self = s + 1;
            }
        }
        unsigned long long lst[KC];
#pragma unroll
        for (int i = 0; i < KC; ++i) lst[i] = i < KC - k ? 0ull : kPad;
        float thr = active ? kInf : -kInf;  // inactive lanes never buffer anything
        int count = 0;
        auto merge = [&]() {
            const int base = count > kBatch ? count - kBatch : 0;
            unsigned long long b[kBatch];
#pragma unroll
            for (int t = 0; t < kBatch; ++t) b[t] = base + t < count ? buf[base + t][lane] : kPad;
            sort8(b);
            merge_batch<KC>(lst, b);
            count = base;
            thr = fminf(thr, __uint_as_float((uint32_t)(lst[KC - 1] >> 32)));
        };

        for (int64_t t0 = 0; t0 < g.n; t0 += kBruteTile) {
            const int tn = g.n - t0 < kBruteTile ? (int)(g.n - t0) : kBruteTile;
            __syncthreads();  // the block is done with the last tile
            for (int i = threadIdx.x; i < tn; i += kBruteWarps * 32)
                s_obj[i] = make_float4(g.x[t0 + i], g.y[t0 + i],
                                       __int_as_float((int32_t)(t0 + i) + 1), 0.f);
            __syncthreads();
            for (int u0 = 0; u0 < tn; u0 += kBatch) {
                while (__any_sync(kFull, count >= kBruteFlushAt)) merge();
                const int nh = tn - u0 < kBatch ? tn - u0 : kBatch;
                const float th = thr;
                auto test = [&](int u) {
                    const float4 o = s_obj[u0 + u];
                    const float dx = __fsub_rn(qx, o.x);
                    const float dy = __fsub_rn(qy, o.y);
                    const float d = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
                    const int32_t idp1 = __float_as_int(o.z);
                    if (d <= th && idp1 != self) {
                        buf[count][lane] =
                            ((unsigned long long)__float_as_uint(d) << 32) | (uint32_t)idp1;
                        ++count;
                    }
                };
                if (nh == kBatch) {
#pragma unroll
                    for (int u = 0; u < kBatch; ++u) test(u);
                } else {
                    for (int u = 0; u < nh; ++u) test(u);
                }
            }
        }
        while (__any_sync(kFull, count > 0)) merge();

        // the row in caller order (padded with (-1, +inf))
        if (qi < g.n_q) {
            int32_t *oi = g.out_ids + qi * k;
            float *od = g.out_d2 + qi * k;
#pragma unroll
            for (int i = 0; i < KC; ++i) {
                if (i >= KC - k) {
                    const unsigned long long key = active ? lst[i] : kPad;
                    oi[i - (KC - k)] = key_id(key);
                    od[i - (KC - k)] = __uint_as_float((uint32_t)(key >> 32));
                }
            }
        }
    }
}

template <int KC>
void run_brute(const BruteArgs &a, cudaStream_t s) {
    const int64_t groups = (a.n_q + 32 * kBruteWarps - 1) / (32 * kBruteWarps);
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_brute<KC>, kBruteWarps * 32, 0);
    int dev = 0;
    cudaGetDevice(&dev);
    int64_t grid = (int64_t)num_sms(dev) * (per_sm > 0 ? per_sm : 1);
    if (grid > groups) grid = groups;
    if (grid < 1) grid = 1;
    k_brute<KC><<<(unsigned)grid, kBruteWarps * 32, 0, s>>>(a);
}

}  // namespace
}  // namespace knnq

extern "C" knn_status knn_brute_force(const float *x_dev, const float *y_dev, int64_t n,
                                      const int32_t *q_id_dev, const float *q_x_dev,
                                      const float *q_y_dev, int64_t n_q, int32_t k,
                                      int32_t *out_ids_dev, float *out_d2_dev, void *stream) {
    if (n < 0 || n > (1ll << 30) || n_q < 0 || k < 1 || k > knnq::kMaxPacketK) {
        knnq::set_last_error("knn_brute_force: n, n_q or k out of range (k in [1, 64])");
        return KNN_ERR_INVALID;
    }
    if (n_q == 0) return KNN_OK;
    if ((n > 0 && (!x_dev || !y_dev)) || !q_id_dev || !out_ids_dev || !out_d2_dev ||
        (q_x_dev == nullptr) != (q_y_dev == nullptr)) {
        knnq::set_last_error("knn_brute_force: NULL array");
        return KNN_ERR_INVALID;
    }
    knnq::BruteArgs a{x_dev, y_dev, q_id_dev, q_x_dev, q_y_dev, out_ids_dev, out_d2_dev, n, n_q,
                      k};
    cudaStream_t s = (cudaStream_t)stream;
    if (k <= 4) knnq::run_brute<4>(a, s);
    else if (k <= 8) knnq::run_brute<8>(a, s);
    else if (k <= 16) knnq::run_brute<16>(a, s);
    else if (k <= 32) knnq::run_brute<32>(a, s);
    else knnq::run_brute<64>(a, s);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        knnq::set_last_error(cudaGetErrorString(e));
        return KNN_ERR_CUDA;
    }
    return KNN_OK;
}
