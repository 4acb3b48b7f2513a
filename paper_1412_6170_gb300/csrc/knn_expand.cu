// a7 + a8 -- per-query expansion with top-k, the covered-disc check, and the
// result write in caller order (Sections 4.2.1-4.2.2, Alg. 1, Section 3.3.2).
//
// One warp serves a packet of up to 32 queries that share a level-Gp cell; lane
// i owns query i of the packet and keeps its k best (d^2, id) keys sorted in
// registers.  Objects are read 32 at a time with coalesced loads and broadcast
// to the lanes by warp shuffles, so every lane tests every candidate of the
// packet while each lane keeps its own list and its own k-th distance.
//
// Expansion: (1) scan the leaves holding the packet's queries, widened along
// the Morton leaf order until they hold at least k + 1 objects (the paper's
// first iteration plus its left/right walk); (2) the largest k-th distance of
// the packet bounds a rectangle of level-G cells around the packet; every leaf
// of those cells whose bounding box may still hold a better object for some
// lane is scanned (the paper's "useful" leaves: borders nearer than the current
// farthest result).  Leaves outside the rectangle are farther than every
// lane's k-th distance, so the k-th disc of every query is covered when the
// loop ends and the lists are exact.
#include <cstdio>

#include "knn_device.cuh"
#include "knn_internal.h"

namespace knnq {

struct ExpandArgs {
    const float *xs, *ys;
    const int32_t *sid;
    const int32_t *bstart;
    const uint32_t *bcode;
    const float4 *baabb;
    const int32_t *cb;
    const float *qs_x, *qs_y;
    const int32_t *qs_id, *qs_orig;
    const uint32_t *qs_key;
    const int32_t *pk_start, *pk_len;
    const int32_t *scalars;
    uint32_t *pk_counter;
    int32_t *out_ids;
    float *out_d2;
    float x0, y0, scale_g;
    int L, G, k;
    int64_t n, n_q, pk_cap;
};

// key = (float bits of d^2) << 32 | (id + 1): for d >= 0 the unsigned order of
// keys is the lexicographic (d^2, id) order.  kPad (+inf, 0xFFFFFFFF) is above
// every real key and marks an empty slot; 0 is below every real key.
constexpr unsigned long long kPad = 0x7f800000FFFFFFFFull;

template <int KC>
__device__ __forceinline__ void list_insert(unsigned long long (&a)[KC], unsigned long long key) {
#pragma unroll
    for (int i = KC - 1; i > 0; --i) {
        const unsigned long long prev = a[i - 1];
        const unsigned long long cur = a[i];
        a[i] = key < prev ? prev : (key < cur ? key : cur);
    }
    a[0] = key < a[0] ? key : a[0];
}

template <int KC>
__device__ __forceinline__ void scan_range(const ExpandArgs &g, int32_t s, int32_t e, float qx,
                                           float qy, int32_t qid, bool active,
                                           unsigned long long (&lst)[KC]) {
    const int lane = threadIdx.x & 31;
    for (int32_t base = s; base < e; base += 32) {
        const int32_t cnt = e - base < 32 ? e - base : 32;
        float ox = 0.f, oy = 0.f;
        int32_t oid = 0;
        if (lane < cnt) {
            ox = g.xs[base + lane];
            oy = g.ys[base + lane];
            oid = g.sid[base + lane];
        }
        for (int t = 0; t < cnt; ++t) {
            const float bx = __shfl_sync(kFull, ox, t);
            const float by = __shfl_sync(kFull, oy, t);
            const int32_t bid = __shfl_sync(kFull, oid, t);
            const float dx = __fsub_rn(qx, bx);
            const float dy = __fsub_rn(qy, by);
            const float d = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
            const unsigned long long key =
                ((unsigned long long)__float_as_uint(d) << 32) | (uint32_t)(bid + 1);
            if (active && bid != qid && key < lst[KC - 1]) list_insert<KC>(lst, key);
        }
    }
}

// Leaf of the cell map closest (in Morton order) to a query key: the last leaf
// of the key's level-G cell whose first code is <= key, or the cell's first
// leaf.  Returns the insertion point when the cell has no leaf.
__device__ __forceinline__ int32_t leaf_near(const ExpandArgs &g, uint32_t key) {
    uint32_t c = key >> (2 * (g.L - g.G));
    const uint32_t last = (1u << (2 * g.G)) - 1u;
    c = c < last ? c : last;
    int32_t lo = g.cb[c], hi = g.cb[c + 1];
    if (lo == hi) return lo;
    const int32_t first = lo;
    while (lo < hi) {  // first leaf with code > key
        const int32_t mid = (lo + hi) >> 1;
        if (g.bcode[mid] <= key) lo = mid + 1;
        else hi = mid;
    }
    return lo > first ? lo - 1 : first;
}

__device__ __forceinline__ int cell_g(float v, float v0, float scale, int G) {
    const float t = __fmul_rn(__fsub_rn(v, v0), scale);
    const int lim = 1 << G;
    if (!(t >= 0.0f)) return 0;
    if (t >= (float)lim) return lim - 1;
    return (int)t;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

template <int KC>
__global__ void __launch_bounds__(128) k_expand(const ExpandArgs g) {
    const int lane = threadIdx.x & 31;
    // device scalars are exact unless a look-back timed out; clamp anyway
    int32_t P = g.scalars[kScalarPackets];
    P = P < 0 ? 0 : (P > g.pk_cap ? (int32_t)g.pk_cap : P);
    int32_t m = g.scalars[kScalarLeaves];
    m = m < 0 ? 0 : (m > g.n ? (int32_t)g.n : m);
    const int k = g.k;
    const float kInf = __int_as_float(0x7f800000);

    for (;;) {
        int32_t p = 0;
        if (lane == 0) p = (int32_t)atomicAdd(g.pk_counter, 1u);
        p = __shfl_sync(kFull, p, 0);
        if (p >= P) break;
        const int32_t q0 = g.pk_start[p];
        int32_t ql = g.pk_len[p];
        if (q0 < 0 || ql < 1 || q0 >= g.n_q) continue;
        if (ql > 32) ql = 32;
        if (q0 + ql > g.n_q) ql = (int32_t)(g.n_q - q0);
        const bool has = lane < ql;
        const int32_t j = q0 + (has ? lane : 0);
        const int32_t orig = has ? g.qs_orig[j] : -1;
        const bool active = has && orig >= 0;
        const float qx = active ? g.qs_x[j] : 0.f;
        const float qy = active ? g.qs_y[j] : 0.f;
        const int32_t qid = active ? g.qs_id[j] : -1;
        if (__ballot_sync(kFull, active) == 0u) continue;

        unsigned long long lst[KC];
#pragma unroll
        for (int i = 0; i < KC; ++i) lst[i] = i < KC - k ? 0ull : kPad;

        // (1) leaves of the packet, widened along the leaf order to >= k+1 objects
        int32_t b_lo = leaf_near(g, g.qs_key[q0]);
        int32_t b_hi = leaf_near(g, g.qs_key[q0 + ql - 1]);
        b_hi = b_hi < m ? b_hi + 1 : m;
        if (b_hi < b_lo) b_hi = b_lo;
        {
            bool left = true;
            for (;;) {
                const int32_t cnt = g.bstart[b_hi] - g.bstart[b_lo];
                if (cnt >= k + 1 || (b_lo == 0 && b_hi == m)) break;
                if ((left && b_lo > 0) || b_hi == m) --b_lo;
                else ++b_hi;
                left = !left;
            }
        }
        scan_range<KC>(g, g.bstart[b_lo], g.bstart[b_hi], qx, qy, qid, active, lst);

        // (2) rectangle of cells that can hold a better object for some lane
        if (!(b_lo == 0 && b_hi == m)) {
            const float bx0 = warp_min(active ? qx : kInf), bx1 = warp_max(active ? qx : -kInf);
            const float by0 = warp_min(active ? qy : kInf), by1 = warp_max(active ? qy : -kInf);
            int cx0 = 0, cx1 = 0, cy0 = 0, cy1 = 0;
            auto bound = [&](bool first) {
                float kd = lst[KC - 1] == kPad ? kInf : __uint_as_float((uint32_t)(lst[KC - 1] >> 32));
                const float R2 = warp_max(active ? kd : 0.f);
                const int lim = (1 << g.G) - 1;
                if (!(R2 < kInf)) {
                    cx0 = 0; cx1 = lim; cy1 = lim;
                    if (first) cy0 = 0;
                    return;
                }
                // |q - p| per axis is at most sqrt(R2) (1 + 2^-22) for any object
                // that can enter a list; round the box outward.
                const float R = __fmul_ru(__fsqrt_ru(R2), 1.0000010f);
                cx0 = cell_g(__fsub_rd(bx0, R), g.x0, g.scale_g, g.G);
                cx1 = cell_g(__fadd_ru(bx1, R), g.x0, g.scale_g, g.G);
                cy1 = cell_g(__fadd_ru(by1, R), g.y0, g.scale_g, g.G);
                if (first) cy0 = cell_g(__fsub_rd(by0, R), g.y0, g.scale_g, g.G);
            };
            bound(true);
            for (int cy = cy0; cy <= cy1; ++cy) {
                for (int cx = cx0; cx <= cx1; ++cx) {
                    const uint32_t c = interleave((uint32_t)cx, (uint32_t)cy);
                    const int32_t lo = g.cb[c], hi = g.cb[c + 1];
                    for (int32_t b = lo; b < hi; ++b) {
                        if (b >= b_lo && b < b_hi) continue;
                        const float4 bb = g.baabb[b];
                        float dx = 0.f, dy = 0.f;
                        if (qx < bb.x) dx = __fsub_rn(bb.x, qx);
                        else if (qx > bb.z) dx = __fsub_rn(qx, bb.z);
                        if (qy < bb.y) dy = __fsub_rn(bb.y, qy);
                        else if (qy > bb.w) dy = __fsub_rn(qy, bb.w);
                        const float lb = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
                        const float kd = lst[KC - 1] == kPad
                                             ? kInf
                                             : __uint_as_float((uint32_t)(lst[KC - 1] >> 32));
                        const bool need = active && lb <= kd;
                        if (__any_sync(kFull, need))
                            scan_range<KC>(g, g.bstart[b], g.bstart[b + 1], qx, qy, qid, active,
                                           lst);
                    }
                }
                bound(false);  // the k-th distances only shrink
            }
        }

        // (3) write the row in caller order
        if (active) {
            int32_t *oi = g.out_ids + (int64_t)orig * k;
            float *od = g.out_d2 + (int64_t)orig * k;
#pragma unroll
            for (int i = 0; i < KC; ++i) {
                if (i >= KC - k) {
                    const int r = i - (KC - k);
                    const unsigned long long key = lst[i];
                    if (key == kPad) {
                        oi[r] = -1;
                        od[r] = kInf;
                    } else {
                        oi[r] = (int32_t)((uint32_t)key) - 1;
                        od[r] = __uint_as_float((uint32_t)(key >> 32));
                    }
                }
            }
        }
    }
}

template <int KC>
static void run(const ExpandArgs &a, int device, cudaStream_t s) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_expand<KC>, 128, 0);
    if (per_sm < 1) per_sm = 1;
    k_expand<KC><<<num_sms(device) * per_sm, 128, 0, s>>>(a);
}

void launch_expand(World &w, const Plan &p, int32_t k, int64_t n_q, int32_t *out_ids,
                   float *out_d2, cudaStream_t s) {
    if (n_q <= 0) return;
    ExpandArgs a;
    a.xs = w.xs;
    a.ys = w.ys;
    a.sid = w.sid;
    a.bstart = w.bstart;
    a.bcode = w.bcode;
    a.baabb = w.baabb;
    a.cb = w.cb;
    a.qs_x = w.qs_x;
    a.qs_y = w.qs_y;
    a.qs_id = w.qs_id;
    a.qs_orig = w.qs_orig;
    a.qs_key = w.qs_key;
    a.pk_start = w.pk_start;
    a.pk_len = w.pk_len;
    a.scalars = w.scalars;
    a.pk_counter = w.counters + kCtrExpand;
    a.out_ids = out_ids;
    a.out_d2 = out_d2;
    a.x0 = w.desc.x0;
    a.y0 = w.desc.y0;
    a.scale_g = ldexpf(w.scale, -(p.L - p.G));
    a.L = p.L;
    a.G = p.G;
    a.k = k;
    a.n = w.n;
    a.n_q = n_q;
    a.pk_cap = packet_capacity(w);
    if (k <= 4) run<4>(a, w.device, s);
    else if (k <= 8) run<8>(a, w.device, s);
    else if (k <= 16) run<16>(a, w.device, s);
    else if (k <= 32) run<32>(a, w.device, s);
    else run<64>(a, w.device, s);
    ++w.launches;
}

}  // namespace knnq
