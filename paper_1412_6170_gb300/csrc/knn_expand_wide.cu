// a7 + a8 for large k: one warp per query (Sections 4.2.1-4.2.2, Alg. 1,
// Section 3.3.2; the paper's coalesced-writes variant).
//
// For k beyond a register list (up to kMaxK = 512) a whole warp serves one
// query.  The query's candidates -- objects within its current threshold --
// are appended to a shared-memory buffer of 2 * KW keys, 32 objects per step
// (one per lane, compacted by ballot).  When the buffer cannot take another
// 32 it is cut to the k smallest -- for KW >= 128 by a radix select of the
// k-th smallest d^2 (the keys within it move to the front, unsorted), for
// shorter lists by a sort -- and the k-th d^2 bounds the appends from then
// on.  At the end the buffer is cut the same way if it holds more than KW
// keys, then sorted, and the first k keys are the row, written by the whole
// warp (coalesced).  (Measured on 1M uniform objects: the select halves the
// expansion at k = 256 and 512 and saves 31 % at k = 128; at k <= 64 the
// sort of at most 128 keys is the cheaper cut.)  Sorts of up to 128 keys run
// in registers, four keys per lane with shuffles between lanes (k = 64: 2.99
// -> 2.58 ms per tick, k = 128: 4.68 -> 4.43 ms, against the sort through
// shared memory, which longer sorts keep).
//
// The walk is the packet kernel's, for a single point: the query's level-G
// cell and the rings around it, gathered 32 cells at a time, every leaf whose
// box lies within the threshold scanned.  Like Alg. 1, the threshold comes
// first: alpha^2 times the squared radius that holds k objects at the density
// of the query's own leaves (widened along the leaf order to k + 1 objects);
// a query that finds fewer than k objects within it is redone with four times
// the threshold, then with none.  Every object within the final threshold has
// been appended, so the k smallest keys of the buffer are the exact answer.
#include "knn_device.cuh"
#include "knn_internal.h"

namespace knnq {

struct WideArgs {
    const float *xs, *ys;
    const int32_t *sid;
    const int32_t *bstart;
    const uint8_t *blevel;
    const float4 *baabb;
    const int2 *brange;
    const int32_t *cb;
    const float *qs_x, *qs_y;
    const int32_t *qs_id, *qs_orig, *qs_leaf;
    const int32_t *scalars;
    uint32_t *q_counter;
    int32_t *out_ids;
    float *out_d2;
    float x0, y0, scale_g, side;
    float spec2;  // > 0: start from the speculative threshold (alpha^2 from the query's k)
    int G, k;
    int64_t n, n_q;
    int64_t leaf_cap;  // room for leaves (m <= leaf_cap)
    const int32_t *q_k;  // per-query list sizes by caller index (NULL: all k)
    uint32_t *err;
};

constexpr int kWideWarps = 4;  // warps per block

// Ascending bitonic sort of buf[0, count) by one warp; the tail up to the
// next power of two (at least 32, at most the buffer) is padded with kPad.
__device__ __forceinline__ void warp_sort_keys(unsigned long long *buf, int count, int cap,
                                               int lane) {
    int P = 32;
    while (P < count && P < cap) P <<= 1;
    for (int i = count + lane; i < P; i += 32) buf[i] = kPad;
    __syncwarp();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = lane; i < (P >> 1); i += 32) {
                const int a = 2 * i - (i & (stride - 1));
                const int b = a + stride;
                const unsigned long long x = buf[a], y = buf[b];
                if ((x > y) == ((a & size) == 0)) {
                    buf[a] = y;
                    buf[b] = x;
                }
            }
            __syncwarp();
        }
    }
}

// The same sort in registers for 32 R keys (entries from count on padded with
// kPad): lane i holds the keys i R .. i R + R - 1, a compare-exchange between
// two keys of one lane stays in registers and one between lanes goes through
// a shuffle; no shared-memory round trip per stage.
template <int R>
__device__ __forceinline__ void warp_sort_regs(unsigned long long *buf, int count, int lane) {
    constexpr int P = 32 * R;
    __syncwarp();
    unsigned long long x[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const int e = lane * R + j;
        x[j] = e < count ? buf[e] : kPad;
    }
#pragma unroll
    for (int size = 2; size <= P; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride < R) {
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    const int pj = j ^ stride;
                    if (pj > j) {
                        const bool asc = ((lane * R + j) & size) == 0;
                        const unsigned long long a = x[j], b = x[pj];
                        const bool sw = asc ? b < a : a < b;
                        x[j] = sw ? b : a;
                        x[pj] = sw ? a : b;
                    }
                }
            } else {
                const int ls = stride / R;
                const bool lower = (lane & ls) == 0;
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    const unsigned long long y = __shfl_xor_sync(kFull, x[j], ls);
                    const bool asc = ((lane * R + j) & size) == 0;
                    const bool ylo = y < x[j];
                    x[j] = (lower == asc) == ylo ? y : x[j];
                }
            }
        }
    }
    __syncwarp();  // every lane has read its keys
#pragma unroll
    for (int j = 0; j < R; ++j) buf[lane * R + j] = x[j];
    __syncwarp();
}

// Ascending sort of buf[0, count) (count <= cap): in registers up to 32 RMAX
// keys, else in shared memory.
template <int RMAX>
__device__ __forceinline__ void warp_sort(unsigned long long *buf, int count, int cap, int lane) {
    if (count <= 32) warp_sort_regs<1>(buf, count, lane);
    else if (count <= 64) warp_sort_regs<2>(buf, count, lane);
    else if (RMAX >= 4 && count <= 128) warp_sort_regs<(RMAX >= 4 ? 4 : 1)>(buf, count, lane);
    else if (RMAX >= 8 && count <= 256) warp_sort_regs<(RMAX >= 8 ? 8 : 1)>(buf, count, lane);
    else warp_sort_keys(buf, count, cap, lane);
}

// Moves the keys of buf[0, count) whose d^2 is at most the kq-th smallest d^2
// (kq <= count) to the front, in their old order, and returns their number
// (kq plus the keys tied with the kq-th at that d^2).  The kq-th smallest d^2
// is found by a radix select over its four 8-bit digits (d^2 >= 0, so its
// bits order like the value) with a 256-bin warp histogram in shared memory.
__device__ __forceinline__ int warp_select_front(unsigned long long *buf, int count, int kq,
                                                 uint32_t *hist, int lane) {
    uint32_t prefix = 0, mask = 0;
    int want = kq;  // rank (from 1) of the wanted d^2 among the keys matching prefix
#pragma unroll 1
    for (int shift = 24; shift >= 0; shift -= 8) {
#pragma unroll
        for (int b = 0; b < 8; ++b) hist[lane * 8 + b] = 0u;
        __syncwarp();
        for (int i = lane; i < count; i += 32) {
            const uint32_t d = (uint32_t)(buf[i] >> 32);
            if ((d & mask) == prefix) atomicAdd(&hist[(d >> shift) & 255u], 1u);
        }
        __syncwarp();
        uint32_t h[8], loc = 0;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            h[b] = hist[lane * 8 + b];
            loc += h[b];
        }
        uint32_t inc = loc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += y;
        }
        const uint32_t exc = inc - loc;
        const bool mine = exc < (uint32_t)want && (uint32_t)want <= inc;
        uint32_t bin = 0, before = 0;
        if (mine) {
            uint32_t run = exc;
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                if (run + h[b] >= (uint32_t)want) {
                    bin = (uint32_t)(lane * 8 + b);
                    before = run;
                    break;
                }
                run += h[b];
            }
        }
        const int src = __ffs(__ballot_sync(kFull, mine)) - 1;
        bin = __shfl_sync(kFull, bin, src < 0 ? 0 : src);
        before = __shfl_sync(kFull, before, src < 0 ? 0 : src);
        want -= (int)before;
        prefix |= bin << shift;
        mask |= 255u << shift;
        __syncwarp();
    }
    // keep the keys with d^2 <= prefix, compacted to the front in order
    int out = 0;
    for (int i0 = 0; i0 < count; i0 += 32) {
        const int i = i0 + lane;
        const unsigned long long key = i < count ? buf[i] : kPad;
        const bool keep = i < count && (uint32_t)(key >> 32) <= prefix;
        const unsigned km = __ballot_sync(kFull, keep);
        __syncwarp();
        if (keep) buf[out + __popc(km & ((1u << lane) - 1u))] = key;
        out += __popc(km);
        __syncwarp();
    }
    return out;
}

template <int KW>
__global__ void __launch_bounds__(kWideWarps * 32) k_expand_wide(const WideArgs g) {
    constexpr int B = 2 * KW;  // candidate buffer (keys) per warp
    __shared__ unsigned long long s_buf[kWideWarps][B];
    __shared__ float4 s_bb[kWideWarps][32];  // gathered leaf boxes, one per lane
    __shared__ int2 s_rg[kWideWarps][32];    // and their objects [x, y)
    __shared__ uint32_t s_hist[KW >= 128 ? kWideWarps : 1][256];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long *buf = s_buf[wid];
    // device scalars are exact unless a look-back timed out; clamp anyway
    int32_t nv = g.scalars[kScalarValidQueries];
    nv = nv < 0 ? 0 : (nv > g.n_q ? (int32_t)g.n_q : nv);
    int32_t m = g.scalars[kScalarLeaves];
    m = m < 0 ? 0 : (m > g.leaf_cap ? (int32_t)g.leaf_cap : m);
    const int k = g.k;
    const float kInf = __int_as_float(0x7f800000);
    const int lim = (1 << g.G) - 1;
    const unsigned lt = (1u << lane) - 1u;

    for (;;) {
        int32_t j = 0;
        if (lane == 0) j = (int32_t)atomicAdd(g.q_counter, 1u);
        j = __shfl_sync(kFull, j, 0);
        if (j >= nv) break;
        const int32_t orig = g.qs_orig[j];
        if (orig < 0) continue;
        const float qx = g.qs_x[j], qy = g.qs_y[j];
        const int32_t self = g.qs_id[j] + 1;  // id + 1 of the issuer; 0 matches nothing
        // this query's list size (Section 2.1, q = (x, y, k)); 0: no neighbours
        int kq = k;
        if (g.q_k) {
            kq = g.q_k[orig];
            if (kq < 0 || kq > k) {
                if (lane == 0) atomicOr(g.err, kErrBadQuery);
                kq = 0;
            }
        }
        if (kq == 0) {
            for (int r = lane; r < k; r += 32) {
                g.out_ids[(int64_t)orig * k + r] = -1;
                g.out_d2[(int64_t)orig * k + r] = kInf;
            }
            continue;
        }

        // the query's own leaves, widened along the leaf order to >= k + 1 objects
        int32_t b_lo = g.qs_leaf[j];
        b_lo = b_lo < 0 ? 0 : (b_lo >= m ? (m > 0 ? m - 1 : 0) : b_lo);
        int32_t b_hi = b_lo < m ? b_lo + 1 : m;
        {
            bool left = true;
            for (;;) {
                const int32_t cnt = g.bstart[b_hi] - g.bstart[b_lo];
                if (cnt >= kq + 1 || (b_lo == 0 && b_hi == m)) break;
                if ((left && b_lo > 0) || b_hi == m) --b_lo;
                else ++b_hi;
                left = !left;
            }
        }
        float spec = kInf;
        if (g.spec2 > 0.f && !(b_lo == 0 && b_hi == m)) {
            float area = 0.f;
            for (int32_t b = b_lo + lane; b < b_hi; b += 32)
                area += ldexpf(1.f, -2 * (int)g.blevel[b]);
            area = warp_sum(area);
            const float cnt1 = (float)(g.bstart[b_hi] - g.bstart[b_lo]);
            const float a2 = 1.f + 3.f / sqrtf((float)kq) + 2.f / (float)kq;
            spec = a2 * (float)kq * area * g.side * g.side / (3.14159265f * cnt1);
        }
        const int ccx = cell_g(qx, g.x0, g.scale_g, g.G);
        const int ccy = cell_g(qy, g.y0, g.scale_g, g.G);

        int count = 0;
        for (int attempt = 0;; ++attempt) {
            float thr = attempt == 0 ? spec : (attempt == 1 ? 4.f * spec : kInf);
            count = 0;
            for (int u0 = 0;;) {
                // the box of cells that can hold an object within thr
                int cx0 = 0, cx1 = lim, cy0 = 0, cy1 = lim;
                if (thr < kInf) {
                    const float R = __fmul_ru(__fsqrt_ru(thr), 1.0000010f);
                    cx0 = cell_g(__fsub_rd(qx, R), g.x0, g.scale_g, g.G);
                    cx1 = cell_g(__fadd_ru(qx, R), g.x0, g.scale_g, g.G);
                    cy0 = cell_g(__fsub_rd(qy, R), g.y0, g.scale_g, g.G);
                    cy1 = cell_g(__fadd_ru(qy, R), g.y0, g.scale_g, g.G);
                }
                const int rmax = max(max(ccx - cx0, cx1 - ccx), max(ccy - cy0, cy1 - ccy));
                if (ring_of(u0) > rmax) break;
                // the next 32 ring cells, one per lane
                int2 lc = make_int2(0, 0);
                {
                    const int u = u0 + lane;
                    const int r = ring_of(u);
                    if (r <= rmax) {
                        int cx, cy;
                        ring_cell(u, r, ccx, ccy, cx, cy);
                        if (cx >= cx0 && cx <= cx1 && cy >= cy0 && cy <= cy1) {
                            const uint32_t c = interleave((uint32_t)cx, (uint32_t)cy);
                            lc.x = g.cb[c];
                            lc.y = g.cb[c + 1];
                            lc.x = lc.x > 0 ? lc.x : 0;
                            lc.y = lc.y < m ? lc.y : m;
                        }
                    }
                }
                u0 += 32;
                // one leaf of every lane's cell per round
                while (__any_sync(kFull, lc.x < lc.y)) {
                    bool keep = false;
                    __syncwarp();  // every lane is done with the last gathered leaves
                    if (lc.x < lc.y) {
                        const int32_t b = lc.x++;
                        const float4 bb = g.baabb[b];
                        const int2 rg = g.brange[b];
                        keep = rg.x < rg.y && box_lb(bb.x, bb.y, bb.z, bb.w, qx, qy, qx, qy) <= thr;
                        s_bb[wid][lane] = bb;
                        s_rg[wid][lane] = rg;
                    }
                    unsigned pend = __ballot_sync(kFull, keep);
                    __syncwarp();
                    while (pend) {
                        const int i = __ffs(pend) - 1;
                        pend &= pend - 1u;
                        const float4 bb = s_bb[wid][i];
                        // the threshold may have dropped since the leaf was gathered
                        if (!(box_lb(bb.x, bb.y, bb.z, bb.w, qx, qy, qx, qy) <= thr)) continue;
                        const int2 rg = s_rg[wid][i];
                        for (int32_t s0 = rg.x; s0 < rg.y; s0 += 32) {
                            const int32_t o = s0 + lane;
                            float d = kInf;
                            uint32_t idp1 = 0u;
                            if (o < rg.y) {
                                const float dx = __fsub_rn(qx, g.xs[o]);
                                const float dy = __fsub_rn(qy, g.ys[o]);
                                d = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
                                idp1 = (uint32_t)(g.sid[o] + 1);
                            }
                            bool pass = o < rg.y && d <= thr && (int32_t)idp1 != self;
                            unsigned pm = __ballot_sync(kFull, pass);
                            if (count + __popc(pm) > B) {
                                // full: keep the keys within the k-th smallest d^2 (a
                                // radix select for long lists, a sort for short ones);
                                // that d^2 bounds the rest
                                const int kept =
                                    KW >= 128 ? warp_select_front(buf, count, kq, s_hist[wid], lane)
                                              : B;
                                if (kept + 32 <= B) {
                                    // the front is unsorted; its largest d^2 is the k-th
                                    float mx = 0.f;
                                    for (int t = lane; t < kept; t += 32)
                                        mx = fmaxf(mx, __uint_as_float((uint32_t)(buf[t] >> 32)));
                                    thr = fminf(thr, warp_max(mx));
                                    count = kept;
                                } else {
                                    warp_sort<(B >= 128 ? 4 : B / 32)>(buf, count, B, lane);
                                    if (count > kq) count = kq;
                                    thr = fminf(thr, __uint_as_float((uint32_t)(buf[kq - 1] >> 32)));
                                }
                                pass = pass && d <= thr;
                                pm = __ballot_sync(kFull, pass);
                            }
                            if (pass)
                                buf[count + __popc(pm & lt)] =
                                    ((unsigned long long)__float_as_uint(d) << 32) | idp1;
                            count += __popc(pm);
                            __syncwarp();
                        }
                    }
                }
            }
            // every object within thr is in the buffer (or was cut for k smaller ones)
            if (count >= kq || !(thr < kInf) || attempt >= 2) break;
        }

        // a8: the row, in caller order, written by the whole warp
        if (KW >= 128 && count > KW)
            count = warp_select_front(buf, count, kq, s_hist[wid], lane);
        warp_sort<(B >= 128 ? 4 : B / 32)>(buf, count, B, lane);
        int32_t *oi = g.out_ids + (int64_t)orig * k;
        float *od = g.out_d2 + (int64_t)orig * k;
        for (int r = lane; r < k; r += 32) {
            const unsigned long long key = r < count && r < kq ? buf[r] : kPad;
            oi[r] = key_id(key);
            od[r] = __uint_as_float((uint32_t)(key >> 32));
        }
        __syncwarp();
    }
}

template <int KW>
static int wide_blocks_per_sm(int device) {
    static int cached[64] = {0};
    const int slot = device >= 0 && device < 64 ? device : 0;
    int per_sm = cached[slot];
    if (per_sm == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_expand_wide<KW>,
                                                      kWideWarps * 32, 0);
        if (per_sm < 1) per_sm = 1;
        cached[slot] = per_sm;
    }
    return per_sm;
}

void prepare_expand_wide(int device) {
    wide_blocks_per_sm<64>(device);
    wide_blocks_per_sm<128>(device);
    wide_blocks_per_sm<256>(device);
    wide_blocks_per_sm<512>(device);
}

template <int KW>
static void run_wide(const WideArgs &a, int device, cudaStream_t s) {
    k_expand_wide<KW><<<num_sms(device) * wide_blocks_per_sm<KW>(device), kWideWarps * 32, 0,
                        s>>>(a);
}

void launch_expand_wide(World &w, const Plan &p, int32_t k, int64_t n_q, int32_t *out_ids,
                        float *out_d2, const int32_t *q_k, cudaStream_t s) {
    if (n_q <= 0) return;
    WideArgs a;
    a.xs = w.xs;
    a.ys = w.ys;
    a.sid = w.sid;
    a.bstart = w.bstart;
    a.blevel = w.blevel;
    a.baabb = w.baabb;
    a.brange = w.brange;
    a.cb = w.cb;
    a.qs_x = w.qs_x;
    a.qs_y = w.qs_y;
    a.qs_id = w.qs_id;
    a.qs_orig = w.qs_orig;
    a.qs_leaf = w.qs_leaf;
    a.scalars = w.scalars;
    a.q_counter = w.counters + kCtrExpand;
    a.out_ids = out_ids;
    a.out_d2 = out_d2;
    a.x0 = w.desc.x0;
    a.y0 = w.desc.y0;
    a.side = w.desc.side;
    a.scale_g = ldexpf(w.scale, -(p.L - p.G));
    // the same first-threshold rule as the packet kernel
    a.spec2 = 1.0f;
    a.G = p.G;
    a.k = k;
    a.n = w.n;
    a.leaf_cap = w.leaf_cap;
    a.q_k = q_k;
    a.err = w.err;
    a.n_q = n_q;
    if (k <= 64) run_wide<64>(a, w.device, s);
    else if (k <= 128) run_wide<128>(a, w.device, s);
    else if (k <= 256) run_wide<256>(a, w.device, s);
    else run_wide<512>(a, w.device, s);
    ++w.launches;
}

}  // namespace knnq
