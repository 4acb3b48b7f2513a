// a7 + a8 -- per-query expansion with top-k, the covered-disc check, and the
// result write in caller order (Sections 4.2.1-4.2.2, Alg. 1, Section 3.3.2).
//
// One warp serves a packet of up to 32 queries that share a level-Gp cell; lane
// i owns query i of the packet and keeps its k best (d^2, id) keys sorted in
// registers.  Objects are staged 32 at a time in shared memory with coalesced
// loads and read back by every lane (broadcast reads), so every lane tests
// every candidate of the packet while each lane keeps its own list and its
// own k-th distance.
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
#include <cstring>

#include "knn_device.cuh"
#include "knn_internal.h"

namespace knnq {

struct ExpandArgs {
    const float *xs, *ys;
    const int32_t *sid;
    const int32_t *bstart;
    const uint8_t *blevel;
    const float4 *baabb;
    const int2 *brange;
    const int32_t *cb;
    const float *qs_x, *qs_y;
    const int32_t *qs_id, *qs_orig, *qs_leaf;
    const int32_t *pk_start, *pk_len;
    const int2 *hb;  // non-null: the packets are hb[0 .. scalars[kScalarHandedBack])
    const int32_t *scalars;
    uint32_t *pk_counter;
    int32_t *out_ids;
    float *out_d2;
    float x0, y0, scale_g, side;
    float scale_l;  // level-L scale of the keys
    const uint32_t *bcode;
    int narrow;  // crowded cells: only leaves whose key range meets the packet box
    float spec2;  // alpha^2 of the speculative first threshold (0: none)
    int L, G, k;
    int vec_out;  // rows may be written with 16-byte stores
    const int32_t *q_k;  // per-query list sizes by caller index (NULL: all k)
    uint32_t *err;
    int64_t n, n_q, pk_cap;
    int64_t leaf_cap;  // room for leaves (m <= leaf_cap)
};


// Per-lane candidate buffer (shared memory, a stack of slots per lane):
// candidates whose d^2 is within the lane's current threshold are pushed
// there.  Once some lane's buffer is within kBatch of full, every lane merges
// its newest kBatch into its sorted register list -- one batch, not the whole
// buffer, so that lanes that buffer slowly fill their batches before they are
// merged.
constexpr int kWarps = 4;  // warps per block

// Buffer slots per lane and resident blocks per SM by list size.  Lists of up
// to 8 keys fit in 72 registers, and 24 slots leave room for seven blocks per
// SM instead of five (measured on 1M uniform objects, all querying: the
// expansion runs 11 % faster at k = 8 and 18-19 % faster at k = 1 and 4 than
// with 32 slots); longer lists keep 32 slots and leave the register count to
// the compiler (k = 16 measured alike with six blocks in 80 registers).
template <int KC>
struct Shape {
    static constexpr int kBufCap = KC <= 8 ? 24 : 32;
    static constexpr int kFlushAt = kBufCap - kBatch;
    static constexpr int kMinBlocks = KC <= 8 ? 7 : 0;
};

template <int CAP>
struct WarpSmem {
    float4 obj[32];                              // staged objects (x, y, id bits, -)
    unsigned long long buf[CAP][32];             // [slot][lane]
    float4 lbb[32];                              // gathered leaf box, per lane
    int2 lrg[32];                                // its objects [x, y)
    int2 lc[32];                                 // leaves [x, y) of the lane's cell
};

template <int KC>
struct Lane {
    unsigned long long lst[KC];  // ascending; slots below KC - k hold 0
    float thr;                   // d^2 of the k-th entry (+inf while not full)
    int count;                   // buffered candidates (slots 0 .. count-1)
};

// Merge the newest kBatch buffered candidates (or all, if fewer) into the
// list.  The threshold becomes the list's k-th distance once the list is full
// (it never rises above the threshold the walk started with).
template <int KC, int CAP>
__device__ __forceinline__ void merge_top(Lane<KC> &L, WarpSmem<CAP> &sm, int lane) {
    const int base = L.count > kBatch ? L.count - kBatch : 0;
    unsigned long long b[kBatch];
#pragma unroll
    for (int t = 0; t < kBatch; ++t) b[t] = base + t < L.count ? sm.buf[base + t][lane] : kPad;
    sort8(b);
    merge_batch<KC>(L.lst, b);
    L.count = base;
    L.thr = fminf(L.thr, __uint_as_float((uint32_t)(L.lst[KC - 1] >> 32)));
}

// The leaves of a crowded level-G cell whose key range can meet the box
// [bx0 - R, bx1 + R] x [by0 - R, by1 + R] (binary searches on the leaf codes).
// Every point of the box has a key between the keys of its lower-left and
// upper-right corners (clamped to the cell, rounded outward like the cell
// box), so a leaf whose quadrant meets the box has its first code at most
// the upper key, and is the leaf holding the lower key or a later one.  This
// needs every object inside its leaf's quadrant, which holds for leaves built
// this tick (not for reused ones, whose objects may have moved).  Kept out of
// line: the rare call costs less than the registers it would take inline
// (measured: 3.5 % and 8 % faster on clustered objects at k = 32 and 8,
// uniform objects unchanged).
__device__ __noinline__ int2 narrow_leaves(const ExpandArgs &g, int2 lc, int cx, int cy, float bx0,
                                           float bx1, float by0, float by1, float Rb) {
    const int sh = g.L - g.G;
    const uint32_t ax0 = (uint32_t)cx << sh, ax1 = ax0 + ((1u << sh) - 1u);
    const uint32_t ay0 = (uint32_t)cy << sh, ay1 = ay0 + ((1u << sh) - 1u);
    uint32_t kx0 = cell_coord(__fsub_rd(bx0, Rb), g.x0, g.scale_l, g.L);
    uint32_t kx1 = cell_coord(__fadd_ru(bx1, Rb), g.x0, g.scale_l, g.L);
    uint32_t ky0 = cell_coord(__fsub_rd(by0, Rb), g.y0, g.scale_l, g.L);
    uint32_t ky1 = cell_coord(__fadd_ru(by1, Rb), g.y0, g.scale_l, g.L);
    kx0 = kx0 > ax0 ? kx0 : ax0;
    kx1 = kx1 < ax1 ? kx1 : ax1;
    ky0 = ky0 > ay0 ? ky0 : ay0;
    ky1 = ky1 < ay1 ? ky1 : ay1;
    if (kx0 > kx1 || ky0 > ky1) return make_int2(0, 0);
    const uint32_t zlo = interleave(kx0, ky0), zhi = interleave(kx1, ky1);
    int32_t a0 = lc.x, b0 = lc.y, a1 = lc.x, b1 = lc.y;
    while (a0 < b0 || a1 < b1) {  // first codes > zhi and > zlo
        if (a0 < b0) {
            const int32_t mid = (a0 + b0) >> 1;
            if (g.bcode[mid] <= zhi) a0 = mid + 1; else b0 = mid;
        }
        if (a1 < b1) {
            const int32_t mid = (a1 + b1) >> 1;
            if (g.bcode[mid] <= zlo) a1 = mid + 1; else b1 = mid;
        }
    }
    return make_int2(a1 > lc.x ? a1 - 1 : lc.x, a0);
}

// One packet = one pass of a single loop.  Each iteration (a) merges a batch
// of the buffers if some lane holds kFlushAt candidates, (b) finds the next objects
// to test -- first the packet's own leaves widened to >= k+1 objects (the
// paper's first iteration and left/right walk), then, ring by ring outward from
// the packet, every leaf of the level-G cells that can still hold a better
// object for some lane -- and (c) tests up to kBatch objects against every lane.
// The rings are gathered 32 cells at a time, one per lane: the lanes read the
// cell map and then the leaf records of their cells side by side, a leaf
// whose box is out of reach of the whole packet is dropped at once, and the
// others wait in a ballot mask, tested exactly per lane against the lanes'
// thresholds of the moment they are taken.  Keeping one copy of the scan and
// one of the merge keeps the kernel small.
template <int KC>
__device__ __forceinline__ void expand_packet(const ExpandArgs &g, WarpSmem<Shape<KC>::kBufCap> &sm,
                                              int64_t pi, int32_t m, int lane) {
    constexpr int kFlushAt = Shape<KC>::kFlushAt;
    const int k = g.k;
    const float kInf = __int_as_float(0x7f800000);
    const int lim = (1 << g.G) - 1;
    const int32_t q0 = g.hb ? g.hb[pi].x : g.pk_start[pi];
    int32_t ql = g.hb ? g.hb[pi].y : g.pk_len[pi];
    if (q0 < 0 || ql < 1 || q0 >= g.n_q) return;
    if (ql > 32) ql = 32;
    if (q0 + ql > g.n_q) ql = (int32_t)(g.n_q - q0);
    const bool has = lane < ql;
    const int32_t j = q0 + (has ? lane : 0);
    const int32_t orig = has ? g.qs_orig[j] : -1;
    const bool active = has && orig >= 0;
    const float qx = active ? g.qs_x[j] : 0.f;
    const float qy = active ? g.qs_y[j] : 0.f;
    // id + 1 of the issuer (excluded); 0 matches no object
    const int32_t self = active ? g.qs_id[j] + 1 : 0;
    if (__ballot_sync(kFull, active) == 0u) return;
    // this query's list size (Section 2.1, q = (x, y, k)); 0: no neighbours
    int kq = k;
    if (g.q_k && active) {
        kq = g.q_k[orig];
        if (kq < 0 || kq > k) {
            atomicOr(g.err, kErrBadQuery);
            kq = 0;
        }
    }

    // phase 1: the packet's own leaves, widened along the leaf order
    int32_t b_lo = g.qs_leaf[q0];
    int32_t b_hi = g.qs_leaf[q0 + ql - 1];
    b_lo = b_lo < 0 ? 0 : (b_lo > m ? m : b_lo);
    b_hi = b_hi < 0 ? 0 : (b_hi < m ? b_hi + 1 : m);
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
    const bool all_in_phase1 = b_lo == 0 && b_hi == m;

    // Speculative first threshold: alpha^2 times the area that holds k objects
    // at the density of the packet's own leaves (objects / quadtree area).  A
    // lane that finds fewer than k objects within it is redone below, first
    // within four times that area, then without a threshold.
    float spec = kInf;
    if (g.spec2 > 0.f && !all_in_phase1 && b_hi - b_lo <= 64) {
        float area = 0.f;
        for (int32_t b = b_lo + lane; b < b_hi; b += 32)
            area += ldexpf(1.f, -2 * (int)g.blevel[b]);
        area = warp_sum(area);
        const float cnt1 = (float)(g.bstart[b_hi] - g.bstart[b_lo]);
        spec = g.spec2 * (float)k * area * g.side * g.side / (3.14159265f * cnt1);
    }

    // the same rule for this lane's own list size
    float spec_q = spec;
    if (g.q_k && spec < kInf)
        spec_q = kq > 0 ? spec * ((1.f + 3.f / sqrtf((float)kq) + 2.f / (float)kq) *
                                  (float)kq) / (g.spec2 * (float)k)
                        : -kInf;

    Lane<KC> L;
#pragma unroll
    for (int i = 0; i < KC; ++i) L.lst[i] = i < KC - kq ? 0ull : kPad;
    L.thr = active && kq > 0 ? spec_q : -kInf;  // other lanes never buffer anything
    L.count = 0;

    int32_t cur, end;                     // objects to test
    int32_t staged, staged_end;           // objects held in sm.obj
    int phase;                            // 1: own leaves, 2: rings, 3: draining
    bool flushing = false;                // small lists: a full buffer drains them all
    // phase-2 cursor: number u0 of the next ring cell (see ring_of); the
    // lanes' cells and last gathered leaves sit in sm.lc / sm.lbb / sm.lrg
    // (shared memory keeps them out of the registers the merges need); bit
    // i of pend: lane i's gathered leaf still waits for its exact test
    int u0;
    unsigned pend;
    float bx0 = 0.f, bx1 = 0.f, by0 = 0.f, by1 = 0.f;
    int ccx = 0, ccy = 0, cx0 = 0, cx1 = 0, cy0 = 0, cy1 = 0, rmax = 0;
    float Rb = kInf;
    auto bound = [&]() {
        const float R2 = warp_max(active ? L.thr : 0.f);
        if (!(R2 < kInf)) {
            cx0 = 0; cx1 = lim; cy0 = 0; cy1 = lim;
            Rb = kInf;
        } else {
            // |q - p| per axis is at most sqrt(R2) (1 + 2^-22) for any object
            // that can enter a list; round the box outward.
            const float R = __fmul_ru(__fsqrt_ru(R2), 1.0000010f);
            Rb = R;
            cx0 = cell_g(__fsub_rd(bx0, R), g.x0, g.scale_g, g.G);
            cx1 = cell_g(__fadd_ru(bx1, R), g.x0, g.scale_g, g.G);
            cy0 = cell_g(__fsub_rd(by0, R), g.y0, g.scale_g, g.G);
            cy1 = cell_g(__fadd_ru(by1, R), g.y0, g.scale_g, g.G);
        }
        rmax = max(max(ccx - cx0, cx1 - ccx), max(ccy - cy0, cy1 - ccy));
    };

    for (int attempt = 0;; ++attempt) {
    cur = g.bstart[b_lo];
    end = g.bstart[b_hi];
    staged = -1;
    staged_end = -1;
    phase = 1;
    u0 = 0;
    sm.lc[lane] = make_int2(0, 0);
    pend = 0u;
    for (;;) {
        // (a) merge a batch when a buffer is full, when a list must fill up to
        // bound the box, or when the walk is over (the only merge site)
        const bool drain = phase == 3 || flushing ||
                           (phase == 1 && cur >= end && !all_in_phase1 && !(L.thr < kInf));
        const bool full = __any_sync(kFull, L.count >= kFlushAt);
        if (full || __any_sync(kFull, drain && L.count > 0)) {
            flushing = KC <= 8 && (flushing || full);
            merge_top(L, sm, lane);
            continue;
        }
        flushing = false;
        if (phase == 3) break;
        // (b) next objects
        if (cur >= end) {
            if (phase == 1) {
                if (all_in_phase1) {
                    phase = 3;
                    continue;
                }
                phase = 2;
                bx0 = warp_min(active ? qx : kInf);
                bx1 = warp_max(active ? qx : -kInf);
                by0 = warp_min(active ? qy : kInf);
                by1 = warp_max(active ? qy : -kInf);
                ccx = cell_g(0.5f * (bx0 + bx1), g.x0, g.scale_g, g.G);
                ccy = cell_g(0.5f * (by0 + by1), g.y0, g.scale_g, g.G);
            }
            bool found = false;
            for (;;) {
                if (pend) {  // a gathered leaf: exact test of every lane
                    const int i = __ffs(pend) - 1;
                    pend &= pend - 1u;
                    const float4 ab = sm.lbb[i];
                    const float lb = box_lb(ab.x, ab.y, ab.z, ab.w, qx, qy, qx, qy);
                    if (__any_sync(kFull, lb <= L.thr)) {
                        const int2 rg = sm.lrg[i];
                        cur = rg.x;
                        end = rg.y;
                        found = true;
                        break;
                    }
                    continue;
                }
                int2 lc = sm.lc[lane];
                if (__any_sync(kFull, lc.x < lc.y)) {
                    // next leaf of every lane's cell; the packet's box against
                    // the largest threshold drops what no lane can use
                    const float R2 = warp_max(active ? L.thr : 0.f);
                    bool keep = false;
                    __syncwarp();  // every lane is done with the last gathered boxes
                    if (lc.x < lc.y) {
                        const int32_t b = lc.x++;
                        sm.lc[lane] = lc;
                        if (b < b_lo || b >= b_hi) {
                            const float4 bb = g.baabb[b];
                            const int2 rg = g.brange[b];
                            keep = rg.x < rg.y &&
                                   box_lb(bb.x, bb.y, bb.z, bb.w, bx0, by0, bx1, by1) <= R2;
                            sm.lbb[lane] = bb;
                            sm.lrg[lane] = rg;
                        }
                    }
                    pend = __ballot_sync(kFull, keep);
                    __syncwarp();
                    continue;
                }
                // the next 32 ring cells, one per lane, inside the box that the
                // current thresholds allow (the k-th distances only shrink);
                // done once the next cell's ring lies outside it
                bound();
                if (ring_of(u0) > rmax) break;
                const int u = u0 + lane;
                const int r = ring_of(u);
                lc = make_int2(0, 0);
                if (r <= rmax) {
                    int cx, cy;
                    ring_cell(u, r, ccx, ccy, cx, cy);
                    if (cx >= cx0 && cx <= cx1 && cy >= cy0 && cy <= cy1) {
                        const uint32_t c = interleave((uint32_t)cx, (uint32_t)cy);
                        lc.x = g.cb[c];
                        lc.y = g.cb[c + 1];
                        lc.x = lc.x > 0 ? lc.x : 0;
                        lc.y = lc.y < m ? lc.y : m;
                        if (g.narrow && lc.y - lc.x > 8 && Rb < kInf)
                            lc = narrow_leaves(g, lc, cx, cy, bx0, bx1, by0, by1, Rb);
                    }
                }
                sm.lc[lane] = lc;
                u0 += 32;
            }
            if (!found) {
                phase = 3;
                continue;
            }
        }
        // (c) test up to kBatch objects; stage 32 at a time through shared memory
        if (cur < staged || cur >= staged_end) {
            const int32_t cnt = end - cur < 32 ? end - cur : 32;
            __syncwarp();
            if (lane < cnt && KNN_IN_BOUNDS(cur + lane, 0, g.n, g.err))
                sm.obj[lane] = make_float4(g.xs[cur + lane], g.ys[cur + lane],
                                           __int_as_float(g.sid[cur + lane] + 1), 0.f);
            __syncwarp();
            staged = cur;
            staged_end = cur + cnt;
        }
        const int n_here = staged_end - cur < kBatch ? staged_end - cur : kBatch;
        const float thr = L.thr;
        const int o0 = cur - staged;
        auto test = [&](int u) {
            const float4 o = sm.obj[o0 + u];
            const float dx = __fsub_rn(qx, o.x);
            const float dy = __fsub_rn(qy, o.y);
            const float d = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
            const int32_t idp1 = __float_as_int(o.z);
            if (d <= thr && idp1 != self) {
                sm.buf[L.count][lane] =
                    ((unsigned long long)__float_as_uint(d) << 32) | (uint32_t)idp1;
                ++L.count;
            }
        };
        if (n_here == kBatch) {
#pragma unroll
            for (int u = 0; u < kBatch; ++u) test(u);
        } else {
            for (int u = 0; u < n_here; ++u) test(u);
        }
        cur += n_here;
    }
    // a lane whose speculative threshold held fewer than k objects starts over
    // with four times the threshold, then with none; lanes that are done take
    // no part in the later walks
    if (attempt < 2 && spec < kInf) {
        const bool redo = active && kq > 0 && L.lst[KC - 1] == kPad;
        if (__any_sync(kFull, redo)) {
            if (redo) {
#pragma unroll
                for (int i = 0; i < KC; ++i) L.lst[i] = i < KC - kq ? 0ull : kPad;
                L.thr = attempt == 0 ? 4.f * spec_q : kInf;
            } else {
                L.thr = -kInf;
            }
            continue;
        }
    }
    break;
    }

    // a8: write the rows in caller order
    if constexpr (KC <= 32) {
        // through shared memory, so that neighbouring lanes write
        // neighbouring entries of a row: ids first, then distances
        constexpr int S = KC + 4;  // row stride (words); rows stay 16-byte aligned
        uint32_t *rows = reinterpret_cast<uint32_t *>(&sm.buf[0][0]);
        int32_t *s_orig = reinterpret_cast<int32_t *>(&sm.obj[0]);
        int32_t *s_kq = s_orig + 32;
        __syncwarp();
        s_orig[lane] = active ? orig : -1;
        s_kq[lane] = kq;
        const int vw = g.vec_out ? 4 : 1;
        const int per_row = k / vw;
        const int total = ql * per_row;
        for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
            for (int i = 0; i < KC; i += 4) {
                uint4 v;
                if (pass == 0)
                    v = make_uint4((uint32_t)key_id(L.lst[i]), (uint32_t)key_id(L.lst[i + 1]),
                                   (uint32_t)key_id(L.lst[i + 2]),
                                   (uint32_t)key_id(L.lst[i + 3]));
                else
                    v = make_uint4((uint32_t)(L.lst[i] >> 32), (uint32_t)(L.lst[i + 1] >> 32),
                                   (uint32_t)(L.lst[i + 2] >> 32),
                                   (uint32_t)(L.lst[i + 3] >> 32));
                *reinterpret_cast<uint4 *>(rows + lane * S + i) = v;
            }
            __syncwarp();
            uint32_t *out = pass == 0 ? reinterpret_cast<uint32_t *>(g.out_ids)
                                      : reinterpret_cast<uint32_t *>(g.out_d2);
            for (int base = 0; base < total; base += 32) {
                const int v = base + lane;
                if (v < total) {
                    const int row = v / per_row;
                    const int c = (v - row * per_row) * vw;
                    const int32_t o = s_orig[row];
                    if (o >= 0) {
                        uint32_t *dst = out + (int64_t)o * k + c;
                        if (vw == 4) {  // every row holds k entries
                            *reinterpret_cast<uint4 *>(dst) =
                                *reinterpret_cast<const uint4 *>(rows + row * S + (KC - k) + c);
                        } else {
                            const int kr = s_kq[row];  // entries past it are padding
                            *dst = c < kr ? rows[row * S + (KC - kr) + c]
                                          : (pass == 0 ? 0xFFFFFFFFu : 0x7f800000u);
                        }
                    }
                }
            }
            __syncwarp();
        }
    } else {
        if (active) {
            int32_t *oi = g.out_ids + (int64_t)orig * k;
            float *od = g.out_d2 + (int64_t)orig * k;
#pragma unroll
            for (int i = 0; i < KC; ++i) {
                const int rr = i - (KC - kq);
                if (rr >= 0) {
                    oi[rr] = key_id(L.lst[i]);
                    od[rr] = __uint_as_float((uint32_t)(L.lst[i] >> 32));
                }
            }
            for (int rr = kq; rr < k; ++rr) {  // padding after a shorter list
                oi[rr] = -1;
                od[rr] = kInf;
            }
        }
    }
}

// The packets of a world (device scalars are exact unless a look-back timed
// out; clamp anyway): F full packets at the front of the packet list, P - F
// partial ones at its back, or F = P handed-back packets in hb; m leaves.
__device__ __forceinline__ void walk_counts(const ExpandArgs &g, int32_t &F, int32_t &P,
                                            int32_t &m) {
    F = g.scalars[g.hb ? kScalarHandedBack : kScalarPackets];
    F = F < 0 ? 0 : (F > g.pk_cap ? (int32_t)g.pk_cap : F);
    int32_t Pp = g.hb ? 0 : g.scalars[kScalarPartialPackets];
    Pp = Pp < 0 ? 0 : (Pp > g.pk_cap - F ? (int32_t)(g.pk_cap - F) : Pp);
    P = F + Pp;
    m = g.scalars[kScalarLeaves];
    m = m < 0 ? 0 : (m > g.leaf_cap ? (int32_t)g.leaf_cap : m);
}

// One warp per packet, packets taken from a counter.
template <int KC>
__global__ void __launch_bounds__(kWarps * 32, Shape<KC>::kMinBlocks) k_expand(const ExpandArgs g) {
    __shared__ WarpSmem<Shape<KC>::kBufCap> smem[kWarps];
    const int lane = threadIdx.x & 31;
    WarpSmem<Shape<KC>::kBufCap> &sm = smem[threadIdx.x >> 5];
    int32_t F, P, m;
    walk_counts(g, F, P, m);
    if (P == 0) return;  // (the gathered form finished every packet)
    for (;;) {
        int32_t p = 0;
        if (lane == 0) p = (int32_t)atomicAdd(g.pk_counter, 1u);
        p = __shfl_sync(kFull, p, 0);
        if (p >= P) break;
        const int64_t pi = p < F ? (int64_t)p : g.pk_cap - 1 - (int64_t)(p - F);
        expand_packet<KC>(g, sm, pi, m, lane);
    }
}

// Batched form over many worlds (same list size), as the batched gathered
// form: pfx[w] counts the packets of the worlds before w (their packet lists,
// or the packets the gathered form handed back where hb is set), a warp takes
// global tickets and copies the arguments of the ticket's world into its
// shared memory once per change of world.
struct WalkBatch {
    const ExpandArgs *worlds;
    const long long *pfx;      // n + 1 entries
    unsigned long long *counter;
    int n;
};
static_assert(sizeof(ExpandArgs) % 4 == 0, "copied by 32-bit words");

// (hand-backs are rare: the register count is left to the compiler)
template <int KC>
__global__ void __launch_bounds__(kWarps * 32) k_expand_batch(const WalkBatch b) {
    __shared__ WarpSmem<Shape<KC>::kBufCap> smem[kWarps];
    __shared__ ExpandArgs wargs[kWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    WarpSmem<Shape<KC>::kBufCap> &sm = smem[wid];
    ExpandArgs &ga = wargs[wid];
    const long long total = b.pfx[b.n];
    int cur = 0;
    long long t_lo = 0, t_hi = 0;
    int32_t F = 0, P = 0, m = 0;
    for (;;) {
        long long t = 0;
        if (lane == 0) t = (long long)atomicAdd(b.counter, 1ull);
        t = __shfl_sync(kFull, t, 0);
        if (t >= total) break;
        if (t < t_lo || t >= t_hi) {
            int lo = t < t_lo ? 0 : cur, hi = b.n - 1;  // the last w with pfx[w] <= t
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (b.pfx[mid] <= t) lo = mid;
                else hi = mid - 1;
            }
            cur = lo;
            t_lo = b.pfx[cur];
            t_hi = b.pfx[cur + 1];
            __syncwarp();
            const uint32_t *src = reinterpret_cast<const uint32_t *>(b.worlds + cur);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&ga);
            for (int i = lane; i < (int)(sizeof(ExpandArgs) / 4); i += 32) dst[i] = src[i];
            __syncwarp();
            walk_counts(ga, F, P, m);
        }
        const long long pw = t - t_lo;
        if (pw >= P) continue;
        const int64_t pi = pw < F ? (int64_t)pw : ga.pk_cap - 1 - (int64_t)(pw - F);
        expand_packet<KC>(ga, sm, pi, m, lane);
    }
}

__global__ void __launch_bounds__(1024)
    k_walk_batch_prefix(const ExpandArgs *worlds, int n, long long *pfx,
                        unsigned long long *counter) {
    if (threadIdx.x == 0) *counter = 0ull;
    block_prefix_1024(
        n,
        [&](int i) -> long long {
            int32_t F, P, m;
            walk_counts(worlds[i], F, P, m);
            return P;
        },
        pfx);
}

template <int KC>
static int blocks_per_sm(int device) {
    static int cached[64] = {0};
    const int slot = device >= 0 && device < 64 ? device : 0;
    int per_sm = cached[slot];
    if (per_sm == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_expand<KC>, kWarps * 32, 0);
        if (per_sm < 1) per_sm = 1;
        cached[slot] = per_sm;
    }
    return per_sm;
}

template <int KC>
static int batch_blocks_per_sm(int device) {
    static int cached[64] = {0};
    const int slot = device >= 0 && device < 64 ? device : 0;
    int per_sm = cached[slot];
    if (per_sm == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_expand_batch<KC>, kWarps * 32, 0);
        if (per_sm < 1) per_sm = 1;
        cached[slot] = per_sm;
    }
    return per_sm;
}

void prepare_expand(int device) {
    batch_blocks_per_sm<4>(device);
    batch_blocks_per_sm<8>(device);
    batch_blocks_per_sm<16>(device);
    batch_blocks_per_sm<32>(device);
    batch_blocks_per_sm<64>(device);
    blocks_per_sm<4>(device);
    blocks_per_sm<8>(device);
    blocks_per_sm<16>(device);
    blocks_per_sm<32>(device);
    blocks_per_sm<64>(device);
}

template <int KC>
static void run(const ExpandArgs &a, int device, cudaStream_t s) {
    const int per_sm = blocks_per_sm<KC>(device);
    k_expand<KC><<<num_sms(device) * per_sm, kWarps * 32, 0, s>>>(a);
}

static ExpandArgs expand_args(World &w, const Plan &p, int32_t k, int64_t n_q, int32_t *out_ids,
                              float *out_d2, const int32_t *q_k) {
    ExpandArgs a;
    a.hb = nullptr;
    a.xs = w.xs;
    a.ys = w.ys;
    a.sid = w.sid;
    a.bstart = w.bstart;
    a.baabb = w.baabb;
    a.brange = w.brange;
    a.cb = w.cb;
    a.qs_x = w.qs_x;
    a.qs_y = w.qs_y;
    a.qs_id = w.qs_id;
    a.qs_orig = w.qs_orig;
    a.qs_leaf = w.qs_leaf;
    a.pk_start = w.pk_start;
    a.pk_len = w.pk_len;
    a.scalars = w.scalars;
    a.pk_counter = w.counters + kCtrExpand;
    a.out_ids = out_ids;
    a.out_d2 = out_d2;
    a.x0 = w.desc.x0;
    a.y0 = w.desc.y0;
    a.side = w.desc.side;
    // alpha^2: the disc of the first threshold holds k + 3 sqrt(k) + 2 objects
    // on average, about three standard deviations of a Poisson count above k,
    // so a redo is rare and the first walk stays short for large k
    a.spec2 = 1.0f + 3.0f / sqrtf((float)k) + 2.0f / (float)k;
    a.blevel = w.blevel;
    a.scale_g = ldexpf(w.scale, -(p.L - p.G));
    a.scale_l = w.scale;
    a.bcode = w.bcode;
    a.narrow = p.reuse_age > 0 ? 0 : 1;
    a.L = p.L;
    a.G = p.G;
    a.k = k;
    a.n = w.n;
    a.leaf_cap = w.leaf_cap;
    a.n_q = n_q;
    a.pk_cap = packet_capacity(w);
    a.vec_out = q_k == nullptr && k % 4 == 0 &&
                ((reinterpret_cast<uintptr_t>(out_ids) | reinterpret_cast<uintptr_t>(out_d2)) &
                 15u) == 0;
    a.q_k = q_k;
    a.err = w.err;
    return a;
}

static void run_expand(const ExpandArgs &a, int32_t k, int device, cudaStream_t s) {
    if (k <= 4) run<4>(a, device, s);
    else if (k <= 8) run<8>(a, device, s);
    else if (k <= 16) run<16>(a, device, s);
    else if (k <= 32) run<32>(a, device, s);
    else run<64>(a, device, s);
}

void launch_expand(World &w, const Plan &p, int32_t k, int64_t n_q, int32_t *out_ids,
                   float *out_d2, const int32_t *q_k, cudaStream_t s) {
    if (n_q <= 0) return;
    run_expand(expand_args(w, p, k, n_q, out_ids, out_d2, q_k), k, w.device, s);
    ++w.launches;
}

void launch_expand_handed_back(World &w, const Plan &p, int32_t k, int64_t n_q,
                               int32_t *out_ids, float *out_d2, const int32_t *q_k,
                               cudaStream_t s) {
    if (n_q <= 0) return;
    ExpandArgs a = expand_args(w, p, k, n_q, out_ids, out_d2, q_k);
    a.hb = w.hb;
    a.pk_counter = w.counters + kCtrHandBack;
    run_expand(a, k, w.device, s);
    ++w.launches;
}

// ---------------------------------------------------------------------------
// Batched walk over the packets (or the handed-back packets) of many worlds

size_t walk_batch_entry_bytes() { return sizeof(ExpandArgs); }

void walk_batch_entry(World &w, const Plan &p, const knn_tick_args &t, bool handed_back,
                      void *dst) {
    ExpandArgs a = expand_args(w, p, t.k, t.n_q, t.out_ids_dev, t.out_d2_dev, t.q_k_dev);
    a.hb = handed_back ? w.hb : nullptr;
    a.pk_counter = nullptr;  // tickets come from the batch
    std::memcpy(dst, &a, sizeof(a));
}

template <int KC>
static void run_walk_batch(const WalkBatch &b, int device, cudaStream_t s) {
    const int per_sm = batch_blocks_per_sm<KC>(device);
    k_expand_batch<KC><<<num_sms(device) * per_sm, kWarps * 32, 0, s>>>(b);
}

void launch_walk_batch(int kc, const void *table, int n, long long *pfx,
                       unsigned long long *counter, int device, cudaStream_t s) {
    if (n <= 0) return;
    const ExpandArgs *worlds = static_cast<const ExpandArgs *>(table);
    k_walk_batch_prefix<<<1, 1024, 0, s>>>(worlds, n, pfx, counter);
    const WalkBatch b{worlds, pfx, counter, n};
    if (kc <= 4) run_walk_batch<4>(b, device, s);
    else if (kc <= 8) run_walk_batch<8>(b, device, s);
    else if (kc <= 16) run_walk_batch<16>(b, device, s);
    else if (kc <= 32) run_walk_batch<32>(b, device, s);
    else run_walk_batch<64>(b, device, s);
}
}  // namespace knnq
