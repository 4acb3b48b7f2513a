// a7 + a8, gathered form -- per-query expansion with top-k and the
// covered-disc check, and the rows in caller order (Sections 4.2.1-4.2.2,
// Alg. 1, Section 3.3.2).
//
// One warp serves a packet of up to 32 consecutive sorted queries; lane i owns
// query i and keeps its k best (d^2, id) keys sorted in registers.  Instead of
// walking the quadtree leaf by leaf, the warp first fixes how far it has to
// look -- a first threshold per lane, the squared radius that holds about
// k + 3 sqrt(k) + 2 objects at the local density (Alg. 1's dist_k, found from
// the cell map instead of by k-selection) -- and then gathers in one pass the
// paper's "useful" leaves (Section 4.2.2) of that search box: the level-G
// cells the box covers, the leaves of those cells whose bounding box lies
// within reach of the packet, and the objects of those leaves within reach of
// the packet's bounding box, compacted by ballot into a shared-memory list.
// The list is then tested against every lane in a branch-free loop (broadcast
// reads, eight objects per step); candidates within a lane's threshold go to a
// per-lane buffer that is merged eight at a time into the sorted list.
//
// Exactness: every object within a lane's threshold lies in the gathered list,
// because the box, the leaf boxes and the per-object test all bound the
// distance from below with the rounding of the exact distances.  So a lane
// that holds k keys after the pass has its exact k nearest.  A lane that holds
// fewer is redone with a larger threshold (twice at most); a packet that still
// falls short, has no objects near it, or would gather an unbounded box is
// handed to the packet walk (k_expand), which finishes any packet.
#include <cstdio>
#include <cstring>

#include "knn_device.cuh"
#include "knn_internal.h"

namespace knnq {

namespace {

constexpr int kGatherWarps = 4;        // warps per block
constexpr int kObjCap = 128;           // gathered objects held per round (per warp)
constexpr int kMaxBoxCells = 4096;     // a larger search box goes to the packet walk
constexpr int kDensityCells = 64;      // cells counted around a packet for per-lane densities

template <int KC>
struct GatherShape {
    // Buffer slots per lane.  A merge is forced for every lane as soon as one
    // lane's buffer is kBatch short of full, and then every lane merges its
    // newest kBatch (most of them padding when only a few lanes were near
    // full), so a longer buffer means fewer, fuller merges.  Lists of 32 take
    // 56 slots at 3 blocks per SM (4M clustered objects, a quarter querying:
    // 16 merges per packet with 32 slots, expansion 1.53 -> 1.41 ms; 1M
    // uniform, all querying: 0.87 -> 0.84 ms); shorter lists keep 32 slots and
    // 5 blocks per SM (40 or 44 slots at 4 blocks: clustered k = 16 4 %
    // faster, uniform k = 16 0.5 % slower).  Lists of 64 need 36: the row
    // write reuses the buffer for 32 rows of KC + 4 words.
    static constexpr int kCap = KC <= 16 ? 32 : (KC <= 32 ? 56 : 36);
    static constexpr int kFlushAt = kCap - kBatch;
    static constexpr int kMinBlocks = KC <= 16 ? 5 : (KC <= 32 ? 3 : 2);  // 20, 12 or 8 warps per SM
};

struct GatherArgs {
    const float *xs, *ys;
    const int32_t *sid;
    const int32_t *cb;
    const int32_t *bstart;
    const float4 *baabb;
    const int2 *brange;
    const uint8_t *blevel;
    const float *qs_x, *qs_y;
    const int32_t *qs_id, *qs_orig, *qs_leaf;
    const int32_t *pk_start, *pk_len;
    int32_t *scalars;
    uint32_t *pk_counter;
    int2 *hb;  // packets handed to the packet walk
    int32_t *out_ids;
    float *out_d2;
    const int32_t *q_k;
    uint32_t *err;
    float x0, y0, side, scale_g;
    float spec2;
    int G, k;
    int vec_out;
    int64_t n, n_q, pk_cap, leaf_cap;
};

static_assert(sizeof(GatherArgs) % 4 == 0, "copied by 32-bit words");

template <int KC>
struct GatherSmem {
    // gathered objects in pairs: pair p = (x_2p, x_2p+1, y_2p, y_2p+1), ids + 1
    float4 xy[(kObjCap + kBatch) / 2];
    int32_t idp1[kObjCap + kBatch];
    unsigned long long buf[GatherShape<KC>::kCap][32];  // candidate buffer [slot][lane]
    int32_t lseg_start[32];                         // leaves of 32 cells: first flat index of cell s
    int32_t lseg_base[32];                          // and the leaf that index maps to
    int32_t oseg_start[32];                         // objects of 32 leaves, likewise
    int32_t oseg_base[32];
    int32_t orig[32], kq[32];                       // row write
    int32_t ccount[kDensityCells];                  // objects per cell around the packet
};

template <int KC>
struct GLane {
    unsigned long long lst[KC];  // ascending (d^2, id) keys; slots below KC - k hold 0
    float thr;                   // d^2 bound of what may still enter the list
    int count;                   // buffered candidates
};

// Merge the newest kBatch buffered candidates (or all, if fewer) into the list
// (the batch sorted by a network, then the KC smallest of list and batch by a
// bitonic merge, on the full 64-bit (d^2, id) keys); the issuer's own key
// (id + 1 == self) never enters it.
template <int KC>
__device__ __forceinline__ void gmerge(GLane<KC> &L, GatherSmem<KC> &sm, int lane, uint32_t self) {
    const int base = L.count > kBatch ? L.count - kBatch : 0;
    unsigned long long b[kBatch];
#pragma unroll
    for (int t = 0; t < kBatch; ++t) {
        const unsigned long long v = base + t < L.count ? sm.buf[base + t][lane] : kPad;
        b[t] = (uint32_t)v == self ? kPad : v;
    }
    sort8(b);
    merge_batch<KC>(L.lst, b);
    L.count = base;
    L.thr = fminf(L.thr, __uint_as_float((uint32_t)(L.lst[KC - 1] >> 32)));
}

// Float bits mapped to an unsigned key of the same order (for warp min/max by
// one integer reduction), and back.
__device__ __forceinline__ uint32_t ord_key(float x) {
    const uint32_t u = __float_as_uint(x);
    return u ^ ((u >> 31) ? 0xFFFFFFFFu : 0x80000000u);
}
__device__ __forceinline__ float ord_val(uint32_t k) {
    return __uint_as_float(k ^ ((k >> 31) ? 0x80000000u : 0xFFFFFFFFu));
}

// Lower bound of the squared distance from (x, y) to the box [bx0, bx1] x
// [by0, by1], rounded like the exact distances (so it never exceeds the exact
// d^2 from any point of the box).
__device__ __forceinline__ float point_box_lb(float x, float y, float bx0, float bx1, float by0,
                                              float by1) {
    float dx = 0.f, dy = 0.f;
    if (x < bx0) dx = __fsub_rn(bx0, x);
    else if (x > bx1) dx = __fsub_rn(x, bx1);
    if (y < by0) dy = __fsub_rn(by0, y);
    else if (y > by1) dy = __fsub_rn(y, by1);
    return __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
}


// One packet of the world g: the queries pk_start[pi] .. + pk_len[pi] of the
// sorted order, against the world's m leaves.
template <int KC>
__device__ __forceinline__ void gather_packet(const GatherArgs &g, GatherSmem<KC> &sm, int64_t pi,
                                              int32_t m, int lane) {
    constexpr int FLUSH = GatherShape<KC>::kFlushAt;
    const int k = g.k;
    const float kInf = __int_as_float(0x7f800000);
    const int lim = (1 << g.G) - 1;
    const unsigned lanemask_lt = (1u << lane) - 1u;
    const unsigned lanemask_le = lane == 31 ? kFull : (2u << lane) - 1u;
    const int32_t q0 = g.pk_start[pi];
    int32_t ql = g.pk_len[pi];
    if (q0 < 0 || ql < 1 || q0 >= g.n_q) return;
    if (ql > 32) ql = 32;
    if (q0 + ql > g.n_q) ql = (int32_t)(g.n_q - q0);
    const bool has = lane < ql;
    const int32_t j = q0 + (has ? lane : 0);
    const int32_t orig = has ? g.qs_orig[j] : -1;
    const bool active = has && orig >= 0;
    const float qx = active ? g.qs_x[j] : 0.f;
    const float qy = active ? g.qs_y[j] : 0.f;
    const uint32_t self = active ? (uint32_t)(g.qs_id[j] + 1) : 0u;
    if (__ballot_sync(kFull, active) == 0u) return;
    int kq = k;
    if (g.q_k && active) {
        kq = g.q_k[orig];
        if (kq < 0 || kq > k) {
            atomicOr(g.err, kErrBadQuery);
            kq = 0;
        }
    }
    const float bx0 = ord_val(__reduce_min_sync(kFull, active ? ord_key(qx) : 0xFFFFFFFFu));
    const float bx1 = ord_val(__reduce_max_sync(kFull, active ? ord_key(qx) : 0u));
    const float by0 = ord_val(__reduce_min_sync(kFull, active ? ord_key(qy) : 0xFFFFFFFFu));
    const float by1 = ord_val(__reduce_max_sync(kFull, active ? ord_key(qy) : 0u));

    // local density: objects of the level-G cells under the packet's box
    // grown by one cell (the packet's density), then for each lane the
    // 3 x 3 cells around its own query
    float spec = kInf;
    {
        int ax0 = cell_g(bx0, g.x0, g.scale_g, g.G) - 1, ax1 = cell_g(bx1, g.x0, g.scale_g, g.G) + 1;
        int ay0 = cell_g(by0, g.y0, g.scale_g, g.G) - 1, ay1 = cell_g(by1, g.y0, g.scale_g, g.G) + 1;
        ax0 = ax0 < 0 ? 0 : ax0;
        ay0 = ay0 < 0 ? 0 : ay0;
        ax1 = ax1 > lim ? lim : ax1;
        ay1 = ay1 > lim ? lim : ay1;
        const int nx = ax1 - ax0 + 1, ncl = nx * (ay1 - ay0 + 1);
        const bool keep_cells = ncl <= kDensityCells;
        uint32_t cnt = 0;
        if (ncl <= kMaxBoxCells) {
            __syncwarp();
            for (int c = lane; c < ncl; c += 32) {
                const uint32_t mc = interleave((uint32_t)(ax0 + c % nx), (uint32_t)(ay0 + c / nx));
                int32_t la = g.cb[mc], lb = g.cb[mc + 1];
                la = la < 0 ? 0 : (la > m ? m : la);
                lb = lb < la ? la : (lb > m ? m : lb);
                int32_t d = g.bstart[lb] - g.bstart[la];
                d = d > 0 ? d : 0;
                if (keep_cells) sm.ccount[c] = d;
                cnt += (uint32_t)d;
            }
            cnt = warp_sum_u32(cnt);
            __syncwarp();
        }
        const float cs = g.side / (float)(lim + 1);
        if (cnt > 0)
            spec = g.spec2 * (float)k * (float)ncl * cs * cs / (3.14159265f * (float)cnt);
        if (active && cnt > 0) {
            // the 3 x 3 cells around the lane's query: from the kept counts,
            // else from the cell map
            const int gx = cell_g(qx, g.x0, g.scale_g, g.G), gy = cell_g(qy, g.y0, g.scale_g, g.G);
            const int lx = gx - ax0, ly = gy - ay0;
            const int ny = ncl / nx;
            uint32_t lc = 0, own = 0;
            int lcells = 0;
            for (int dy = -1; dy <= 1; ++dy) {
                for (int dx = -1; dx <= 1; ++dx) {
                    uint32_t c;
                    if (keep_cells) {
                        const int xx = lx + dx, yy = ly + dy;
                        if (xx < 0 || xx >= nx || yy < 0 || yy >= ny) continue;
                        c = (uint32_t)sm.ccount[yy * nx + xx];
                    } else {
                        const int xx = gx + dx, yy = gy + dy;
                        if (xx < 0 || xx > lim || yy < 0 || yy > lim) continue;
                        const uint32_t mc = interleave((uint32_t)xx, (uint32_t)yy);
                        int32_t la = g.cb[mc], lb = g.cb[mc + 1];
                        la = la < 0 ? 0 : (la > m ? m : la);
                        lb = lb < la ? la : (lb > m ? m : lb);
                        const int32_t d = g.bstart[lb] - g.bstart[la];
                        c = (uint32_t)(d > 0 ? d : 0);
                    }
                    lc += c;
                    if (dx == 0 && dy == 0) own = c;
                    ++lcells;
                }
            }
            if (lc > 0)
                spec = g.spec2 * (float)k * (float)lcells * cs * cs / (3.14159265f * (float)lc);
            // the lane's own cell four times off the block's mean (density
            // changes within the block, not count noise): the adaptive leaves
            // instead -- the query's leaf, widened along the leaf order to
            // 2k + 2 objects
            if (4u * own * (uint32_t)lcells < lc || own * (uint32_t)lcells > 4u * lc) {
                int32_t b = g.qs_leaf[j];
                b = b < 0 ? 0 : (b >= m ? m - 1 : b);
                if (b >= 0) {
                    int32_t lo = b, hi = b + 1;
                    float area = ldexpf(1.f, -2 * (int)g.blevel[b]);
                    bool left = true;
                    for (int step = 0; step < 16 && g.bstart[hi] - g.bstart[lo] < 2 * k + 2;
                         ++step) {
                        if ((left && lo > 0) || hi >= m) {
                            if (lo == 0) break;
                            --lo;
                            area += ldexpf(1.f, -2 * (int)g.blevel[lo]);
                        } else {
                            area += ldexpf(1.f, -2 * (int)g.blevel[hi]);
                            ++hi;
                        }
                        left = !left;
                    }
                    const int32_t c2 = g.bstart[hi] - g.bstart[lo];
                    if (c2 > 0)
                        spec = g.spec2 * (float)k * area * g.side * g.side /
                               (3.14159265f * (float)c2);
                }
            }
        }
    }
    float spec_q = spec;
    if (g.q_k && spec < kInf)
        spec_q = kq > 0 ? spec * ((1.f + 3.f / sqrtf((float)kq) + 2.f / (float)kq) *
                                  (float)kq) / (g.spec2 * (float)k)
                        : -kInf;

    GLane<KC> Ln;
#pragma unroll
    for (int i = 0; i < KC; ++i) Ln.lst[i] = i < KC - kq ? 0ull : kPad;
    Ln.thr = active && kq > 0 ? spec_q : -kInf;
    Ln.count = 0;
    bool hand_back = __any_sync(kFull, active && !(spec < kInf));
    const int ccx = cell_g(0.5f * (bx0 + bx1), g.x0, g.scale_g, g.G);
    const int ccy = cell_g(0.5f * (by0 + by1), g.y0, g.scale_g, g.G);

    for (int attempt = 0; !hand_back; ++attempt) {
        // One loop with a single merge site, a single test site and a single
        // gather site (the networks are large: one copy of each keeps the
        // instruction cache warm).  The gather walks the level-G cells ring
        // by ring outward from the packet's centre cell (near objects first,
        // so the lists fill and the thresholds tighten early), inside the
        // box that the lanes' current thresholds allow (re-bounded before
        // every step: thresholds only shrink); per 32 cells it flattens
        // their leaves, keeps the leaves whose box is within reach of the
        // packet, flattens their objects and keeps those within reach of
        // the packet's box, compacted into the pair list sm.xy / sm.idp1.
        int u0 = 0;                          // next ring-numbered cell
        int32_t nleaves = 0, l0 = 0;         // leaves of the current 32 cells
        int32_t nobj = 0, o0 = 0;            // objects of the current 32 leaves
        int lbefore = 0, obefore = 0;        // non-empty segments before l0 / o0
        int32_t lseg_at = 0, oseg_at = 0;    // this lane's segment start, if non-empty
        bool lseg_on = false, oseg_on = false;
        int kept = 0, tpos = 0;              // gathered objects, next to test
        bool gdone = false, testing = false, draining = false;
        int cx0 = 0, cx1 = -1, cy0 = 0, cy1 = -1, rmax = -1;
        float R2 = 0.f;
        const unsigned long long qxx = f2pack(qx, qx), qyy = f2pack(qy, qy);
        float *sxy = reinterpret_cast<float *>(sm.xy);
        const ulonglong2 *sxy2 = reinterpret_cast<const ulonglong2 *>(sm.xy);
        for (;;) {
            // (a) merge a batch (the one merge site): a buffer near full; between
            // passes over the list every accepting lane holding a full batch,
            // or the walk over
            const bool accepting = Ln.thr > -kInf;
            if (__any_sync(kFull, Ln.count >= FLUSH) ||
                (!(testing && tpos < kept) && __any_sync(kFull, Ln.count > 0) &&
                 (draining || __all_sync(kFull, !accepting || Ln.count >= kBatch)))) {
                gmerge<KC>(Ln, sm, lane, self);
                continue;
            }
            if (draining) break;
            // (b) test the gathered objects against every lane, eight (four
            // pairs) per step, until a buffer is near full or the list is done
            if (testing) {
                while (tpos < kept) {
                    if (__any_sync(kFull, Ln.count >= FLUSH)) break;  // to the merge site
                    const float thr = Ln.thr;
#pragma unroll
                    for (int t = 0; t < kBatch / 2; ++t) {
                        const ulonglong2 v = sxy2[(tpos >> 1) + t];
                        const int2 id = *reinterpret_cast<const int2 *>(&sm.idp1[tpos + 2 * t]);
                        const unsigned long long dx = f2sub(qxx, v.x);
                        const unsigned long long dy = f2sub(qyy, v.y);
                        const unsigned long long xx = f2mul(dx, dx), yy = f2mul(dy, dy);
                        // the sum in scalar: a packed multiply chained into a packed
                        // add measured one ulp off the separately rounded steps
                        const uint32_t d0 = __float_as_uint(__fadd_rn(
                            __uint_as_float((uint32_t)xx), __uint_as_float((uint32_t)yy)));
                        const uint32_t d1 = __float_as_uint(__fadd_rn(
                            __uint_as_float((uint32_t)(xx >> 32)),
                            __uint_as_float((uint32_t)(yy >> 32))));
                        if (__uint_as_float(d0) <= thr &&
                            KNN_IN_BOUNDS(Ln.count, 0, GatherShape<KC>::kCap, g.err)) {
                            sm.buf[Ln.count][lane] = ((unsigned long long)d0 << 32) | (uint32_t)id.x;
                            ++Ln.count;
                        }
                        if (__uint_as_float(d1) <= thr &&
                            KNN_IN_BOUNDS(Ln.count, 0, GatherShape<KC>::kCap, g.err)) {
                            sm.buf[Ln.count][lane] = ((unsigned long long)d1 << 32) | (uint32_t)id.y;
                            ++Ln.count;
                        }
                    }
                    tpos += kBatch;
                }
                if (tpos < kept) continue;  // a merge first
                testing = false;
                kept = 0;
                tpos = 0;
                __syncwarp();
                if (gdone) draining = true;
                continue;
            }
            // (c) gather until the list is nearly full or the walk is over; the
            // segment of a flattened index comes from one OR-reduction of the
            // segment starts that fall in its 32-index window.  The search box
            // follows the lanes' thresholds as they stand after the last merge.
            R2 = warp_max(Ln.thr > 0.f ? Ln.thr : 0.f);
            {
                const float R = __fmul_ru(__fsqrt_ru(R2), 1.0000010f);
                cx0 = cell_g(__fsub_rd(bx0, R), g.x0, g.scale_g, g.G);
                cx1 = cell_g(__fadd_ru(bx1, R), g.x0, g.scale_g, g.G);
                cy0 = cell_g(__fsub_rd(by0, R), g.y0, g.scale_g, g.G);
                cy1 = cell_g(__fadd_ru(by1, R), g.y0, g.scale_g, g.G);
                rmax = max(max(ccx - cx0, cx1 - ccx), max(ccy - cy0, cy1 - ccy));
            }
            while (!gdone && kept <= kObjCap - 64) {
                if (o0 < nobj) {
                    // 64 objects of the kept leaves (two per lane, both loads in
                    // flight together); those within reach join the list
                    const unsigned win0 = __reduce_or_sync(
                        kFull, oseg_on && oseg_at >= o0 && oseg_at < o0 + 32 ? 1u << (oseg_at - o0) : 0u);
                    const unsigned win1 = __reduce_or_sync(
                        kFull, oseg_on && oseg_at >= o0 + 32 && oseg_at < o0 + 64
                                   ? 1u << (oseg_at - o0 - 32) : 0u);
                    bool keep0 = false, keep1 = false;
                    float x0 = 0.f, y0 = 0.f, x1 = 0.f, y1 = 0.f;
                    int32_t id0 = 0, id1 = 0;
                    const int32_t j0 = o0 + lane, j1 = o0 + 32 + lane;
                    if (j0 < nobj) {
                        const int r = obefore + __popc(win0 & lanemask_le) - 1;
                        int32_t i = sm.oseg_base[r] + (j0 - sm.oseg_start[r]);
                        if (!KNN_IN_BOUNDS(i, 0, g.n, g.err)) i = 0;
                        x0 = g.xs[i];
                        y0 = g.ys[i];
                        id0 = g.sid[i] + 1;
                    }
                    if (j1 < nobj) {
                        const int r = obefore + __popc(win0) + __popc(win1 & lanemask_le) - 1;
                        int32_t i = sm.oseg_base[r] + (j1 - sm.oseg_start[r]);
                        if (!KNN_IN_BOUNDS(i, 0, g.n, g.err)) i = 0;
                        x1 = g.xs[i];
                        y1 = g.ys[i];
                        id1 = g.sid[i] + 1;
                    }
                    if (j0 < nobj) keep0 = point_box_lb(x0, y0, bx0, bx1, by0, by1) <= R2;
                    if (j1 < nobj) keep1 = point_box_lb(x1, y1, bx0, bx1, by0, by1) <= R2;
                    obefore += __popc(win0) + __popc(win1);
                    const unsigned km0 = __ballot_sync(kFull, keep0);
                    const unsigned km1 = __ballot_sync(kFull, keep1);
                    if (keep0 && KNN_IN_BOUNDS(kept + __popc(km0 & lanemask_lt), 0, kObjCap, g.err)) {
                        const int pos = kept + __popc(km0 & lanemask_lt);
                        sxy[4 * (pos >> 1) + (pos & 1)] = x0;
                        sxy[4 * (pos >> 1) + 2 + (pos & 1)] = y0;
                        sm.idp1[pos] = id0;
                    }
                    if (keep1 && KNN_IN_BOUNDS(kept + __popc(km0) + __popc(km1 & lanemask_lt), 0,
                                               kObjCap, g.err)) {
                        const int pos = kept + __popc(km0) + __popc(km1 & lanemask_lt);
                        sxy[4 * (pos >> 1) + (pos & 1)] = x1;
                        sxy[4 * (pos >> 1) + 2 + (pos & 1)] = y1;
                        sm.idp1[pos] = id1;
                    }
                    kept += __popc(km0) + __popc(km1);
                    o0 += 64;
                    continue;
                }
                if (l0 < nleaves) {
                    // 32 leaves of the current cells: those whose box is within
                    // reach give their objects
                    const unsigned win = __reduce_or_sync(
                        kFull, lseg_on && lseg_at >= l0 && lseg_at < l0 + 32 ? 1u << (lseg_at - l0) : 0u);
                    int32_t ostart = 0, no = 0;
                    if (l0 + lane < nleaves) {
                        const int r = lbefore + __popc(win & lanemask_le) - 1;
                        int32_t b = sm.lseg_base[r] + (l0 + lane - sm.lseg_start[r]);
                        if (!KNN_IN_BOUNDS(b, 0, m, g.err)) b = 0;
                        const int2 rg = g.brange[b];
                        if (rg.y > rg.x) {
                            const float4 bb = g.baabb[b];
                            if (box_lb(bb.x, bb.y, bb.z, bb.w, bx0, by0, bx1, by1) <= R2) {
                                ostart = rg.x;
                                no = rg.y - rg.x;
                            }
                        }
                    }
                    lbefore += __popc(win);
                    int32_t ox = no;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int32_t y = __shfl_up_sync(kFull, ox, o);
                        if (lane >= o) ox += y;
                    }
                    oseg_on = no > 0;
                    oseg_at = ox - no;
                    const unsigned nem = __ballot_sync(kFull, oseg_on);
                    __syncwarp();
                    if (oseg_on) {
                        const int r = __popc(nem & lanemask_lt);
                        sm.oseg_start[r] = oseg_at;
                        sm.oseg_base[r] = ostart;
                    }
                    __syncwarp();
                    nobj = __shfl_sync(kFull, ox, 31);
                    o0 = 0;
                    obefore = 0;
                    l0 += 32;
                    continue;
                }
                // the next 32 cells, ring by ring, inside the current box
                if (ring_of(u0) > rmax) {
                    gdone = true;
                    break;
                }
                if ((int64_t)(cx1 - cx0 + 1) * (cy1 - cy0 + 1) > kMaxBoxCells) {
                    hand_back = true;
                    break;
                }
                int32_t la = 0, nl = 0;
                {
                    const int u = u0 + lane;
                    const int r = ring_of(u);
                    if (r <= rmax) {
                        int cx, cy;
                        ring_cell(u, r, ccx, ccy, cx, cy);
                        if (cx >= cx0 && cx <= cx1 && cy >= cy0 && cy <= cy1) {
                            const uint32_t mc = interleave((uint32_t)cx, (uint32_t)cy);
                            la = g.cb[mc];
                            int32_t lb = g.cb[mc + 1];
                            la = la < 0 ? 0 : (la > m ? m : la);
                            lb = lb < la ? la : (lb > m ? m : lb);
                            nl = lb - la;
                        }
                    }
                }
                int32_t lx = nl;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int32_t y = __shfl_up_sync(kFull, lx, o);
                    if (lane >= o) lx += y;
                }
                lseg_on = nl > 0;
                lseg_at = lx - nl;
                const unsigned nem = __ballot_sync(kFull, lseg_on);
                __syncwarp();
                if (lseg_on) {
                    const int r = __popc(nem & lanemask_lt);
                    sm.lseg_start[r] = lseg_at;
                    sm.lseg_base[r] = la;
                }
                __syncwarp();
                nleaves = __shfl_sync(kFull, lx, 31);
                l0 = 0;
                lbefore = 0;
                u0 += 32;
            }
            if (hand_back) break;
            // far-away sentinels after the list: d^2 = +inf, no step needs a mask
            if (lane < kBatch) {
                const int pos = kept + lane;
                sxy[4 * (pos >> 1) + (pos & 1)] = 3.0e38f;
                sxy[4 * (pos >> 1) + 2 + (pos & 1)] = 3.0e38f;
                sm.idp1[pos] = 0;
            }
            __syncwarp();
            testing = true;
        }
        if (hand_back) break;
        // a lane whose threshold held fewer than k objects is redone with a
        // threshold grown by max(4, 2 (k + 1) / (found + 1)) (the disc's
        // expected count then at least doubles past k); the others take no
        // part
        const bool redo = active && kq > 0 && Ln.lst[KC - 1] == kPad;
        if (!__any_sync(kFull, redo)) break;
        if (attempt >= 2) {
            hand_back = true;
            break;
        }
        if (redo) {
            int found = 0;
#pragma unroll
            for (int i = 0; i < KC; ++i) found += (i >= KC - kq && Ln.lst[i] != kPad) ? 1 : 0;
            const float grow = fmaxf(4.f, 2.f * (float)(kq + 1) / (float)(found + 1));
#pragma unroll
            for (int i = 0; i < KC; ++i) Ln.lst[i] = i < KC - kq ? 0ull : kPad;
            spec_q *= grow;
            Ln.thr = spec_q;
        } else {
            Ln.thr = -kInf;
        }
    }
    if (hand_back) {
        if (lane == 0) {
            const int32_t slot = atomicAdd(g.scalars + kScalarHandedBack, 1);
            if (slot < g.pk_cap) g.hb[slot] = make_int2(q0, ql);
        }
        return;
    }

    // a8: the rows in caller order, through shared memory so that
    // neighbouring lanes write neighbouring entries of a row
    {
        constexpr int S = KC + 4;  // row stride (words); rows stay 16-byte aligned
        uint32_t *rows = reinterpret_cast<uint32_t *>(&sm.buf[0][0]);
        __syncwarp();
        sm.orig[lane] = active ? orig : -1;
        sm.kq[lane] = kq;
        const bool full_rows = g.vec_out && k == KC;  // rows of KC entries, 16-byte stores
        const int vw = g.vec_out ? 4 : 1;
        const int per_row = k / vw;
        const int total = ql * per_row;
        for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
            for (int i = 0; i < KC; i += 4) {
                uint4 v;
                if (pass == 0)
                    v = make_uint4((uint32_t)key_id(Ln.lst[i]), (uint32_t)key_id(Ln.lst[i + 1]),
                                   (uint32_t)key_id(Ln.lst[i + 2]),
                                   (uint32_t)key_id(Ln.lst[i + 3]));
                else
                    v = make_uint4((uint32_t)(Ln.lst[i] >> 32), (uint32_t)(Ln.lst[i + 1] >> 32),
                                   (uint32_t)(Ln.lst[i + 2] >> 32),
                                   (uint32_t)(Ln.lst[i + 3] >> 32));
                *reinterpret_cast<uint4 *>(rows + lane * S + i) = v;
            }
            __syncwarp();
            uint32_t *out = pass == 0 ? reinterpret_cast<uint32_t *>(g.out_ids)
                                      : reinterpret_cast<uint32_t *>(g.out_d2);
            if (full_rows) {
                constexpr int PR = KC / 4;  // 16-byte pieces per row
#pragma unroll
                for (int base = 0; base < 32 * PR; base += 32) {
                    const int v = base + lane;
                    const int row = v / PR, c = (v % PR) * 4;
                    const int32_t o = row < ql ? sm.orig[row] : -1;
                    if (o >= 0 && KNN_IN_BOUNDS(o, 0, g.n_q, g.err))
                        *reinterpret_cast<uint4 *>(out + (int64_t)o * KC + c) =
                            *reinterpret_cast<const uint4 *>(rows + row * S + c);
                }
            } else {
                for (int base = 0; base < total; base += 32) {
                    const int v = base + lane;
                    if (v < total) {
                        const int row = v / per_row;
                        const int c = (v - row * per_row) * vw;
                        const int32_t o = sm.orig[row];
                        if (o >= 0 && KNN_IN_BOUNDS(o, 0, g.n_q, g.err)) {
                            uint32_t *dst = out + (int64_t)o * k + c;
                            if (vw == 4) {
                                *reinterpret_cast<uint4 *>(dst) =
                                    *reinterpret_cast<const uint4 *>(rows + row * S + (KC - k) + c);
                            } else {
                                const int kr = sm.kq[row];
                                *dst = c < kr ? rows[row * S + (KC - kr) + c]
                                              : (pass == 0 ? 0xFFFFFFFFu : 0x7f800000u);
                            }
                        }
                    }
                }
            }
            __syncwarp();
        }
    }
}

// The packets of a world (device scalars are exact unless a look-back timed
// out; clamp anyway): F full packets at the front of the packet list, P - F
// partial ones at its back; m leaves.
__device__ __forceinline__ void gather_counts(const GatherArgs &g, int32_t &F, int32_t &P,
                                              int32_t &m) {
    F = g.scalars[kScalarPackets];
    F = F < 0 ? 0 : (F > g.pk_cap ? (int32_t)g.pk_cap : F);
    int32_t Pp = g.scalars[kScalarPartialPackets];
    Pp = Pp < 0 ? 0 : (Pp > g.pk_cap - F ? (int32_t)(g.pk_cap - F) : Pp);
    P = F + Pp;
    m = g.scalars[kScalarLeaves];
    m = m < 0 ? 0 : (m > g.leaf_cap ? (int32_t)g.leaf_cap : m);
}

}  // namespace

template <int KC>
__global__ void __launch_bounds__(kGatherWarps * 32, GatherShape<KC>::kMinBlocks)
    k_expand_gather(const GatherArgs g) {
    __shared__ GatherSmem<KC> smem[kGatherWarps];
    const int lane = threadIdx.x & 31;
    GatherSmem<KC> &sm = smem[threadIdx.x >> 5];
    int32_t F, P, m;
    gather_counts(g, F, P, m);
    if (P == 0) return;  // (the tiled form finished every packet)
    for (;;) {
        int32_t p = 0;
        if (lane == 0) p = (int32_t)atomicAdd(g.pk_counter, 1u);
        p = __shfl_sync(kFull, p, 0);
        if (p >= P) break;
        const int64_t pi = p < F ? (int64_t)p : g.pk_cap - 1 - (int64_t)(p - F);
        gather_packet<KC>(g, sm, pi, m, lane);
    }
}

// Batched form: one grid pulls the packets of many worlds (same list size).
// pfx[w] counts the packets of the worlds before w (k_gather_batch_prefix
// builds it on the device after the worlds' packets are cut); a warp takes
// global tickets, finds the ticket's world (tickets only grow, so the search
// starts at the warp's last world) and copies that world's arguments into its
// shared memory once per change of world.
struct GatherBatch {
    const GatherArgs *worlds;
    const long long *pfx;  // n + 1 entries
    unsigned long long *counter;
    int n;
};

template <int KC>
__global__ void __launch_bounds__(kGatherWarps * 32, GatherShape<KC>::kMinBlocks)
    k_expand_gather_batch(const GatherBatch b) {
    __shared__ GatherSmem<KC> smem[kGatherWarps];
    __shared__ GatherArgs wargs[kGatherWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    GatherSmem<KC> &sm = smem[wid];
    GatherArgs &ga = wargs[wid];
    const long long total = b.pfx[b.n];
    int cur = 0;
    long long t_lo = 0, t_hi = 0;  // tickets of world cur (empty until the first copy)
    int32_t F = 0, P = 0, m = 0;
    for (;;) {
        long long t = 0;
        if (lane == 0) t = (long long)atomicAdd(b.counter, 1ull);
        t = __shfl_sync(kFull, t, 0);
        if (t >= total) break;
        if (t < t_lo || t >= t_hi) {
            // the last world w >= cur with pfx[w] <= t
            int lo = t < t_lo ? 0 : cur, hi = b.n - 1;
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
            for (int i = lane; i < (int)(sizeof(GatherArgs) / 4); i += 32) dst[i] = src[i];
            __syncwarp();
            gather_counts(ga, F, P, m);
        }
        const long long pw = t - t_lo;
        if (pw >= P) continue;  // (the prefix was built from the same counts)
        const int64_t pi = pw < F ? (int64_t)pw : ga.pk_cap - 1 - (int64_t)(pw - F);
        gather_packet<KC>(ga, sm, pi, m, lane);
    }
}

// pfx over the batch's worlds' packet counts; the tickets start again at 0.
__global__ void __launch_bounds__(1024)
    k_gather_batch_prefix(const GatherArgs *worlds, int n, long long *pfx,
                          unsigned long long *counter) {
    if (threadIdx.x == 0) *counter = 0ull;
    block_prefix_1024(
        n,
        [&](int i) -> long long {
            int32_t F, P, m;
            gather_counts(worlds[i], F, P, m);
            return P;
        },
        pfx);
}

namespace {

template <int KC>
int gather_blocks_per_sm(int device) {
    static int cached[64] = {0};
    const int slot = device >= 0 && device < 64 ? device : 0;
    if (cached[slot] == 0) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_expand_gather<KC>,
                                                      kGatherWarps * 32, 0);
        cached[slot] = per_sm < 1 ? 1 : per_sm;
    }
    return cached[slot];
}

template <int KC>
int gather_batch_blocks_per_sm(int device) {
    static int cached[64] = {0};
    const int slot = device >= 0 && device < 64 ? device : 0;
    if (cached[slot] == 0) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_expand_gather_batch<KC>,
                                                      kGatherWarps * 32, 0);
        cached[slot] = per_sm < 1 ? 1 : per_sm;
    }
    return cached[slot];
}

template <int KC>
void run_gather(const GatherArgs &a, int device, cudaStream_t s) {
    const int per_sm = gather_blocks_per_sm<KC>(device);
    k_expand_gather<KC><<<num_sms(device) * per_sm, kGatherWarps * 32, 0, s>>>(a);
}

}  // namespace

void prepare_expand_gather(int device) {
    gather_blocks_per_sm<4>(device);
    gather_blocks_per_sm<8>(device);
    gather_blocks_per_sm<16>(device);
    gather_blocks_per_sm<32>(device);
    gather_blocks_per_sm<64>(device);
    gather_batch_blocks_per_sm<4>(device);
    gather_batch_blocks_per_sm<8>(device);
    gather_batch_blocks_per_sm<16>(device);
    gather_batch_blocks_per_sm<32>(device);
    gather_batch_blocks_per_sm<64>(device);
}

static GatherArgs gather_args(World &w, const Plan &p, int32_t k, int64_t n_q, int32_t *out_ids,
                              float *out_d2, const int32_t *q_k) {
    GatherArgs a;
    a.xs = w.xs;
    a.ys = w.ys;
    a.sid = w.sid;
    a.cb = w.cb;
    a.bstart = w.bstart;
    a.baabb = w.baabb;
    a.brange = w.brange;
    a.blevel = w.blevel;
    a.qs_x = w.qs_x;
    a.qs_y = w.qs_y;
    a.qs_id = w.qs_id;
    a.qs_orig = w.qs_orig;
    a.qs_leaf = w.qs_leaf;
    a.pk_start = w.pk_start;
    a.pk_len = w.pk_len;
    a.scalars = w.scalars;
    a.pk_counter = w.counters + kCtrGather;
    a.hb = w.hb;
    a.out_ids = out_ids;
    a.out_d2 = out_d2;
    a.q_k = q_k;
    a.err = w.err;
    a.x0 = w.desc.x0;
    a.y0 = w.desc.y0;
    a.side = w.desc.side;
    a.scale_g = ldexpf(w.scale, -(p.L - p.G));
    a.spec2 = 1.0f + 3.0f / sqrtf((float)k) + 2.0f / (float)k;
    a.G = p.G;
    a.k = k;
    a.vec_out = q_k == nullptr && k % 4 == 0 &&
                ((reinterpret_cast<uintptr_t>(out_ids) | reinterpret_cast<uintptr_t>(out_d2)) &
                 15u) == 0;
    a.n = w.n;
    a.n_q = n_q;
    a.pk_cap = packet_capacity(w);
    a.leaf_cap = w.leaf_cap;
    return a;
}

void launch_expand_gather(World &w, const Plan &p, int32_t k, int64_t n_q, int32_t *out_ids,
                          float *out_d2, const int32_t *q_k, cudaStream_t s, bool then_walk) {
    if (n_q <= 0) return;
    const GatherArgs a = gather_args(w, p, k, n_q, out_ids, out_d2, q_k);
    if (k <= 4) run_gather<4>(a, w.device, s);
    else if (k <= 8) run_gather<8>(a, w.device, s);
    else if (k <= 16) run_gather<16>(a, w.device, s);
    else if (k <= 32) run_gather<32>(a, w.device, s);
    else run_gather<64>(a, w.device, s);
    ++w.launches;
    // the packets handed back, through the packet walk
    if (then_walk) launch_expand_handed_back(w, p, k, n_q, out_ids, out_d2, q_k, s);
}

// ---------------------------------------------------------------------------
// Batched expansion (many worlds, one grid per list size)

size_t gather_batch_entry_bytes() { return sizeof(GatherArgs); }

void gather_batch_entry(World &w, const Plan &p, const knn_tick_args &t, void *dst) {
    const GatherArgs a = gather_args(w, p, t.k, t.n_q, t.out_ids_dev, t.out_d2_dev, t.q_k_dev);
    std::memcpy(dst, &a, sizeof(a));
}

namespace {
template <int KC>
void run_gather_batch(const GatherBatch &b, int device, cudaStream_t s) {
    const int per_sm = gather_batch_blocks_per_sm<KC>(device);
    k_expand_gather_batch<KC><<<num_sms(device) * per_sm, kGatherWarps * 32, 0, s>>>(b);
}
}  // namespace

void launch_gather_batch(int kc, const void *table, int n, long long *pfx,
                         unsigned long long *counter, int device, cudaStream_t s) {
    if (n <= 0) return;
    const GatherArgs *worlds = static_cast<const GatherArgs *>(table);
    k_gather_batch_prefix<<<1, 1024, 0, s>>>(worlds, n, pfx, counter);
    const GatherBatch b{worlds, pfx, counter, n};
    if (kc <= 4) run_gather_batch<4>(b, device, s);
    else if (kc <= 8) run_gather_batch<8>(b, device, s);
    else if (kc <= 16) run_gather_batch<16>(b, device, s);
    else if (kc <= 32) run_gather_batch<32>(b, device, s);
    else run_gather_batch<64>(b, device, s);
}

}  // namespace knnq
