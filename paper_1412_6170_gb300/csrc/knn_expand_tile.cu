// a7 + a8, tiled form -- per-query expansion with top-k and the covered-disc
// check, and the rows in caller order (Sections 4.2.1-4.2.2, Alg. 1).
//
// A persistent grid of blocks takes tiles by ticket: a tile is one or two
// consecutive level-Gp cells of the sorted queries (queries at their issuers
// only).  The block first stages, once for all of the tile's queries, every
// object of the level-G cells within a margin H of the tile's queries (the
// paper's per-cell shared scan of Alg. 1, with the neighbouring cells' objects
// brought in once per tile instead of once per query): the objects are
// counting-sorted in shared memory into a row-major grid of micro-cells of
// about one object each.  Then the warps take the tile's packets of 32
// queries, and every lane (one query) scans only its own search box, one
// micro-cell row at a time, its own row first and then alternately the rows
// above and below (near objects first), and shrinks the box whenever its
// threshold tightens (Alg. 1's "keep only what is closer than dist_k").  One
// thread loads the next tile's metadata while the packets are scanned.  The
// batched form runs the same per-tile work over the tiles of many worlds.
//
// Selection keys are 32-bit: (code of d^2 << 11) | (staged index + 1), where
// the code is floor(d^2 * 2^21 / t) for the lane's first threshold t, so the
// compare-exchange networks take two integer min/max instructions.  The code
// is monotone in d^2, so the 32-bit order is the (d^2, id) order wherever the
// codes differ.  A lane is exact when the codes of its k keys are distinct
// and the smallest code it dropped is above its k-th: then its keys are the k
// nearest by (d^2, id) and in order.  Equal codes (ties or near-ties of d^2)
// are settled by exact (d^2, id) keys recomputed from the staged positions;
// what that cannot settle (two dropped keys with the k-th code), a lane that
// still holds fewer than k keys after its threshold reached the staged margin,
// and tiles whose margin holds too many objects go to the gathered form as
// packets of up to 32 consecutive queries (the packets k_packets would cut),
// which finishes them exactly.
//
// Exactness of the box: every object within a lane's threshold lies in its
// box (the box bounds round outward), every object of the box is staged, and
// an object outside the staged margin is at least t_fit away (a bound rounded
// like the exact distances), so a lane whose threshold stays below t_fit sees
// every object that can enter its list.
#include <cstdio>
#include <cstring>

#include "knn_device.cuh"
#include "knn_internal.h"

namespace knnq {

namespace {

constexpr int kTileThreads = 256;               // 8 warps; warp w serves packets w, w + 8, ...
constexpr int kTileWarps = kTileThreads / 32;
constexpr int kTileObj = 2047;                  // staged objects (index + 1 fits 11 bits)
constexpr int kTileCells = 1024;                // micro-cells
constexpr int kTileStage = 256;                 // level-G cells staged per tile
constexpr int kTileMaxQ = 4096;                 // a tile with more queries goes to the gathered form
constexpr int kTileMaxCells = 4;                // level-Gp cells per tile
constexpr int kTileSlots = 16;                  // candidate buffer slots per lane
constexpr int kTileFlush = kBatch;              // a merge as soon as one lane holds a batch
constexpr int kTileStep = 4;                    // objects a lane tests per step of its row
static_assert(kTileFlush - 1 + kTileStep <= kTileSlots, "a step never overfills a buffer");
constexpr float kTileAspect = 1.f;              // micro-cell height / width
constexpr uint32_t kPad32 = 0xFFFFFFFFu;        // empty slot (above every real key)
constexpr float kCodeMax = 2097150.f;           // 2^21 - 2: largest distance code

struct TileArgs {
    const float *xs, *ys;
    const int32_t *sid;
    const int32_t *cb;
    const int32_t *bstart;
    const float *qs_x, *qs_y;
    const int32_t *qs_id, *qs_orig;
    const int32_t *qcs;
    int32_t *scalars;
    uint32_t *tile_counter;
    int32_t *pk_start, *pk_len;  // packets passed to the gathered form
    int32_t *out_ids;
    float *out_d2;
    const int32_t *q_k;
    uint32_t *err;
    float x0, y0, side, scale_g;
    int G, Gp, k;
    int tcells;  // level-Gp cells per tile (consecutive in Morton order): 1, 2 or 4
    int vec_out;
    int64_t n, n_q, pk_cap, leaf_cap;
};

// What a tile's staging needs first, loaded by one thread (for the next tile
// while the current one's packets are scanned): the ticket, its query range,
// its object count, and per cell the first query, the query count and the
// packets before it.
struct TileMeta {
    int64_t t;                      // the tile within its world
    int32_t valid;                  // 0: no tile left
    int32_t as;                     // which world-argument slot (batched form)
    int64_t w;                      // its world (batched form)
    int32_t nv, m, T;               // the world's valid queries, leaves, cells per tile
    int32_t qa, qb, cnt;            // sorted queries [qa, qb); objects in its cells
    int32_t cq[kTileMaxCells];      // the tile's cells: first sorted query,
    int32_t cn[kTileMaxCells];      // query count
    int32_t pp[kTileMaxCells + 1];  // and first packet,
    int32_t pf[kTileMaxCells + 1];  // full packets before the cell
    int32_t ppart[kTileMaxCells + 1];  // partial packets before the cell
};

struct TileSmem {
    float2 xy[kTileObj + 1];   // staged objects in micro-cell order
    int32_t id[kTileObj + 1];
    int32_t cs[kTileCells + 1];     // first staged object of each micro-cell (counts while sorting)
    int32_t gofs[kTileStage + 1];   // first staged index of each staged level-G cell
    int32_t goa[kTileStage];        // and its first object in the leaf-ordered store
    uint32_t buf[kTileSlots][kTileThreads];  // candidate keys [slot][thread]
    float red[4][kTileWarps];
    uint32_t scan_tmp[8];
    uint32_t scan_total;
    float hx0, hx1, hy0, hy1;  // the staged margin (a box around the tile's queries)
    float iw, ih;              // micro-cells per unit length
    float rho;                 // the tile's object density
    int nmx, nmy, ngx, ng, gx0, gx1, gy0, gy1, ok, pk_full, pk_part;
    TileMeta meta[2];               // the current tile's and the next one's
    int32_t mi;                     // which meta is the current tile's
    int32_t next_pk;                // next packet to hand to a warp
};

// Passes packet (q0, ql) on to the gathered form: full packets to the front
// of the packet list, partial ones to its back (the order k_packets gives).
__device__ __forceinline__ void pass_on(const TileArgs &g, int32_t q0, int32_t ql) {
    const int64_t slot = ql == 32 ? (int64_t)atomicAdd(g.scalars + kScalarPackets, 1)
                                  : g.pk_cap - 1 - atomicAdd(g.scalars + kScalarPartialPackets, 1);
    if (slot >= 0 && slot < g.pk_cap) {
        g.pk_start[slot] = q0;
        g.pk_len[slot] = ql;
    }
}

// Packet pw of the current tile: the cell's queries 32 at a time (the packets
// k_packets cuts).
__device__ __forceinline__ void tile_pk(const TileMeta &M, int T, int32_t pw, int32_t &q0,
                                        int32_t &ql) {
    int c = 0;
#pragma unroll
    for (int i = 1; i < kTileMaxCells; ++i)
        if (i < T && pw >= M.pp[i]) c = i;
    const int32_t o = pw - M.pp[c];
    q0 = M.cq[c] + 32 * o;
    ql = min(32, M.cn[c] - 32 * o);
}

// Micro-cell coordinate of v in a grid starting at v0 with `inv` cells per
// unit length and n cells: monotone in v (clamped at both ends).
__device__ __forceinline__ int mcell(float v, float v0, float inv, int n) {
    const float t = __fmul_rn(__fsub_rn(v, v0), inv);
    if (!(t >= 0.0f)) return 0;
    if (t >= (float)n) return n - 1;
    return (int)t;
}

__device__ __forceinline__ void cmpx32(uint32_t &x, uint32_t &y) {
    const uint32_t lo = min(x, y);
    y = max(x, y);
    x = lo;
}

// Sort 8 keys ascending (the 19-comparator network of sort8).
__device__ __forceinline__ void sort8_32(uint32_t (&b)[kBatch]) {
    cmpx32(b[0], b[2]); cmpx32(b[1], b[3]); cmpx32(b[4], b[6]); cmpx32(b[5], b[7]);
    cmpx32(b[0], b[4]); cmpx32(b[1], b[5]); cmpx32(b[2], b[6]); cmpx32(b[3], b[7]);
    cmpx32(b[0], b[1]); cmpx32(b[2], b[3]); cmpx32(b[4], b[5]); cmpx32(b[6], b[7]);
    cmpx32(b[2], b[4]); cmpx32(b[3], b[5]);
    cmpx32(b[1], b[4]); cmpx32(b[3], b[6]);
    cmpx32(b[1], b[2]); cmpx32(b[3], b[4]); cmpx32(b[5], b[6]);
}

// a (KC keys, ascending) := the KC smallest of a and b (8 keys, ascending), as
// merge_batch does; d1 <= d2 become the two smallest keys dropped so far.
template <int KC>
__device__ __forceinline__ void merge32(uint32_t (&a)[KC], const uint32_t (&b)[kBatch],
                                        uint32_t &d1, uint32_t &d2) {
    static_assert(KC >= kBatch, "lists of at least one batch");
#pragma unroll
    for (int i = KC - kBatch; i < KC; ++i) {
        const uint32_t v = b[KC - 1 - i];
        const uint32_t h = max(v, a[i]);
        d2 = min(d2, max(d1, h));
        d1 = min(d1, h);
        a[i] = min(v, a[i]);
    }
#pragma unroll
    for (int span = KC / 2; span >= 1; span >>= 1) {
#pragma unroll
        for (int i = 0; i < KC; ++i)
            if ((i & span) == 0) cmpx32(a[i], a[i + span]);
    }
}

// Exact squared distance from the query (packed qx, qy) to a staged object.
__device__ __forceinline__ float tile_d2(unsigned long long qq, float2 v) {
    const unsigned long long o = f2pack(v.x, v.y);
    const unsigned long long dxy = f2sub(qq, o);
    const unsigned long long sq = f2mul(dxy, dxy);
    return __fadd_rn(__uint_as_float((uint32_t)sq), __uint_as_float((uint32_t)(sq >> 32)));
}

// One packet: the sorted queries q0 .. q0 + ql - 1 of the current tile, lane
// i owning query q0 + i.  Returns nothing; rows are written, or the packet is
// passed to the gathered form.
template <int KC>
__device__ __forceinline__ void tile_packet(const TileArgs &g, TileSmem &s, int32_t q0, int32_t ql,
                                            int tid) {
    const int lane = tid & 31;
    const float kInf = __int_as_float(0x7f800000);
    const bool has = lane < ql;
    const int32_t j = q0 + (has ? lane : 0);
    const int32_t orig = has ? g.qs_orig[j] : -1;
    const bool active = has && orig >= 0;
    const float qx = active ? g.qs_x[j] : 0.f;
    const float qy = active ? g.qs_y[j] : 0.f;
    int kq = g.k;
    if (g.q_k && active) {
        kq = g.q_k[orig];
        if (kq < 0 || kq > g.k) {
            atomicOr(g.err, kErrBadQuery);
            kq = 0;
        }
    }
    const bool want = active && kq > 0;
    const float hx0 = s.hx0, hy0 = s.hy0, iw = s.iw, ih = s.ih;
    const int nmx = s.nmx, nmy = s.nmy;
    const int mxq = mcell(qx, hx0, iw, nmx), myq = mcell(qy, hy0, ih, nmy);

    bool fail = false;
    // the issuer's own staged object (its position is the query's, so it sits
    // in the query's micro-cell); its key (code 0) is dropped at the merges
    int selfp = -1;
    if (want) {
        const int32_t me = g.qs_id[j];
        const int c = myq * nmx + mxq;
        const int pe = s.cs[c + 1];
        for (int p = s.cs[c]; p < pe; ++p)
            if (s.id[p] == me) selfp = p;
        if (me >= 0 && selfp < 0) fail = true;
    }
    // first threshold: the squared radius holding about k + 3 sqrt(k) + 2
    // objects at the density of the 7 x 7 micro-cells around the query
    float t0 = kInf;
    if (want) {
        const int xa = max(mxq - 3, 0), xb = min(mxq + 3, nmx - 1);
        const int ya = max(myq - 3, 0), yb = min(myq + 3, nmy - 1);
        int cnt = 0;
        for (int r = ya; r <= yb; ++r) cnt += s.cs[r * nmx + xb + 1] - s.cs[r * nmx + xa];
        const float cells = (float)((xb - xa + 1) * (yb - ya + 1));
        const float rho = cnt > 0 ? (float)cnt * iw * ih / cells : s.rho;
        const float fk = (float)kq;
        t0 = (fk + 3.f * sqrtf(fk) + 2.f) / (3.14159265f * rho);
    }
    // t_fit: an object outside the staged margin is at least this far (in
    // d^2, rounded like the exact distances); the threshold stays below it
    // (a side of the margin whose staged cells reach the edge of the cell map
    // has nothing unstaged beyond it: every object past the world's edge lies
    // in an edge cell)
    float tcap = -1.f;
    if (want) {
        const int lim = (1 << g.G) - 1;
        float gm = kInf;
        if (s.gx0 > 0) gm = fminf(gm, __fsub_rd(qx, s.hx0));
        if (s.gx1 < lim) gm = fminf(gm, __fsub_rd(s.hx1, qx));
        if (s.gy0 > 0) gm = fminf(gm, __fsub_rd(qy, s.hy0));
        if (s.gy1 < lim) gm = fminf(gm, __fsub_rd(s.hy1, qy));
        if (gm == kInf) {
            tcap = 3.0e38f;
        } else if (gm > 0.f) {
            const float tf = __fmul_rd(gm, gm);
            if (tf > 0.f) tcap = __uint_as_float(__float_as_uint(tf) - 1u);
        }
        if (!(tcap > 0.f)) fail = true;
    }
    float thr = fminf(t0, tcap);
    bool ok = !want;
    uint32_t lst[KC];
#pragma unroll
    for (int i = 0; i < KC; ++i) lst[i] = kPad32;
    uint32_t disc = kPad32, disc2 = kPad32;  // the two smallest keys dropped
    const unsigned long long qq = f2pack(qx, qy);
    const uint32_t selfkey = selfp >= 0 ? (uint32_t)(selfp + 1) : 0u;  // 0: no real key

    for (int attempt = 0; attempt < 3; ++attempt) {
        bool run = want && !ok && !fail;
        const float tstart = thr;
        const float tmax = run ? thr : 1.f;
        // codes: floor(d^2 * inv) <= kCodeMax for every d^2 <= tmax; a code c
        // bounds d^2 from above by (c + 1) * rstep (a threshold so small or
        // large that either factor leaves the normal range goes on)
        const float inv = __fmul_rd(kCodeMax, __frcp_rd(tmax));
        const float rstep = __fmul_ru(__frcp_ru(inv), 1.0000002f);
        if (run && !(inv > 1.0e-30f && inv < 1.0e30f && rstep > 1.0e-30f && rstep < 1.0e30f)) {
            fail = true;
            run = false;
        }
        if (!__any_sync(kFull, run)) break;
        if (run) {
#pragma unroll
            for (int i = 0; i < KC; ++i) lst[i] = i < KC - kq ? 0u : kPad32;
            disc = disc2 = kPad32;
        }
        float th = run ? thr : -1.f;
        int mx_lo = 0, mx_hi = -1, my_lo = 0, my_hi = -1, omax = 0;
        auto box = [&]() {
            const float R = __fmul_ru(__fsqrt_ru(th), 1.0000010f);
            mx_lo = mcell(__fsub_rd(qx, R), hx0, iw, nmx);
            mx_hi = mcell(__fadd_ru(qx, R), hx0, iw, nmx);
            my_lo = mcell(__fsub_rd(qy, R), hy0, ih, nmy);
            my_hi = mcell(__fadd_ru(qy, R), hy0, ih, nmy);
            omax = 2 * max(myq - my_lo, my_hi - myq);
        };
        int p = 0, e = 0, o = 0, cnt = 0;
        if (run) {
            box();
            const int b = myq * nmx;
            p = s.cs[b + mx_lo];
            e = s.cs[b + mx_hi + 1];
        }
        for (;;) {
            // the one merge site: the newest batch of every lane
            if (__any_sync(kFull, cnt >= kTileFlush)) {
                const int base = cnt > kBatch ? cnt - kBatch : 0;
                uint32_t bt[kBatch];
#pragma unroll
                for (int t = 0; t < kBatch; ++t) {
                    const uint32_t v = base + t < cnt ? s.buf[base + t][tid] : kPad32;
                    bt[t] = v == selfkey ? kPad32 : v;
                }
                sort8_32(bt);
                merge32<KC>(lst, bt, disc, disc2);
                cnt = base;
                const uint32_t last = lst[KC - 1];
                if (run && last != kPad32) {
                    const float tf = __fmul_ru((float)((last >> 11) + 1u), rstep);
                    if (tf < th) {
                        th = tf;
                        box();
                    }
                }
                continue;
            }
            // next non-empty row of the box: offsets 0, +1, -1, +2, -2, ...
            while (p >= e && o < omax) {
                ++o;
                const int r = myq + ((o & 1) ? ((o + 1) >> 1) : -(o >> 1));
                if (r >= my_lo && r <= my_hi) {
                    const int b = r * nmx;
                    p = s.cs[b + mx_lo];
                    e = s.cs[b + mx_hi + 1];
                }
            }
            if (!__any_sync(kFull, p < e)) break;
#pragma unroll
            for (int u = 0; u < kTileStep; ++u) {
                const int j = p + u;
                const bool okj = j < e;
                const float d = tile_d2(qq, s.xy[okj ? j : 0]);
                if (okj && d <= th) {
                    const uint32_t c = __float2uint_rz(__fmul_rn(d, inv));
                    s.buf[cnt][tid] = (c << 11) | (uint32_t)(j + 1);
                    ++cnt;
                }
            }
            p += kTileStep;
        }
        // drain the buffers
        while (__any_sync(kFull, cnt > 0)) {
            const int base = cnt > kBatch ? cnt - kBatch : 0;
            uint32_t bt[kBatch];
#pragma unroll
            for (int t = 0; t < kBatch; ++t) {
                const uint32_t v = base + t < cnt ? s.buf[base + t][tid] : kPad32;
                bt[t] = v == selfkey ? kPad32 : v;
            }
            sort8_32(bt);
            merge32<KC>(lst, bt, disc, disc2);
            cnt = base;
        }
        if (run) {
            if (lst[KC - 1] != kPad32) {
                ok = true;
            } else if (tstart < tcap) {
                // fewer than k objects within the threshold: grow it (the disc's
                // expected count at least doubles past k), up to the margin
                int found = 0;
#pragma unroll
                for (int i = 0; i < KC; ++i) found += (i >= KC - kq && lst[i] != kPad32) ? 1 : 0;
                const float grow = fmaxf(4.f, 2.f * (float)(kq + 1) / (float)(found + 1));
                thr = fminf(__fmul_ru(tstart, grow), tcap);
            } else {
                fail = true;
            }
        }
    }
    if (want && !ok) fail = true;
    // Codes that are equal among the k keys, or between the k-th and a dropped
    // key, leave the order open: those keys are compared by their exact
    // (d^2, id) keys (bubble passes within runs of equal codes, and the one
    // dropped key with the k-th code against the k-th).  Two dropped keys with
    // the k-th code, or runs too long for the passes, go on.
    bool fix = false;
    if (want && ok) {
        const uint32_t ck = lst[KC - 1] >> 11;
        fix = (disc >> 11) == ck;
#pragma unroll
        for (int i = 0; i + 1 < KC; ++i)
            if (i >= KC - kq) fix = fix || (lst[i] >> 11) == (lst[i + 1] >> 11);
        if ((disc2 >> 11) == ck) fail = true;
    }
    if (__any_sync(kFull, fix && !fail)) {
        auto exact = [&](uint32_t key) -> unsigned long long {
            int x = (int)(key & 0x7FFu) - 1;
            if (!KNN_IN_BOUNDS(x, 0, kTileObj, g.err)) x = 0;
            const float d = tile_d2(qq, s.xy[x]);
            return ((unsigned long long)__float_as_uint(d) << 32) | (uint32_t)(s.id[x] + 1);
        };
        auto order_runs = [&](bool &sorted) {
            sorted = true;
#pragma unroll
            for (int i = 0; i + 1 < KC; ++i) {
                if (i >= KC - kq && (lst[i] >> 11) == (lst[i + 1] >> 11) &&
                    exact(lst[i]) > exact(lst[i + 1])) {
                    const uint32_t t = lst[i];
                    lst[i] = lst[i + 1];
                    lst[i + 1] = t;
                    sorted = false;
                }
            }
        };
        if (fix && !fail) {
            bool sorted = false;
            for (int pass = 0; pass < 4 && !sorted; ++pass) order_runs(sorted);
            if ((disc >> 11) == (lst[KC - 1] >> 11) && exact(disc) < exact(lst[KC - 1])) {
                lst[KC - 1] = disc;
                sorted = false;
                for (int pass = 0; pass < 4 && !sorted; ++pass) order_runs(sorted);
            }
            if (!sorted) fail = true;
        }
    }
    if (__any_sync(kFull, fail)) {
        if (lane == 0) pass_on(g, q0, ql);
        return;
    }
    // a8: the row of this lane's query in caller order
    if (!active || !KNN_IN_BOUNDS(orig, 0, g.n_q, g.err)) return;
    const int k = g.k;
    int32_t *orow = g.out_ids + (int64_t)orig * k;
    float *drow = g.out_d2 + (int64_t)orig * k;
    if (g.vec_out && k == KC && kq == KC) {
#pragma unroll
        for (int i = 0; i < KC; i += 4) {
            int32_t idv[4];
            float dv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                int x = (int)(lst[i + u] & 0x7FFu) - 1;
                if (!KNN_IN_BOUNDS(x, 0, kTileObj, g.err)) x = 0;
                idv[u] = s.id[x];
                dv[u] = tile_d2(qq, s.xy[x]);
            }
            *reinterpret_cast<int4 *>(orow + i) = make_int4(idv[0], idv[1], idv[2], idv[3]);
            *reinterpret_cast<float4 *>(drow + i) = make_float4(dv[0], dv[1], dv[2], dv[3]);
        }
    } else {
#pragma unroll
        for (int sl = 0; sl < KC; ++sl) {
            const int i = sl - (KC - kq);
            if (i >= 0) {
                int x = (int)(lst[sl] & 0x7FFu) - 1;
                if (!KNN_IN_BOUNDS(x, 0, kTileObj, g.err)) x = 0;
                orow[i] = s.id[x];
                drow[i] = tile_d2(qq, s.xy[x]);
            }
        }
        for (int i = kq; i < k; ++i) {
            orow[i] = -1;
            drow[i] = kInf;
        }
    }
}

__device__ __forceinline__ int32_t clamp_leaf(int32_t b, int32_t m) {
    return b < 0 ? 0 : (b > m ? m : b);
}

// (one thread) the metadata of tile t of world g: the tile's level-G cells
// are consecutive in the cell map; its packets are each cell's queries 32 at
// a time
__device__ __forceinline__ void meta_fill(const TileArgs &g, TileMeta &M, int64_t t) {
    int32_t nv = g.scalars[kScalarValidQueries];
    nv = nv < 0 ? 0 : (nv > g.n_q ? (int32_t)g.n_q : nv);
    int32_t m = g.scalars[kScalarLeaves];
    m = m < 0 ? 0 : (m > g.leaf_cap ? (int32_t)g.leaf_cap : m);
    const int T = g.tcells;
    const int64_t ntiles = (1ll << (2 * g.Gp)) / T;
    const int dsh = 2 * (g.G - g.Gp);
    M.t = t;
    M.valid = t >= 0 && t < ntiles;
    M.nv = nv;
    M.m = m;
    M.T = T;
    M.qa = M.qb = M.cnt = 0;
    M.pp[T] = 0;
    if (!M.valid) return;
    const int64_t c0 = t * T;
    int32_t qa = g.qcs[c0], qb = g.qcs[c0 + T];
    qa = qa < 0 ? 0 : (qa > nv ? nv : qa);
    qb = qb < qa ? qa : (qb > nv ? nv : qb);
    M.qa = qa;
    M.qb = qb;
    if (qb == qa) return;
    const int32_t la = clamp_leaf(g.cb[c0 << dsh], m);
    const int32_t lb = clamp_leaf(g.cb[(c0 + T) << dsh], m);
    M.cnt = g.bstart[lb] - g.bstart[la];
    int32_t acc = 0, af = 0, ap = 0;
    for (int i = 0; i < T; ++i) {
        int32_t a = g.qcs[c0 + i], b = g.qcs[c0 + i + 1];
        a = a < qa ? qa : (a > qb ? qb : a);
        b = b < a ? a : (b > qb ? qb : b);
        M.cq[i] = a;
        M.cn[i] = b - a;
        M.pp[i] = acc;
        M.pf[i] = af;
        M.ppart[i] = ap;
        acc += (b - a + 31) >> 5;
        af += (b - a) >> 5;
        ap += ((b - a) & 31) != 0 ? 1 : 0;
    }
    M.pp[T] = acc;
    M.pf[T] = af;
    M.ppart[T] = ap;
}

}  // namespace

// One tile of world g (its metadata M, already loaded): query box, margin,
// staging, then the packets; `prefetch` (called by every thread once, while
// no thread reads the other metadata slot) starts loading the next tile.
template <int KC, class Prefetch>
__device__ __forceinline__ void tile_body(const TileArgs &g, TileSmem &s, const TileMeta &M,
                                          const Prefetch &prefetch) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const float kInf = __int_as_float(0x7f800000);
    const int T = M.T;
    const int32_t m = M.m;
    const float cside = ldexpf(g.side, -g.Gp);
    const int32_t qa = M.qa, qb = M.qb, nq = qb - qa, npk = M.pp[T];
    if (nq == 0) {
        __syncthreads();  // every thread has read M
        prefetch();
        return;
    }
    // a tile that cannot be staged (too many objects or queries) goes on
    // at once
    const bool early_ok = nq <= kTileMaxQ && M.cnt > 0 && M.cnt <= kTileObj;
    if (tid == 0) {
        s.rho = (float)M.cnt / ((float)T * cside * cside);
        s.ok = 0;
        s.next_pk = 0;
    }

    // the tile's query box
    float bx0 = kInf, bx1 = -kInf, by0 = kInf, by1 = -kInf;
    for (int32_t q = qa + tid; early_ok && q < qb; q += kTileThreads) {
        const float x = g.qs_x[q], y = g.qs_y[q];
        bx0 = fminf(bx0, x);
        bx1 = fmaxf(bx1, x);
        by0 = fminf(by0, y);
        by1 = fmaxf(by1, y);
    }
    bx0 = warp_min(bx0);
    bx1 = warp_max(bx1);
    by0 = warp_min(by0);
    by1 = warp_max(by1);
    if (lane == 0) {
        s.red[0][wid] = bx0;
        s.red[1][wid] = bx1;
        s.red[2][wid] = by0;
        s.red[3][wid] = by1;
    }
    __syncthreads();
    if (tid == 0 && early_ok) {
        for (int w = 1; w < kTileWarps; ++w) {
            bx0 = fminf(bx0, s.red[0][w]);
            bx1 = fmaxf(bx1, s.red[1][w]);
            by0 = fminf(by0, s.red[2][w]);
            by1 = fmaxf(by1, s.red[3][w]);
        }
        int ok = bx0 <= bx1 && by0 <= by1;
        const float rho = s.rho;
        // the margin: a disc of twice the area the first thresholds
        // expect at the tile's density
        const float fk = (float)g.k;
        const float H = __fsqrt_ru(2.f * (fk + 4.f * sqrtf(fk) + 4.f) / (3.14159265f * rho));
        const float hx0 = __fsub_rd(bx0, H), hx1 = __fadd_ru(bx1, H);
        const float hy0 = __fsub_rd(by0, H), hy1 = __fadd_ru(by1, H);
        ok = ok && H > 0.f && H < kInf && hx0 < hx1 && hy0 < hy1;
        const int gx0 = cell_g(hx0, g.x0, g.scale_g, g.G), gx1 = cell_g(hx1, g.x0, g.scale_g, g.G);
        const int gy0 = cell_g(hy0, g.y0, g.scale_g, g.G), gy1 = cell_g(hy1, g.y0, g.scale_g, g.G);
        const int ngx = gx1 - gx0 + 1, ngy = gy1 - gy0 + 1;
        ok = ok && (int64_t)ngx * ngy <= kTileStage;
        // micro-cells of about one object (kTileAspect times as high as
        // wide), at most kTileCells
        const float W = hx1 - hx0, Hh = hy1 - hy0;
        float c = sqrtf(1.f / (kTileAspect * rho));
        int nmx = 1, nmy = 1;
        if (ok) {
            nmx = max(1, min(kTileCells, (int)ceilf(W / c)));
            nmy = max(1, min(kTileCells, (int)ceilf(Hh / (kTileAspect * c))));
            if (nmx * nmy > kTileCells) {
                c *= sqrtf((float)(nmx * nmy) / (float)kTileCells) * 1.02f;
                nmx = max(1, min(kTileCells, (int)ceilf(W / c)));
                nmy = max(1, min(kTileCells / nmx, (int)ceilf(Hh / (kTileAspect * c))));
            }
        }
        s.ok = ok;
        s.hx0 = hx0;
        s.hx1 = hx1;
        s.hy0 = hy0;
        s.hy1 = hy1;
        s.nmx = nmx;
        s.nmy = nmy;
        s.iw = (float)nmx / W;
        s.ih = (float)nmy / Hh;
        s.rho = rho;
        s.ngx = ngx;
        s.ng = ok ? ngx * ngy : 0;
        s.gx0 = gx0;
        s.gx1 = gx1;
        s.gy0 = gy0;
        s.gy1 = gy1;
    }
    __syncthreads();
    int ok = s.ok;
    const int ng = s.ng, nmx = s.nmx, nmy = s.nmy, ncells = nmx * nmy;
    uint32_t S = 0;
    if (ok) {
        // staged level-G cells: counts, then their first staged index
        int32_t cc = 0, oa = 0;
        if (tid < ng) {
            const int cx = s.gx0 + tid % s.ngx, cy = s.gy0 + tid / s.ngx;
            const uint32_t mc = interleave((uint32_t)cx, (uint32_t)cy);
            const int32_t la = clamp_leaf(g.cb[mc], m);
            const int32_t lb = clamp_leaf(g.cb[mc + 1], m);
            oa = g.bstart[la];
            cc = g.bstart[lb] - oa;
            cc = cc > 0 ? cc : 0;
        }
        for (int i = tid; i <= ncells; i += kTileThreads) s.cs[i] = 0;
        const uint32_t ex = block_excl_scan_256((uint32_t)cc, s.scan_tmp, &s.scan_total);
        if (tid < ng) {
            s.gofs[tid] = (int32_t)ex;
            s.goa[tid] = oa;
        }
        S = s.scan_total;
        if (tid == 0) s.gofs[ng] = (int32_t)S;
        ok = S > 0 && S <= (uint32_t)kTileObj;
        __syncthreads();
    }
    if (!ok) {
        // the tile goes to the gathered form, as the packets k_packets cuts
        if (tid == 0) {
            s.pk_full = atomicAdd(g.scalars + kScalarPackets, M.pf[T]);
            s.pk_part = atomicAdd(g.scalars + kScalarPartialPackets, M.ppart[T]);
        }
        __syncthreads();
        prefetch();
        for (int32_t i = tid; i < npk; i += kTileThreads) {
            int c = 0;
#pragma unroll
            for (int u = 1; u < kTileMaxCells; ++u)
                if (u < T && i >= M.pp[u]) c = u;
            const int32_t o = i - M.pp[c];
            const int32_t q0 = M.cq[c] + 32 * o, ql = min(32, M.cn[c] - 32 * o);
            const int64_t slot = ql == 32
                                     ? (int64_t)s.pk_full + M.pf[c] + o
                                     : g.pk_cap - 1 - ((int64_t)s.pk_part + M.ppart[c]);
            if (slot >= 0 && slot < g.pk_cap) {
                g.pk_start[slot] = q0;
                g.pk_len[slot] = ql;
            }
        }
        return;
    }
    // stage the objects: counting sort by micro-cell (row-major)
    {
        const float hx0 = s.hx0, hy0 = s.hy0, iw = s.iw, ih = s.ih;
        constexpr int kPer = (kTileObj + kTileThreads) / kTileThreads;
        float lx[kPer], ly[kPer];
        int32_t lid[kPer], lm[kPer], lr[kPer];
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int si = tid + u * kTileThreads;
            lm[u] = -1;
            lx[u] = ly[u] = 0.f;
            lid[u] = lr[u] = 0;
            if (si < (int)S) {
                int lo = 0, hi = ng - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s.gofs[mid] <= si) lo = mid;
                    else hi = mid - 1;
                }
                int64_t gi = (int64_t)s.goa[lo] + (si - s.gofs[lo]);
                if (!KNN_IN_BOUNDS(gi, 0, g.n, g.err)) gi = 0;
                lx[u] = g.xs[gi];
                ly[u] = g.ys[gi];
                lid[u] = g.sid[gi];
                const int mc = mcell(ly[u], hy0, ih, nmy) * nmx + mcell(lx[u], hx0, iw, nmx);
                lm[u] = mc;
                lr[u] = atomicAdd(&s.cs[mc], 1);
            }
        }
        __syncthreads();
        // exclusive scan of the micro-cell counts, four cells per thread
        {
            int32_t v[4];
            uint32_t sum = 0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = tid * 4 + u;
                v[u] = i < ncells ? s.cs[i] : 0;
                sum += (uint32_t)v[u];
            }
            uint32_t ex = block_excl_scan_256(sum, s.scan_tmp, nullptr);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = tid * 4 + u;
                if (i < ncells) s.cs[i] = (int32_t)ex;
                ex += (uint32_t)v[u];
            }
            if (tid == 0) s.cs[ncells] = (int32_t)S;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            if (lm[u] >= 0) {
                int pos = s.cs[lm[u]] + lr[u];
                if (!KNN_IN_BOUNDS(pos, 0, kTileObj, g.err)) pos = 0;
                s.xy[pos] = make_float2(lx[u], ly[u]);
                s.id[pos] = lid[u];
            }
        }
        __syncthreads();
    }
    // the next tile's metadata (thread 0, while the other warps start on
    // the packets), then the tile's packets, taken by the warps one at a
    // time
    prefetch();
    for (;;) {
        int32_t pw = 0;
        if (lane == 0) pw = atomicAdd(&s.next_pk, 1);
        pw = __shfl_sync(kFull, pw, 0);
        if (pw >= npk) break;
        int32_t q0, ql;
        tile_pk(M, T, pw, q0, ql);
        if (ql > 0) tile_packet<KC>(g, s, q0, ql, tid);
    }
}

template <int KC>
__global__ void __launch_bounds__(kTileThreads, KC <= 16 ? 4 : 2)
    k_expand_tile(const TileArgs g) {
    __shared__ TileSmem s;
    if (threadIdx.x == 0) {
        s.mi = 0;
        meta_fill(g, s.meta[0], atomicAdd(g.tile_counter, 1u));
    }
    for (;;) {
        __syncthreads();  // the last tile's staged objects are no longer read
        const int mi = s.mi;  // this tile's metadata (thread 0 fills the other slot)
        const TileMeta &M = s.meta[mi];
        if (!M.valid) break;
        tile_body<KC>(g, s, M, [&]() {
            if (threadIdx.x == 0) {
                meta_fill(g, s.meta[mi ^ 1], atomicAdd(g.tile_counter, 1u));
                s.mi = mi ^ 1;
            }
        });
    }
}

// Batched form: one grid takes the tiles of many worlds (same list size
// class).  pfx[w] counts the tiles of the worlds before w (from the worlds'
// plans, on the host); a ticket's world is found by binary search, and its
// arguments are copied into one of two shared-memory slots when the world
// changes (the other slot may still serve the tile being scanned).
struct TileBatch {
    const TileArgs *worlds;
    const long long *pfx;  // n + 1 entries
    unsigned long long *counter;
    int n;
};
static_assert(sizeof(TileArgs) % 4 == 0, "copied by 32-bit words");

template <int KC>
__global__ void __launch_bounds__(kTileThreads, KC <= 16 ? 4 : 2)
    k_expand_tile_batch(const TileBatch b) {
    __shared__ TileSmem s;
    __shared__ TileArgs wa[2];
    const long long total = b.pfx[b.n];
    // (thread 0) the next ticket's world and tile metadata into meta[slot]
    auto next = [&](int slot, int as_prev, int64_t w_prev) {
        TileMeta &M = s.meta[slot];
        const long long t = (long long)atomicAdd(b.counter, 1ull);
        if (t >= total) {
            M.valid = 0;
            return;
        }
        int lo = 0, hi = b.n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (b.pfx[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        int as = as_prev;
        if (lo != w_prev) {
            as = as_prev ^ 1;
            const uint32_t *src = reinterpret_cast<const uint32_t *>(b.worlds + lo);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&wa[as]);
            for (int i = 0; i < (int)(sizeof(TileArgs) / 4); ++i) dst[i] = src[i];
        }
        meta_fill(wa[as], M, t - b.pfx[lo]);
        M.as = as;
        M.w = lo;
    };
    if (threadIdx.x == 0) {
        s.mi = 0;
        next(0, 1, -1);
    }
    for (;;) {
        __syncthreads();  // the last tile's staged objects are no longer read
        const int mi = s.mi;
        const TileMeta &M = s.meta[mi];
        if (!M.valid) break;
        tile_body<KC>(wa[M.as], s, M, [&]() {
            if (threadIdx.x == 0) {
                next(mi ^ 1, M.as, M.w);
                s.mi = mi ^ 1;
            }
        });
    }
}

namespace {

template <int KC>
int tile_batch_blocks_per_sm(int device) {
    static int cached[64] = {0};
    const int slot = device >= 0 && device < 64 ? device : 0;
    if (cached[slot] == 0) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_expand_tile_batch<KC>,
                                                      kTileThreads, 0);
        cached[slot] = per_sm < 1 ? 1 : per_sm;
    }
    return cached[slot];
}

template <int KC>
int tile_blocks_per_sm(int device) {
    static int cached[64] = {0};
    const int slot = device >= 0 && device < 64 ? device : 0;
    if (cached[slot] == 0) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_expand_tile<KC>, kTileThreads, 0);
        cached[slot] = per_sm < 1 ? 1 : per_sm;
    }
    return cached[slot];
}

template <int KC>
void run_tile(const TileArgs &a, int device, cudaStream_t s) {
    const int per_sm = tile_blocks_per_sm<KC>(device);
    k_expand_tile<KC><<<num_sms(device) * per_sm, kTileThreads, 0, s>>>(a);
}

}  // namespace

void prepare_expand_tile(int device) {
    tile_blocks_per_sm<8>(device);
    tile_blocks_per_sm<16>(device);
    tile_blocks_per_sm<32>(device);
    tile_batch_blocks_per_sm<8>(device);
    tile_batch_blocks_per_sm<16>(device);
    tile_batch_blocks_per_sm<32>(device);
}

static TileArgs tile_args(World &w, const Plan &p, int32_t k, int64_t n_q, int32_t *out_ids,
                          float *out_d2, const int32_t *q_k) {
    TileArgs a;
    a.xs = w.xs;
    a.ys = w.ys;
    a.sid = w.sid;
    a.cb = w.cb;
    a.bstart = w.bstart;
    a.qs_x = w.qs_x;
    a.qs_y = w.qs_y;
    a.qs_id = w.qs_id;
    a.qs_orig = w.qs_orig;
    a.qcs = w.qcs;
    a.scalars = w.scalars;
    a.tile_counter = w.counters + kCtrTile;
    a.pk_start = w.pk_start;
    a.pk_len = w.pk_len;
    a.out_ids = out_ids;
    a.out_d2 = out_d2;
    a.q_k = q_k;
    a.err = w.err;
    a.x0 = w.desc.x0;
    a.y0 = w.desc.y0;
    a.side = w.desc.side;
    a.scale_g = ldexpf(w.scale, -(p.L - p.G));
    a.G = p.G;
    a.Gp = p.Gp;
    a.k = k;
    // two cells per tile while a cell holds fewer than about 400 queries
    // (fewer barriers per query; a warp takes about two packets per tile)
    const int64_t ncell = 1ll << (2 * p.Gp);
    a.tcells = ncell >= 2 && (double)n_q < 400.0 * (double)ncell ? 2 : 1;
    a.vec_out = q_k == nullptr && k % 4 == 0 &&
                ((reinterpret_cast<uintptr_t>(out_ids) | reinterpret_cast<uintptr_t>(out_d2)) &
                 15u) == 0;
    a.n = w.n;
    a.n_q = n_q;
    a.pk_cap = packet_capacity(w);
    a.leaf_cap = w.leaf_cap;
    return a;
}

void launch_expand_tile(World &w, const Plan &p, int32_t k, int64_t n_q, int32_t *out_ids,
                        float *out_d2, const int32_t *q_k, cudaStream_t s) {
    if (n_q <= 0) return;
    const TileArgs a = tile_args(w, p, k, n_q, out_ids, out_d2, q_k);
    if (k <= 8) run_tile<8>(a, w.device, s);
    else if (k <= 16) run_tile<16>(a, w.device, s);
    else run_tile<32>(a, w.device, s);
    ++w.launches;
}

// ---------------------------------------------------------------------------
// Batched tiles (many worlds, one grid per list size)

size_t tile_batch_entry_bytes() { return sizeof(TileArgs); }

int64_t tile_batch_entry(World &w, const Plan &p, const knn_tick_args &t, void *dst) {
    const TileArgs a = tile_args(w, p, t.k, t.n_q, t.out_ids_dev, t.out_d2_dev, t.q_k_dev);
    std::memcpy(dst, &a, sizeof(a));
    return (1ll << (2 * p.Gp)) / a.tcells;
}

namespace {
template <int KC>
void run_tile_batch(const TileBatch &b, int device, cudaStream_t s) {
    const int per_sm = tile_batch_blocks_per_sm<KC>(device);
    k_expand_tile_batch<KC><<<num_sms(device) * per_sm, kTileThreads, 0, s>>>(b);
}
}  // namespace

void launch_tile_batch(int kc, const void *table, int n, const long long *pfx,
                       unsigned long long *counter, int device, cudaStream_t s) {
    if (n <= 0) return;
    cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    const TileBatch b{static_cast<const TileArgs *>(table), pfx, counter, n};
    if (kc <= 8) run_tile_batch<8>(b, device, s);
    else if (kc <= 16) run_tile_batch<16>(b, device, s);
    else run_tile_batch<32>(b, device, s);
}

}  // namespace knnq
