// a7 + a8 in the paper's multi-pass form (Section 4.2, first iteration and
// subsequent iterations, Alg. 2): an ablation of the single-pass expansion
// with identical rows.
//
// One thread per query (the paper's cached variant); the query's list lives
// in its output row between iterations and in registers within one.
//  * First iteration: every query scans the leaves of its own level-G cell.
//  * Subsequent iterations alternate the two sub-visits, left then right in
//    Morton order: each query active in the direction moves from the cell it
//    reached last to the next cell in that direction whose quadrant may still
//    hold an object nearer than its k-th distance (or any object while its
//    list is not full), skipping whole quadrants of the virtual full quadtree
//    above level G that are out of reach, and scans that cell's leaves.  A
//    query that runs off the end of the order is done in that direction.
//  * The loop stops once an iteration of each direction found no cell.
// The cells a query never scans are farther than its final k-th distance, so
// the rows are exact.  Iterations are separated by grid-wide barriers of one
// cooperative launch (no host round trip).  Unlike the paper, the active
// queries keep their Morton order between iterations instead of being sorted
// by their new cells; the rows do not depend on the order.
#include <cooperative_groups.h>

#include "knn_device.cuh"
#include "knn_internal.h"

namespace cg = cooperative_groups;

namespace knnq {

struct IterArgs {
    const float *xs, *ys;
    const int32_t *sid;
    const float4 *baabb;
    const int2 *brange;
    const int32_t *cb;
    const float *qs_x, *qs_y;
    const int32_t *qs_id, *qs_orig;
    const int32_t *scalars;
    uint32_t *nav;       // per sorted query: [2j] left position, [2j + 1] right position
    uint32_t *counters;  // [0], [1]: cumulative active counts of even / odd iterations
    int32_t *out_ids;
    float *out_d2;
    float x0, y0, side, scale_g;
    float pad;  // outward move of interior quadrant edges (a few ulps of the coordinates)
    int G, k;
    int64_t n_q;
    const int32_t *q_k;  // per-query list sizes by caller index (NULL: all k)
    uint32_t *err;
};

constexpr uint32_t kNavDone = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t compact_bits(uint32_t v) {  // inverse of spread_bits
    v &= 0x55555555u;
    v = (v | (v >> 1)) & 0x33333333u;
    v = (v | (v >> 2)) & 0x0F0F0F0Fu;
    v = (v | (v >> 4)) & 0x00FF00FFu;
    v = (v | (v >> 8)) & 0x0000FFFFu;
    return v;
}

// Lower bound of the squared distance from (qx, qy) to the objects the cell
// mapping puts in the quadrant with level-l code z: the quadrant's edges, each
// moved outward by a few ulps, and open to infinity on the sides of the domain
// (positions outside the domain are clamped into the edge cells).
__device__ __forceinline__ float quad_lb(uint32_t z, int l, float qx, float qy,
                                        const IterArgs &g) {
    const float inf = __int_as_float(0x7f800000);
    const float w = ldexpf(g.side, -l);
    const uint32_t ix = compact_bits(z), iy = compact_bits(z >> 1), last = (1u << l) - 1u;
    const float cx = (float)ix, cy = (float)iy;
    const float x0 = ix == 0 ? -inf : __fsub_rd(__fmaf_rd(cx, w, g.x0), g.pad);
    const float x1 = ix == last ? inf : __fadd_ru(__fmaf_ru(cx + 1.f, w, g.x0), g.pad);
    const float y0 = iy == 0 ? -inf : __fsub_rd(__fmaf_rd(cy, w, g.y0), g.pad);
    const float y1 = iy == last ? inf : __fadd_ru(__fmaf_ru(cy + 1.f, w, g.y0), g.pad);
    return box_lb(x0, y0, x1, y1, qx, qy, qx, qy);
}

// Insert key into the ascending list (the largest entry drops out).
template <int KC>
__device__ __forceinline__ void insert_key(unsigned long long (&lst)[KC],
                                           unsigned long long key) {
    if (!(key < lst[KC - 1])) return;
#pragma unroll
    for (int i = KC - 1; i > 0; --i) {
        const bool shift = key < lst[i - 1];
        lst[i] = shift ? lst[i - 1] : (key < lst[i] ? key : lst[i]);
    }
    lst[0] = key < lst[0] ? key : lst[0];
}

// Scan the leaves of level-G cell c that may hold a better object.
template <int KC>
__device__ void scan_cell(uint32_t c, float qx, float qy, int32_t self, int32_t m,
                          unsigned long long (&lst)[KC], const IterArgs &g) {
    int32_t lo = g.cb[c], hi = g.cb[c + 1];
    lo = lo < 0 ? 0 : lo;
    hi = hi < m ? hi : m;
    for (int32_t b = lo; b < hi; ++b) {
        const int2 rg = g.brange[b];
        if (!(rg.x < rg.y)) continue;
        const float4 bb = g.baabb[b];
        const float thr = __uint_as_float((uint32_t)(lst[KC - 1] >> 32));
        if (!(box_lb(bb.x, bb.y, bb.z, bb.w, qx, qy, qx, qy) <= thr)) continue;
        for (int32_t o = rg.x; o < rg.y; ++o) {
            const float dx = __fsub_rn(qx, g.xs[o]);
            const float dy = __fsub_rn(qy, g.ys[o]);
            const float d = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
            const int32_t idp1 = g.sid[o] + 1;
            if (idp1 != self)
                insert_key<KC>(lst,
                               ((unsigned long long)__float_as_uint(d) << 32) | (uint32_t)idp1);
        }
    }
}

// The next level-G cell after `from` (exclusive) in direction dir (0 left,
// 1 right) that has leaves and whose quadrant lies within thr; kNavDone if
// none.  Quadrants above G that are out of reach are skipped whole.
__device__ uint32_t next_cell(uint32_t from, int dir, float qx, float qy, float thr,
                              const IterArgs &g) {
    const int G = g.G;
    const uint32_t ncell = 1u << (2 * G);
    if (dir == 0 && from == 0) return kNavDone;
    if (dir == 1 && from + 1 >= ncell) return kNavDone;
    uint32_t c = dir == 0 ? from - 1 : from + 1;
    for (;;) {
        // the largest quadrant that starts (right) or ends (left) at c
        int l = G;
        while (l > 0) {
            const uint32_t span = 1u << (2 * (G - l + 1));
            const bool aligned = dir == 1 ? (c & (span - 1)) == 0 : ((c + 1) & (span - 1)) == 0;
            if (!aligned) break;
            --l;
        }
        // descend until a quadrant is within reach
        for (;;) {
            const uint32_t z = c >> (2 * (G - l));
            if (quad_lb(z, l, qx, qy, g) <= thr) {
                if (l == G) break;
                ++l;  // look at its first (right) or last (left) child
                continue;
            }
            // out of reach: skip it whole
            const uint32_t span = 1u << (2 * (G - l));
            if (dir == 1) {
                const uint32_t first = z << (2 * (G - l));
                if (first + span >= ncell) return kNavDone;
                c = first + span;
            } else {
                const uint32_t first = z << (2 * (G - l));
                if (first == 0) return kNavDone;
                c = first - 1;
            }
            l = -1;
            break;
        }
        if (l < 0) continue;  // skipped; find the quadrant at the new position
        if (g.cb[c] < g.cb[c + 1]) return c;
        // an empty cell: step on
        if (dir == 1) {
            if (c + 1 >= ncell) return kNavDone;
            ++c;
        } else {
            if (c == 0) return kNavDone;
            --c;
        }
    }
}

// The query's list, kept in its row (k wide; the first kq entries are the
// list, the rest padding), as kq keys after KC - kq zero slots.
template <int KC>
__device__ __forceinline__ void load_row(unsigned long long (&lst)[KC], int32_t orig, int k,
                                         int kq, const IterArgs &g) {
    const int32_t *oi = g.out_ids + (int64_t)orig * k;
    const float *od = g.out_d2 + (int64_t)orig * k;
#pragma unroll
    for (int i = 0; i < KC; ++i) {
        const int r = i - (KC - kq);
        if (r < 0) {
            lst[i] = 0ull;
        } else {
            const int32_t id = oi[r];
            lst[i] = ((unsigned long long)__float_as_uint(od[r]) << 32) |
                     (uint32_t)(id < 0 ? 0xFFFFFFFFu : (uint32_t)(id + 1));
        }
    }
}

template <int KC>
__device__ __forceinline__ void store_row(const unsigned long long (&lst)[KC], int32_t orig,
                                          int k, int kq, const IterArgs &g) {
    int32_t *oi = g.out_ids + (int64_t)orig * k;
    float *od = g.out_d2 + (int64_t)orig * k;
#pragma unroll
    for (int i = 0; i < KC; ++i) {
        const int r = i - (KC - kq);
        if (r >= 0) {
            oi[r] = key_id(lst[i]);
            od[r] = __uint_as_float((uint32_t)(lst[i] >> 32));
        }
    }
}

// This query's list size (Section 2.1, q = (x, y, k)); 0: no neighbours.
__device__ __forceinline__ int query_k(int32_t orig, const IterArgs &g) {
    if (!g.q_k) return g.k;
    const int kq = g.q_k[orig];
    if (kq < 0 || kq > g.k) {
        atomicOr(g.err, kErrBadQuery);
        return 0;
    }
    return kq;
}

template <int KC>
__global__ void __launch_bounds__(128) k_expand_iter(const IterArgs g) {
    cg::grid_group grid = cg::this_grid();
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int32_t nv = g.scalars[kScalarValidQueries];
    nv = nv < 0 ? 0 : (nv > g.n_q ? (int32_t)g.n_q : nv);
    int32_t m = g.scalars[kScalarLeaves];
    m = m < 0 ? 0 : m;
    const int k = g.k;

    // first iteration: the query's own cell
    for (int64_t j = tid; j < nv; j += T) {
        const int32_t orig = g.qs_orig[j];
        if (orig < 0) {
            g.nav[2 * j] = g.nav[2 * j + 1] = kNavDone;
            continue;
        }
        const float qx = g.qs_x[j], qy = g.qs_y[j];
        const int kq = query_k(orig, g);
        // padding after the list (and the whole row when kq is 0)
        for (int r = kq; r < k; ++r) {
            g.out_ids[(int64_t)orig * k + r] = -1;
            g.out_d2[(int64_t)orig * k + r] = __int_as_float(0x7f800000);
        }
        if (kq == 0) {
            g.nav[2 * j] = g.nav[2 * j + 1] = kNavDone;
            continue;
        }
        const uint32_t c = interleave((uint32_t)cell_g(qx, g.x0, g.scale_g, g.G),
                                      (uint32_t)cell_g(qy, g.y0, g.scale_g, g.G));
        unsigned long long lst[KC];
#pragma unroll
        for (int i = 0; i < KC; ++i) lst[i] = i < KC - kq ? 0ull : kPad;
        scan_cell<KC>(c, qx, qy, g.qs_id[j] + 1, m, lst, g);
        store_row<KC>(lst, orig, k, kq, g);
        g.nav[2 * j] = c;
        g.nav[2 * j + 1] = c;
    }
    grid.sync();

    // subsequent iterations: left, right, left, ...
    uint32_t seen[2] = {0u, 0u};
    uint32_t last_active[2] = {1u, 1u};
    for (int it = 0;; ++it) {
        const int dir = it & 1;
        uint32_t found = 0;
        for (int64_t j = tid; j < nv; j += T) {
            const uint32_t from = g.nav[2 * j + dir];
            if (from == kNavDone) continue;
            const int32_t orig = g.qs_orig[j];
            const float qx = g.qs_x[j], qy = g.qs_y[j];
            const int kq = g.q_k ? g.q_k[orig] : k;  // checked in the first iteration
            unsigned long long lst[KC];
            load_row<KC>(lst, orig, k, kq, g);
            const float thr = __uint_as_float((uint32_t)(lst[KC - 1] >> 32));
            const uint32_t c = next_cell(from, dir, qx, qy, thr, g);
            g.nav[2 * j + dir] = c;
            if (c == kNavDone) continue;
            scan_cell<KC>(c, qx, qy, g.qs_id[j] + 1, m, lst, g);
            store_row<KC>(lst, orig, k, kq, g);
            ++found;
        }
        if (found) atomicAdd(g.counters + dir, found);
        grid.sync();
        // every thread reads the same count: this parity is not touched again
        // before the next barrier
        const uint32_t total = *reinterpret_cast<volatile uint32_t *>(g.counters + dir);
        last_active[dir] = total - seen[dir];
        seen[dir] = total;
        if (last_active[0] == 0u && last_active[1] == 0u) break;
    }
}

template <int KC>
static void run_iter(const IterArgs &a, int device, cudaStream_t s) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_expand_iter<KC>, 128, 0);
    if (per_sm < 1) per_sm = 1;
    dim3 grid((unsigned)(num_sms(device) * per_sm)), block(128);
    IterArgs args = a;
    void *params[] = {&args};
    cudaLaunchCooperativeKernel((const void *)k_expand_iter<KC>, grid, block, params, 0, s);
}

void launch_expand_iter(World &w, const Plan &p, int32_t k, int64_t n_q, int32_t *out_ids,
                        float *out_d2, const int32_t *q_k, cudaStream_t s) {
    if (n_q <= 0) return;
    IterArgs a;
    a.xs = w.xs;
    a.ys = w.ys;
    a.sid = w.sid;
    a.baabb = w.baabb;
    a.brange = w.brange;
    a.cb = w.cb;
    a.qs_x = w.qs_x;
    a.qs_y = w.qs_y;
    a.qs_id = w.qs_id;
    a.qs_orig = w.qs_orig;
    a.scalars = w.scalars;
    a.nav = w.nav;
    a.counters = w.counters + kCtrIterLeft;
    a.out_ids = out_ids;
    a.out_d2 = out_d2;
    a.x0 = w.desc.x0;
    a.y0 = w.desc.y0;
    a.side = w.desc.side;
    a.scale_g = ldexpf(w.scale, -(p.L - p.G));
    a.pad = 8e-7f * (fabsf(w.desc.x0) + fabsf(w.desc.y0) + w.desc.side);
    a.G = p.G;
    a.k = k;
    a.n_q = n_q;
    a.q_k = q_k;
    a.err = w.err;
    if (k <= 4) run_iter<4>(a, w.device, s);
    else if (k <= 8) run_iter<8>(a, w.device, s);
    else if (k <= 16) run_iter<16>(a, w.device, s);
    else if (k <= 32) run_iter<32>(a, w.device, s);
    else run_iter<64>(a, w.device, s);
    ++w.launches;
}

}  // namespace knnq
