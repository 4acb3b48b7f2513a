// Index construction for one tick (Sections 2.2, 4.1.1, 4.1.2, 4.2.1):
// update scatter, Morton keys, onesweep radix sort, PR-quadtree leaf split,
// leaf bounding boxes, the uniform cell map, query ordering and packets.
#include <algorithm>
#include <cstdio>

#include "knn_device.cuh"
#include "knn_internal.h"

namespace knnq {

static inline int grid_for(int64_t work, int threads, int cap) {
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

// ---------------------------------------------------------------------------
// Position validation (world creation).

__global__ void k_validate_positions(const float *__restrict__ x, const float *__restrict__ y,
                                     int64_t n, uint32_t *flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (!isfinite(x[i]) || !isfinite(y[i])) atomicOr(flag, 1u);
    }
}

void launch_validate_positions(const float *x, const float *y, int64_t n, uint32_t *flag,
                               cudaStream_t s) {
    k_validate_positions<<<grid_for(n, 256, 4096), 256, 0, s>>>(x, y, n, flag);
}

// ---------------------------------------------------------------------------
// a1 -- updates (Section 2.2): the most recent valid update of an object in the
// batch wins.  Pass 1 stamps each object with the largest (tick, index) of a
// valid entry; pass 2 lets only that entry write.

// Index reuse (Section 4 pipeline): the index (the leaves) is rebuilt only
// when needed -- when the last tick's cost grew past a factor of the cost
// right after the last build, after reuse_age ticks at the most, when the
// plan changed, or (decided later in the tick) when an object moved into a
// level-G cell without leaves.  The cost proxy is the sum over leaves of the
// squared object count (candidate pairs).  The decision is taken here, on
// the device, so a recorded tick graph needs no host round trip.
__global__ void k_tick_begin(uint32_t *tickinfo, uint32_t *counters, int n_counters,
                             uint32_t *err, int32_t *scalars, int reuse_age, int reuse_f16,
                             int32_t sig) {
    const int i = threadIdx.x;
    if (i == 0) {
        tickinfo[0] += 64u;  // room for 64 look-back launches per tick
        tickinfo[1] += 1u;
        err[2] = 0u;
        unsigned long long *cost_base =
            reinterpret_cast<unsigned long long *>(scalars + kScalarCostBase);
        unsigned long long *cost_now =
            reinterpret_cast<unsigned long long *>(scalars + kScalarCostNow);
        if (scalars[kScalarRebuild]) {  // the last tick built the leaves
            *cost_base = *cost_now;
            scalars[kScalarIndexAge] = 0;
        }
        const int age = scalars[kScalarIndexAge] + 1;
        const bool rebuild = reuse_age <= 0 || scalars[kScalarIndexSig] != sig ||
                             age > reuse_age ||
                             (reuse_f16 > 0 &&
                              *cost_now * 16ull > (unsigned long long)reuse_f16 * *cost_base);
        scalars[kScalarRebuild] = rebuild ? 1 : 0;
        scalars[kScalarIndexAge] = age;
        *cost_now = 0ull;
    }
    if (i < n_counters) counters[i] = 0u;
}

// The plan an index is built for; bit 29: built for reuse (with empty leaves).
static int32_t index_signature(const Plan &p) {
    return (int32_t)(0x40000000u | (p.reuse_age > 0 ? 0x20000000u : 0u) |
                     ((uint32_t)p.L << 24) | ((uint32_t)p.G << 16) | (uint32_t)p.th);
}

void launch_tick_begin(World &w, const Plan &p, cudaStream_t s) {
    w.site = 0;
    k_tick_begin<<<1, kNumCounters, 0, s>>>(w.tickinfo, w.counters, kNumCounters, w.err,
                                            w.scalars, p.reuse_age, p.reuse_f16,
                                            index_signature(p));
    ++w.launches;
}

__global__ void k_update_stamp(const int32_t *__restrict__ id, const float *__restrict__ ux,
                               const float *__restrict__ uy, int64_t n_upd, int64_t n,
                               unsigned long long *stamp, const uint32_t *__restrict__ tickinfo,
                               uint32_t *err) {
    const unsigned long long tick = tickinfo[1];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_upd;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t o = id[i];
        if (o < 0 || o >= n) {
            atomicOr(err, kErrBadUpdateId);
            continue;
        }
        if (!isfinite(ux[i]) || !isfinite(uy[i])) {
            atomicOr(err, kErrNonFiniteUpdate);
            continue;
        }
        atomicMax(&stamp[o], (tick << 32) | (unsigned long long)i);
    }
}

__global__ void k_update_apply(const int32_t *__restrict__ id, const float *__restrict__ ux,
                               const float *__restrict__ uy, int64_t n_upd, int64_t n,
                               const unsigned long long *__restrict__ stamp,
                               const uint32_t *__restrict__ tickinfo, float *px, float *py) {
    const unsigned long long tick = tickinfo[1];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_upd;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t o = id[i];
        if (o < 0 || o >= n) continue;
        if (stamp[o] == ((tick << 32) | (unsigned long long)i)) {
            px[o] = ux[i];
            py[o] = uy[i];
        }
    }
}

void launch_updates(World &w, const int32_t *id, const float *ux, const float *uy,
                    int64_t n_upd, cudaStream_t s) {
    if (n_upd <= 0) return;
    const int g = grid_for(n_upd, 256, num_sms(w.device) * 8);
    k_update_stamp<<<g, 256, 0, s>>>(id, ux, uy, n_upd, w.n, w.stamp, w.tickinfo, w.err);
    k_update_apply<<<g, 256, 0, s>>>(id, ux, uy, n_upd, w.n, w.stamp, w.tickinfo, w.px, w.py);
    w.launches += 2;
}

// ---------------------------------------------------------------------------
// a2 -- Morton keys at level L plus the digit histograms of every radix pass.

__global__ void __launch_bounds__(256) k_keys_hist(
    const float *__restrict__ px, const float *__restrict__ py, int64_t n, float x0, float y0,
    float scale, int L, int passes, uint32_t *__restrict__ key, int32_t *__restrict__ val,
    uint32_t *hist, const int32_t *rebuild, bool vec4) {
    if (rebuild && *rebuild == 0) return;  // this tick reuses the leaves
    __shared__ uint32_t h[4][256];
    for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    // four objects per thread with 16-byte loads and stores when every array
    // is 16-byte aligned (world arrays are; caller arrays may not be)
    const int64_t n4 = vec4 ? n & ~int64_t(3) : 0;
    for (int64_t i = 4 * (blockIdx.x * (int64_t)blockDim.x + threadIdx.x); i < n4;
         i += 4 * (int64_t)gridDim.x * blockDim.x) {
        const float4 xv = *reinterpret_cast<const float4 *>(px + i);
        const float4 yv = *reinterpret_cast<const float4 *>(py + i);
        uint4 kv;
        kv.x = morton_key(xv.x, yv.x, x0, y0, scale, L);
        kv.y = morton_key(xv.y, yv.y, x0, y0, scale, L);
        kv.z = morton_key(xv.z, yv.z, x0, y0, scale, L);
        kv.w = morton_key(xv.w, yv.w, x0, y0, scale, L);
        *reinterpret_cast<uint4 *>(key + i) = kv;
        *reinterpret_cast<int4 *>(val + i) =
            make_int4((int32_t)i, (int32_t)i + 1, (int32_t)i + 2, (int32_t)i + 3);
        for (int p = 0; p < passes; ++p) {
            atomicAdd(&h[p][(kv.x >> (8 * p)) & 255u], 1u);
            atomicAdd(&h[p][(kv.y >> (8 * p)) & 255u], 1u);
            atomicAdd(&h[p][(kv.z >> (8 * p)) & 255u], 1u);
            atomicAdd(&h[p][(kv.w >> (8 * p)) & 255u], 1u);
        }
    }
    for (int64_t i = n4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = morton_key(px[i], py[i], x0, y0, scale, L);
        key[i] = k;
        val[i] = (int32_t)i;
        for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(k >> (8 * p)) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += blockDim.x) {
        const uint32_t c = (&h[0][0])[i];
        if (c) atomicAdd(&hist[i], c);
    }
}

// Query centres given explicitly: key of the centre, value = caller index.
// Invalid queries (issuer outside [-1, n) or non-finite centre) get a padded
// row now, the largest level-L key and value -1 - i so that later stages skip
// them.
__global__ void __launch_bounds__(256) k_query_keys_hist(
    const int32_t *__restrict__ q_id, const float *__restrict__ q_x,
    const float *__restrict__ q_y, int64_t n_q, int64_t n, float x0, float y0, float scale,
    int L, int passes, int k, uint32_t *__restrict__ key, int32_t *__restrict__ val,
    uint32_t *hist, int32_t *out_ids, float *out_d2, uint32_t *err) {
    __shared__ uint32_t h[4][256];
    for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_q;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = q_id[i];
        const float qx = q_x[i], qy = q_y[i];
        const bool ok = s >= -1 && s < n && isfinite(qx) && isfinite(qy);
        uint32_t kk = (uint32_t)((1ull << (2 * L)) - 1ull);  // last level-L cell
        if (ok) {
            kk = morton_key(qx, qy, x0, y0, scale, L);
            val[i] = (int32_t)i;
        } else {
            val[i] = -1 - (int32_t)i;
            atomicOr(err, kErrBadQuery);
            for (int r = 0; r < k; ++r) {
                out_ids[i * k + r] = -1;
                out_d2[i * k + r] = __int_as_float(0x7f800000);
            }
        }
        key[i] = kk;
        for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(kk >> (8 * p)) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += blockDim.x) {
        const uint32_t c = (&h[0][0])[i];
        if (c) atomicAdd(&hist[i], c);
    }
}

// ---------------------------------------------------------------------------
// a3 -- one stable LSD radix pass over 8 bits (onesweep: ranks within the tile
// by warp multi-split -- the lanes holding the same digit found by one ballot
// per digit bit -- and digit offsets across tiles by decoupled look-back).

__global__ void __launch_bounds__(kSortThreads) k_onesweep(
    const uint32_t *__restrict__ kin, const int32_t *__restrict__ vin,
    uint32_t *__restrict__ kout, int32_t *__restrict__ vout, int64_t n, int shift,
    const uint32_t *__restrict__ hist, uint64_t *status, uint32_t *ticket,
    const uint32_t *__restrict__ tickinfo, uint32_t site, uint32_t *err, const int32_t *rebuild) {
    if (rebuild && *rebuild == 0) return;  // this tick reuses the leaves
    __shared__ uint32_t s_wcnt[8][256];
    __shared__ uint32_t s_texcl[256];
    __shared__ uint32_t s_gbase[256];
    __shared__ uint32_t s_keys[kSortTile];
    __shared__ int32_t s_vals[kSortTile];
    __shared__ uint32_t s_tmp[8];
    __shared__ uint32_t s_tile;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(ticket, 1u);
    for (int i = tid; i < 8 * 256; i += kSortThreads) (&s_wcnt[0][0])[i] = 0;
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint32_t epoch = tickinfo[0] + site;
    const int64_t base = (int64_t)tile * kSortTile;
    const int64_t wbase = base + (int64_t)warp * (32 * kSortItems);

    uint32_t k[kSortItems];
    int32_t v[kSortItems];
    uint32_t r[kSortItems];
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const int64_t idx = wbase + j * 32 + lane;
        k[j] = idx < n ? kin[idx] : 0u;
        v[j] = idx < n ? vin[idx] : 0;
        r[j] = 0;
    }
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const bool valid = wbase + j * 32 + lane < n;
        const unsigned vm = __ballot_sync(kFull, valid);
        const uint32_t d = (k[j] >> shift) & 255u;
        // lanes holding the same digit: one ballot per digit bit
        unsigned peers = vm;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const unsigned bb = __ballot_sync(kFull, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? bb : ~bb;
        }
        uint32_t before = 0;
        if (valid) {
            before = s_wcnt[warp][d];
            r[j] = before + __popc(peers & lt);
        }
        __syncwarp();
        if (valid && (peers & lt) == 0u) s_wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();

    const int d = tid;  // one digit per thread
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const uint32_t c = s_wcnt[w][d];
        s_wcnt[w][d] = run;
        run += c;
    }
    const uint32_t tcnt = run;
    const uint32_t texcl = block_excl_scan_256(tcnt, s_tmp, nullptr);
    const uint32_t gdig = block_excl_scan_256(hist[d], s_tmp, nullptr);
    s_texcl[d] = texcl;
    // the tile's digit counts go out first; the local sort runs while the
    // predecessors' counts arrive, then the look-back takes them
    lookback_publish(status + d, tile, 256u, epoch, tcnt);
    __syncthreads();

#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        if (wbase + j * 32 + lane < n) {
            const uint32_t dd = (k[j] >> shift) & 255u;
            const uint32_t lpos = s_texcl[dd] + s_wcnt[warp][dd] + r[j];
            s_keys[lpos] = k[j];
            s_vals[lpos] = v[j];
        }
    }
    const uint32_t back = lookback_resolve(status + d, tile, 256u, epoch, tcnt, err);
    s_gbase[d] = gdig + back;
    __syncthreads();
    const int64_t rem = n - base;
    const int tn = rem < kSortTile ? (int)rem : kSortTile;
    for (int i = tid; i < tn; i += kSortThreads) {
        const uint32_t key = s_keys[i];
        const uint32_t dd = (key >> shift) & 255u;
        const uint32_t dst = s_gbase[dd] + (uint32_t)(i - (int)s_texcl[dd]);
        if (dst < (uint64_t)n && KNN_IN_BOUNDS(i, 0, kSortTile, err)) {  // (a look-back timeout)
            kout[dst] = key;
            vout[dst] = s_vals[i];
        }
    }
}

// Sort (key[0], val[0]) of n entries; the result lands in buffer (passes & 1).
static void radix_sort(World &w, int64_t n, int passes, int counter_base, cudaStream_t s,
                       const int32_t *rebuild = nullptr) {
    if (n <= 0) return;
    const int tiles = (int)((n + kSortTile - 1) / kSortTile);
    for (int p = 0; p < passes; ++p) {
        const int src = p & 1, dst = src ^ 1;
        k_onesweep<<<tiles, kSortThreads, 0, s>>>(w.key[src], w.val[src], w.key[dst],
                                                   w.val[dst], n, 8 * p, w.hist + 256 * p,
                                                   w.status, w.counters + counter_base + p,
                                                   w.tickinfo, w.site++, w.err, rebuild);
        ++w.launches;
    }
}

void launch_object_sort(World &w, const Plan &p, cudaStream_t s) {
    // with index reuse on, the sort and the leaf split run only on rebuild ticks
    const int32_t *rebuild = p.reuse_age > 0 ? w.scalars + kScalarRebuild : nullptr;
    cudaMemsetAsync(w.hist, 0, sizeof(uint32_t) * 4 * 256, s);
    const bool vec4 = ((reinterpret_cast<uintptr_t>(w.px) | reinterpret_cast<uintptr_t>(w.py) |
                        reinterpret_cast<uintptr_t>(w.key[0]) |
                        reinterpret_cast<uintptr_t>(w.val[0])) & 15u) == 0;
    // two blocks per SM: the per-block histograms merge with few global atomics
    k_keys_hist<<<grid_for(vec4 ? (w.n + 3) / 4 : w.n, 256, num_sms(w.device) * 2), 256, 0, s>>>(
        w.px, w.py, w.n, w.desc.x0, w.desc.y0, w.scale, p.L, p.passes, w.key[0], w.val[0],
        w.hist, rebuild, vec4);
    ++w.launches;
    radix_sort(w, w.n, p.passes, kCtrObjSort, s, rebuild);
}

// ---------------------------------------------------------------------------
// a4 + a5 -- PR-quadtree leaves over the sorted keys, and the leaf-ordered SoA.
//
// The quadrant at level l holding sorted element i has more than th objects
// exactly when some run of th + 1 consecutive elements containing i shares the
// level-l prefix, i.e. when  W_i = max_{i-th <= j <= i} lcp(key_j, key_{j+th})
// is at least l.  So the leaf level of i is lambda_i = min(W_i + 1, L) (raised
// to the cell-map level G, below which every quadrant is split), and the leaf
// is the level-lambda_i quadrant holding key_i.  This is the same leaf set that
// the level-by-level splitting of Section 4.1.1 produces, computed in one pass.
// Leaves start where (lambda, code) changes; a look-back scan numbers them.

template <bool EMIT_EMPTY>
__global__ void __launch_bounds__(256) k_leaves(
    const uint32_t *__restrict__ skeys, const int32_t *__restrict__ svals, int64_t n, int L,
    int th, int G, const float *__restrict__ px, const float *__restrict__ py,
    float *__restrict__ xs, float *__restrict__ ys, int32_t *__restrict__ sid,
    int32_t *__restrict__ inv, int32_t *__restrict__ bstart, uint32_t *__restrict__ bcode,
    uint8_t *__restrict__ blevel, int32_t *__restrict__ obj_leaf, int32_t *__restrict__ cb,
    int64_t ncell, int32_t *scalars,
    uint64_t *status, uint32_t *ticket, const uint32_t *__restrict__ tickinfo, uint32_t site,
    uint32_t *err, bool guarded, int32_t sig, int64_t leaf_cap, bool write_inv) {
    constexpr bool emit_empty = EMIT_EMPTY;
    if (guarded && scalars[kScalarRebuild] == 0) return;  // this tick reuses the leaves
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_tile, s_tmp[8], s_excl;
    // long runs of cells without a leaf, filled by the whole block
    constexpr int kMaxGaps = 64;
    __shared__ int64_t s_gap_lo[kMaxGaps], s_gap_hi[kMaxGaps];
    __shared__ int32_t s_gap_b[kMaxGaps], s_gap_pos[kMaxGaps];
    __shared__ int s_ngap;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const int64_t t0 = (int64_t)tile * kLeafTile;
    const int B = th + 1;            // window length
    int S = 1;
    while (S * 2 <= B) S *= 2;       // largest power of two <= B
    const int nk = kLeafTile + 2 * th + 1;
    const int nw = kLeafTile + th + 1;
    const int64_t o = t0 - th - 1;   // global index of local slot 0

    uint32_t *s_key = reinterpret_cast<uint32_t *>(smem);
    int8_t *s_w0 = reinterpret_cast<int8_t *>(s_key + nk);
    int8_t *s_w1 = s_w0 + nw + S;
    int8_t *s_lam = s_w1 + nw + S;                          // kLeafTile + 1 entries
    uint32_t *s_code = reinterpret_cast<uint32_t *>(
        (reinterpret_cast<uintptr_t>(s_lam + kLeafTile + 1) + 3) & ~uintptr_t(3));

    for (int u = tid; u < nk; u += 256) {
        const int64_t j = o + u;
        s_key[u] = (j >= 0 && j < n) ? skeys[j] : 0u;
    }
    __syncthreads();
    for (int u = tid; u < nw + S; u += 256) {
        const int64_t j = o + u;
        int8_t wv = -1;
        if (u < nw && j >= 0 && j + th < n) wv = (int8_t)common_levels(s_key[u], s_key[u + th], L);
        s_w0[u] = wv;
        s_w1[u] = -1;
    }
    __syncthreads();
    // running maxima over power-of-two spans: after the loop src[u] = max w[u .. u+S-1]
    int8_t *src = s_w0, *dst = s_w1;
    for (int span = 1; span < S; span *= 2) {
        for (int u = tid; u < nw; u += 256) {
            const int8_t a = src[u], b = src[u + span];
            dst[u] = a > b ? a : b;
        }
        __syncthreads();
        int8_t *t = src;
        src = dst;
        dst = t;
    }
    // leaf level and code for elements t0-1 .. t0+kLeafTile-1
    for (int e = tid - 1; e < kLeafTile; e += 256) {
        const int64_t i = t0 + e;
        int lam = 0;
        uint32_t code = 0;
        if (i >= 0 && i < n) {
            const int u = e + th + 1;
            const int8_t a = src[u - th], b = src[u + 1 - S];
            const int W = a > b ? a : b;
            lam = W + 1 < L ? W + 1 : L;
            if (lam < G) lam = G;
            code = (uint32_t)((uint64_t)s_key[e + th + 1] >> (2 * (L - lam)));
        }
        s_lam[e + 1] = (int8_t)lam;
        s_code[e + 1] = code;
    }
    __syncthreads();
    // flags: 4 consecutive elements per thread.  With emit_empty (index reuse)
    // every level-G cell without objects also gets a leaf, empty, at level G,
    // so that any object of a later tick finds a leaf in its cell; an element
    // that starts a leaf then counts the empty cells just before its own.
    auto gcell = [&](int e1) -> int64_t {  // level-G cell of local element e1 - 1
        return (int64_t)(s_code[e1] >> (2 * (s_lam[e1] - G)));
    };
    uint32_t fl = 0, cnt = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int e = tid * 4 + q;
        const int64_t i = t0 + e;
        bool f = false;
        uint32_t wgt = 0;
        if (i < n) {
            f = (i == 0) || s_lam[e + 1] != s_lam[e] || s_code[e + 1] != s_code[e];
            if (f) {
                wgt = 1;
                if (emit_empty) {
                    const int64_t gap = gcell(e + 1) - (i == 0 ? -1 : gcell(e)) - 1;
                    wgt += gap > 0 ? (uint32_t)gap : 0u;
                }
            }
        }
        fl |= (f ? 1u : 0u) << q;
        cnt += wgt;
    }
    uint32_t tile_total;
    __shared__ uint32_t s_total;
    if (tid == 0) s_ngap = 0;
    const uint32_t off = block_excl_scan_256(cnt, s_tmp, &s_total);
    tile_total = s_total;
    if (tid < 32) lookback_warp_publish(status, tile, tickinfo[0] + site, tile_total);
    // leaf-ordered SoA (a5): needs no leaf numbers, so it runs while the
    // predecessors' leaf counts arrive
    for (int e = tid; e < kLeafTile; e += 256) {
        const int64_t i = t0 + e;
        if (i >= n) break;
        int32_t id = svals[i];
        if (id < 0 || id >= n) id = 0;  // only after a timed-out look-back
        xs[i] = px[id];
        ys[i] = py[id];
        sid[i] = id;
        // the inverse order (a scatter to random places) only where the
        // queries are counted by place
        if (write_inv) inv[id] = (int32_t)i;
    }
    if (tid < 32) {
        const uint32_t ex =
            lookback_warp_resolve(status, tile, tickinfo[0] + site, tile_total, err);
        if (tid == 0) s_excl = ex;
    }
    __syncthreads();
    const uint32_t excl = s_excl;
    uint32_t b = excl + off;
    const uint32_t gsh = 2u * (uint32_t)(L - G);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t iq = t0 + tid * 4 + q;
        if (!(fl & (1u << q))) {
            if (iq < n) obj_leaf[iq] = (int32_t)(b - 1u);
            continue;
        }
        const int e = tid * 4 + q;
        const int lam = s_lam[e + 1];
        // cell map (the paper's z_map at level G): cb[c] is the first leaf of cell c
        int64_t c_here = gcell(e + 1);
        if (c_here > ncell) c_here = ncell;
        const int64_t c_prev = iq == 0 ? -1 : gcell(e);
        if (emit_empty && c_here - c_prev > 1) {
            // one empty leaf for each cell strictly between the two
            const int64_t lo = c_prev + 1, hi = c_here - 1;
            int slot = -1;
            if (hi - lo >= 64) {
                slot = atomicAdd(&s_ngap, 1);
                if (slot < kMaxGaps) {
                    s_gap_lo[slot] = lo;
                    s_gap_hi[slot] = hi;
                    s_gap_b[slot] = (int32_t)b;
                    s_gap_pos[slot] = (int32_t)iq;
                }
            }
            if (slot < 0 || slot >= kMaxGaps) {
                for (int64_t c = lo; c <= hi; ++c) {
                    const uint32_t bb = b + (uint32_t)(c - lo);
                    if (bb < (uint64_t)leaf_cap) {
                        bstart[bb] = (int32_t)iq;
                        bcode[bb] = (uint32_t)c << gsh;
                        blevel[bb] = (uint8_t)G;
                        cb[c] = (int32_t)bb;
                    }
                }
            }
            b += (uint32_t)(hi - lo + 1);
        }
        if (iq < n) obj_leaf[iq] = (int32_t)b;
        if (b < (uint64_t)leaf_cap) {
            bstart[b] = (int32_t)iq;
            bcode[b] = (uint32_t)((uint64_t)s_code[e + 1] << (2 * (L - lam)));
            blevel[b] = (uint8_t)lam;
            if (emit_empty) {
                if (c_here != c_prev) cb[c_here] = (int32_t)b;
            } else {
                // the cells from just after the previous leaf's cell up to
                // this leaf's cell start at leaf b
                int slot = -1;
                if (c_here - c_prev > 64) {
                    slot = atomicAdd(&s_ngap, 1);
                    if (slot < kMaxGaps) {
                        s_gap_lo[slot] = c_prev + 1;
                        s_gap_hi[slot] = c_here;
                        s_gap_b[slot] = (int32_t)b;
                        s_gap_pos[slot] = -1;
                    }
                }
                if (slot < 0 || slot >= kMaxGaps)
                    for (int64_t c = c_prev + 1; c <= c_here; ++c) cb[c] = (int32_t)b;
            }
        }
        ++b;
    }
    if (t0 + kLeafTile >= n) {
        // cells after the last object's cell: no leaf (they start at leaf m),
        // or one empty leaf each
        const int e = (int)(n - 1 - t0);
        const int64_t c_last = gcell(e + 1);
        const int64_t trail = emit_empty && c_last + 1 < ncell ? ncell - 1 - c_last : 0;
        const uint64_t m_obj = (uint64_t)excl + tile_total;
        uint64_t m = m_obj + (uint64_t)trail;
        m = m <= (uint64_t)leaf_cap ? m : (uint64_t)leaf_cap;
        if (tid == 0) {
            scalars[kScalarLeaves] = (int32_t)m;
            scalars[kScalarIndexSig] = sig;
            bstart[m] = (int32_t)n;
        }
        for (int64_t c = c_last + 1 + tid; c <= ncell; c += 256) {
            if (c == ncell || !emit_empty) {
                cb[c] = (int32_t)(c == ncell ? m : m_obj);
            } else {
                const uint64_t bb = m_obj + (uint64_t)(c - c_last - 1);
                if (bb < (uint64_t)leaf_cap) {
                    bstart[bb] = (int32_t)n;
                    bcode[bb] = (uint32_t)c << gsh;
                    blevel[bb] = (uint8_t)G;
                    cb[c] = (int32_t)bb;
                }
            }
        }
    }
    __syncthreads();
    const int ngap = s_ngap < kMaxGaps ? s_ngap : kMaxGaps;
    for (int gi = 0; gi < ngap; ++gi) {
        const int64_t lo = s_gap_lo[gi], hi = s_gap_hi[gi];
        const int32_t b0 = s_gap_b[gi], pos = s_gap_pos[gi];
        for (int64_t c = lo + tid; c <= hi; c += 256) {
            if (pos < 0) {
                cb[c] = b0;
            } else {
                const int64_t bb = b0 + (c - lo);
                if (bb < leaf_cap) {
                    bstart[bb] = pos;
                    bcode[bb] = (uint32_t)c << gsh;
                    blevel[bb] = (uint8_t)G;
                    cb[c] = (int32_t)bb;
                }
            }
        }
    }
}

static size_t leaves_smem(int th) {
    const int nk = kLeafTile + 2 * th + 1;
    int S = 1;
    while (S * 2 <= th + 1) S *= 2;
    const int nw = kLeafTile + th + 1;
    size_t bytes = (size_t)nk * 4 + 2 * (size_t)(nw + S) + kLeafTile + 1 + 4;
    bytes = (bytes + 3) & ~size_t(3);
    bytes += (size_t)(kLeafTile + 1) * 4;
    return bytes;
}

// Tight bounding box of every leaf's members (used as conservative lower
// bounds of member distances by the expansion).
// Also sums the squared leaf counts (the cost proxy of index reuse).
__global__ void k_leaf_aabb(const int32_t *__restrict__ bstart, int32_t *scalars,
                            const float *__restrict__ xs, const float *__restrict__ ys,
                            float4 *__restrict__ baabb, int2 *__restrict__ brange, int64_t n) {
    const int32_t m = scalars[kScalarLeaves];
    unsigned long long cost = 0;
    for (int32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < m; b += gridDim.x * blockDim.x) {
        const int32_t s = bstart[b], e = bstart[b + 1];
        if (s < 0 || e <= s || e > n) {  // empty (only a reused leaf can be)
            baabb[b] = make_float4(0.f, 0.f, -1.f, -1.f);
            brange[b] = make_int2(0, 0);
            continue;
        }
        cost += (unsigned long long)(e - s) * (unsigned long long)(e - s);
        brange[b] = make_int2(s, e);
        float x0 = xs[s], x1 = x0, y0 = ys[s], y1 = y0;
        for (int32_t i = s + 1; i < e; ++i) {
            const float x = xs[i], y = ys[i];
            x0 = fminf(x0, x);
            x1 = fmaxf(x1, x);
            y0 = fminf(y0, y);
            y1 = fmaxf(y1, y);
        }
        baabb[b] = make_float4(x0, y0, x1, y1);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cost += __shfl_xor_sync(kFull, cost, o);
    if ((threadIdx.x & 31) == 0 && cost)
        atomicAdd(reinterpret_cast<unsigned long long *>(scalars + kScalarCostNow), cost);
}

void launch_leaves(World &w, const Plan &p, cudaStream_t s) {
    const int r = p.passes & 1;
    const int tiles = (int)((w.n + kLeafTile - 1) / kLeafTile);
    const size_t sm = leaves_smem(p.th);
    prepare_kernels();
    const int64_t ncell = 1ll << (2 * p.G);
    // with index reuse on, empty level-G cells get empty leaves
    auto leaves = p.reuse_age > 0 ? k_leaves<true> : k_leaves<false>;
    leaves<<<tiles, 256, sm, s>>>(w.key[r], w.val[r], w.n, p.L, p.th, p.G, w.px, w.py, w.xs, w.ys,
                                  w.sid, w.inv, w.bstart, w.bcode, w.blevel, w.obj_leaf, w.cb,
                                  ncell, w.scalars, w.status, w.counters + kCtrLeaves, w.tickinfo,
                                  w.site++, w.err, p.reuse_age > 0, index_signature(p),
                                  w.leaf_cap, !p.by_id);
    const int g = grid_for(w.n, 256, num_sms(w.device) * 8);
    k_leaf_aabb<<<g, 256, 0, s>>>(w.bstart, w.scalars, w.xs, w.ys, w.baabb, w.brange, w.n);
    w.launches += 2;
}

// ---------------------------------------------------------------------------
// Exclusive scan of int32 (single pass, look-back).  In place is allowed.

// GATHER: the value of entry c is in[idx[c]] (0 for the last entry);
// otherwise it is in[c].
template <bool GATHER>
__global__ void __launch_bounds__(256) k_scan_excl(const int32_t *in, const int32_t *idx,
                                                   int32_t *out, int64_t len,
                                                   int32_t *total, uint64_t *status,
                                                   uint32_t *ticket,
                                                   const uint32_t *__restrict__ tickinfo,
                                                   uint32_t site, uint32_t *err,
                                                   const int32_t *skip_if, int skip_on_zero,
                                                   const int32_t *len_minus_1) {
    // the same for every block of the launch
    if (skip_if && (*skip_if != 0) != (skip_on_zero != 0)) return;
    if (len_minus_1) {  // the length is known on the device only: *len_minus_1 + 1 <= len
        const int64_t l = (int64_t)*len_minus_1 + 1;
        len = l < len ? (l > 0 ? l : 0) : len;
    }
    __shared__ uint32_t s_tile, s_tmp[8], s_total, s_excl;
    const int tid = threadIdx.x;
    if (tid == 0) s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    // tiles past the end: nothing waits on them
    if ((int64_t)tile * kScanTile >= len && tile > 0) return;
    const int64_t base = (int64_t)tile * kScanTile + tid * 8;
    // 8 consecutive entries per thread, read as two 16-byte words when whole
    // (the buffers are 256-byte aligned and base is a multiple of 8)
    const bool whole = base + 8 <= len;
    int32_t v[8];
    if (GATHER) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int32_t t = base + q + 1 < len ? idx[base + q] : -1;
            v[q] = t >= 0 && t < len - 1 ? in[t] : 0;
        }
    } else if (whole) {
        const int4 a = *reinterpret_cast<const int4 *>(in + base);
        const int4 b = *reinterpret_cast<const int4 *>(in + base + 4);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = base + q < len ? in[base + q] : 0;
    }
    uint32_t sum = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) sum += (uint32_t)v[q];
    const uint32_t off = block_excl_scan_256(sum, s_tmp, &s_total);
    if (tid < 32) {
        const uint32_t ex = lookback_warp(status, tile, tickinfo[0] + site, s_total, err);
        if (tid == 0) s_excl = ex;
    }
    __syncthreads();
    uint32_t run = s_excl + off;
    int32_t o[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        o[q] = (int32_t)run;
        run += (uint32_t)v[q];
    }
    if (whole) {
        *reinterpret_cast<int4 *>(out + base) = make_int4(o[0], o[1], o[2], o[3]);
        *reinterpret_cast<int4 *>(out + base + 4) = make_int4(o[4], o[5], o[6], o[7]);
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (base + q < len) out[base + q] = o[q];
    }
    if ((int64_t)(tile + 1) * kScanTile >= len && tid == 255 && total) *total = (int32_t)run;
}

// skip_if: when non-null and nonzero on the device (zero, with skip_on_zero),
// the launch does nothing.
// len_minus_1: when non-null, the device value + 1 (at most len) is the length.
// gather_idx: when non-null, entry c is in[gather_idx[c]] (and the last entry 0).
static void scan_excl(World &w, const int32_t *in, int32_t *out, int64_t len, int32_t *total,
                      int counter, cudaStream_t s, const int32_t *gather_idx = nullptr,
                      const int32_t *skip_if = nullptr, const int32_t *len_minus_1 = nullptr,
                      bool skip_on_zero = false) {
    const int tiles = (int)((len + kScanTile - 1) / kScanTile);
    if (gather_idx)
        k_scan_excl<true><<<tiles, 256, 0, s>>>(in, gather_idx, out, len, total, w.status,
                                                w.counters + counter, w.tickinfo, w.site++,
                                                w.err, skip_if, skip_on_zero, len_minus_1);
    else
        k_scan_excl<false><<<tiles, 256, 0, s>>>(in, nullptr, out, len, total, w.status,
                                                 w.counters + counter, w.tickinfo, w.site++,
                                                 w.err, skip_if, skip_on_zero, len_minus_1);
    ++w.launches;
}

// ---------------------------------------------------------------------------
// a6 -- query ordering (Section 4.2.1).  Queries centred at their issuers are
// ordered by the issuer's place in the sorted object order (a counting sort),
// which is the Morton order of their centres.

// Two counting sorts order the queries by their issuers' places p in the
// sorted object order.  When most objects query (n_q >= n / 2) the queries are
// counted by issuer id: the counting is then coalesced, an issuer with a
// single query passes that query's index along with its count, and only
// issuers with several queries need the rank placement.  With few queries the
// per-object arrays would cost more than the queries, so they are counted by
// place instead (the issuer's place found through the inverse order).

// By place, first half: every valid query counts one more query at its
// issuer's sorted place p and keeps p and its rank among the queries of that
// issuer (the count before its own).
__global__ void k_query_count(const int32_t *__restrict__ q_id, int64_t n_q, int64_t n,
                              const int32_t *__restrict__ inv, int32_t *qcnt, int k,
                              int32_t *out_ids, float *out_d2, uint32_t *err,
                              int32_t *__restrict__ qp, int32_t *__restrict__ qrank) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_q;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = q_id[i];
        if (s < 0 || s >= n) {
            atomicOr(err, kErrBadQuery);
            qp[i] = -1;
            for (int r = 0; r < k; ++r) {
                out_ids[i * k + r] = -1;
                out_d2[i * k + r] = __int_as_float(0x7f800000);
            }
            continue;
        }
        const int32_t p = inv[s];
        qp[i] = p;
        qrank[i] = atomicAdd(&qcnt[p], 1);
    }
}

// By place, second half: every valid query takes the slot of its rank in its
// issuer's range [qoff[p], qoff[p+1]) and records its caller index there.
__global__ void k_query_place(int64_t n_q, int64_t n, const int32_t *__restrict__ qp,
                              const int32_t *__restrict__ qrank,
                              const int32_t *__restrict__ qoff, int32_t *qs_orig) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_q;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = qp[i];
        if (p < 0 || p >= n) continue;
        const int32_t j = qoff[p] + qrank[i];
        if (j < 0 || j >= n_q) continue;  // only after a timed-out look-back
        qs_orig[j] = (int32_t)i;
    }
}

// By issuer id, first half: every valid query counts one more query at its
// issuer and keeps its rank among that issuer's queries and, in qidx[issuer],
// its own index (the only one there when the issuer has a single query).  A
// second query at one issuer sets bit 0 of qcnt[n], which makes
// k_query_place_id run; an invalid issuer sets bit 1.  With as many queries as
// objects, qcnt[n] == 0 means one query per object: the query offsets are the
// identity and their scan is skipped.
__global__ void k_query_count_id(const int32_t *__restrict__ q_id, int64_t n_q, int64_t n,
                                 int32_t *qcnt, int k, int32_t *out_ids, float *out_d2,
                                 uint32_t *err, int32_t *__restrict__ qrank,
                                 int32_t *__restrict__ qidx) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_q;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = q_id[i];
        if (s < 0 || s >= n) {
            atomicOr(err, kErrBadQuery);
            atomicOr(&qcnt[n], 2);
            for (int r = 0; r < k; ++r) {
                out_ids[i * k + r] = -1;
                out_d2[i * k + r] = __int_as_float(0x7f800000);
            }
            continue;
        }
        const int32_t r = atomicAdd(&qcnt[s], 1);
        qrank[i] = r;
        qidx[s] = (int32_t)i;
        if (r == 1) atomicOr(&qcnt[n], 1);
    }
}

// By issuer id, rank placement, only when some issuer has several queries
// (qcnt[n] set): every query of such an issuer takes the slot of its rank in
// the range of the issuer's place p (which k_query_fill recorded in inv[issuer])
// and records its caller index there.
__global__ void k_query_place_id(const int32_t *__restrict__ q_id, int64_t n_q, int64_t n,
                                 const int32_t *__restrict__ inv,
                                 const int32_t *__restrict__ qrank,
                                 const int32_t *__restrict__ qoff,
                                 const int32_t *__restrict__ qcnt, int32_t *qs_orig) {
    if ((qcnt[n] & 1) == 0) return;  // the same for every block of the launch
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_q;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = q_id[i];
        if (s < 0 || s >= n || qcnt[s] < 2) continue;  // single queries are placed
        const int32_t p = inv[s];
        if (p < 0 || p >= n) continue;
        const int32_t j = qoff[p] + qrank[i];
        if (j < 0 || j >= n_q) continue;  // only after a timed-out look-back
        qs_orig[j] = (int32_t)i;
    }
}

// Walk the sorted objects in order and copy each one's position, id and key
// into the slots of its queries: sequential reads, sequential writes.  With
// qidx (counting by issuer id), an object with a single query also records
// that query's caller index, and one with several records its place in inv.
__global__ void k_query_fill(int64_t n, int64_t n_q, const int32_t *__restrict__ qoff,
                             const float *__restrict__ xs, const float *__restrict__ ys,
                             const int32_t *__restrict__ sid, const uint32_t *__restrict__ skey,
                             const int32_t *__restrict__ obj_leaf,
                             const int32_t *__restrict__ qidx, float *qs_x, float *qs_y,
                             int32_t *qs_id, uint32_t *qs_key, int32_t *qs_leaf,
                             int32_t *qs_orig, int32_t *inv, const int32_t *ident,
                             int32_t *scalars) {
    // one query per object (ident: the flag word of k_query_count_id, zero):
    // object p's query is slot p, the offsets were not scanned
    const bool identity = ident && *ident == 0;
    if (identity && blockIdx.x == 0 && threadIdx.x == 0) scalars[kScalarValidQueries] = (int32_t)n;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = identity ? (int32_t)p : qoff[p];
        int32_t b = identity ? (int32_t)p + 1 : qoff[p + 1];
        if (a >= b) continue;
        const bool single = b - a == 1;
        if (a < 0) a = 0;
        if (b > n_q) b = (int32_t)n_q;
        const float x = xs[p], y = ys[p];
        const int32_t id = sid[p];
        const uint32_t key = skey[p];
        const int32_t leaf = obj_leaf[p];
        for (int32_t j = a; j < b; ++j) {
            qs_x[j] = x;
            qs_y[j] = y;
            qs_id[j] = id;
            qs_key[j] = key;
            qs_leaf[j] = leaf;
        }
        if (qidx && id >= 0 && id < n) {
            if (single && a < b) qs_orig[a] = qidx[id];
            else if (!single) inv[id] = (int32_t)p;
        }
    }
}

void launch_queries_at_issuers(World &w, const Plan &p, const int32_t *q_id, int64_t n_q,
                               int32_t k, int32_t *out_ids, float *out_d2, cudaStream_t s) {
    // per-query and per-issuer scratch lives in the sort's second buffers, free
    // once the leaf-ordered store is written
    const int r = p.passes & 1;
    int32_t *aux = reinterpret_cast<int32_t *>(w.key[r ^ 1]), *qrank = w.val[r ^ 1];
    const bool by_id = p.by_id;
    cudaMemsetAsync(w.qcnt, 0, sizeof(int32_t) * (size_t)(w.n + 1), s);
    const int g = grid_for(n_q, 256, num_sms(w.device) * 8);
    const uint32_t *skey = w.key[p.passes & 1];
    const int gf = grid_for(w.n, 256, num_sms(w.device) * 8);
    if (by_id) {
        // aux: each issuer's last query
        k_query_count_id<<<g, 256, 0, s>>>(q_id, n_q, w.n, w.qcnt, k, out_ids, out_d2, w.err,
                                           qrank, aux);
        // counts taken in sorted-object order; with as many queries as
        // objects the scan is skipped when each object has exactly one
        const int32_t *ident = n_q == w.n ? w.qcnt + w.n : nullptr;
        scan_excl(w, w.qcnt, w.qoff, w.n + 1, w.scalars + kScalarValidQueries, kCtrQueryScan,
                  s, w.sid, ident, nullptr, true);
        k_query_fill<<<gf, 256, 0, s>>>(w.n, n_q, w.qoff, w.xs, w.ys, w.sid, skey, w.obj_leaf,
                                        aux, w.qs_x, w.qs_y, w.qs_id, w.qs_key, w.qs_leaf,
                                        w.qs_orig, w.inv, ident, w.scalars);
        k_query_place_id<<<g, 256, 0, s>>>(q_id, n_q, w.n, w.inv, qrank, w.qoff, w.qcnt,
                                           w.qs_orig);
    } else {
        // aux: each query's issuer place
        k_query_count<<<g, 256, 0, s>>>(q_id, n_q, w.n, w.inv, w.qcnt, k, out_ids, out_d2, w.err,
                                        aux, qrank);
        scan_excl(w, w.qcnt, w.qoff, w.n + 1, w.scalars + kScalarValidQueries, kCtrQueryScan,
                  s);
        k_query_place<<<g, 256, 0, s>>>(n_q, w.n, aux, qrank, w.qoff, w.qs_orig);
        k_query_fill<<<gf, 256, 0, s>>>(w.n, n_q, w.qoff, w.xs, w.ys, w.sid, skey, w.obj_leaf,
                                        nullptr, w.qs_x, w.qs_y, w.qs_id, w.qs_key, w.qs_leaf,
                                        w.qs_orig, w.inv, nullptr, w.scalars);
    }
    w.launches += 3;  // and one counted by scan_excl
}

// Leaf next to a level-L key in Morton order: the last leaf of the key's
// level-G cell whose first code is <= key, else the cell's first leaf, or the
// insertion point when the cell has no leaf.
__device__ __forceinline__ int32_t leaf_near(const int32_t *__restrict__ cb,
                                             const uint32_t *__restrict__ bcode, int L, int G,
                                             uint32_t key) {
    uint32_t c = key >> (2 * (L - G));
    const uint32_t last = (1u << (2 * G)) - 1u;
    c = c < last ? c : last;
    int32_t lo = cb[c], hi = cb[c + 1];
    if (lo == hi) return lo;
    const int32_t first = lo;
    while (lo < hi) {  // first leaf with code > key
        const int32_t mid = (lo + hi) >> 1;
        if (bcode[mid] <= key) lo = mid + 1;
        else hi = mid;
    }
    return lo > first ? lo - 1 : first;
}

__global__ void k_query_gather(const uint32_t *__restrict__ skey, const int32_t *__restrict__ sval,
                               int64_t n_q, const int32_t *__restrict__ q_id,
                               const float *__restrict__ q_x, const float *__restrict__ q_y,
                               float *qs_x, float *qs_y, int32_t *qs_id, int32_t *qs_orig,
                               uint32_t *qs_key, int32_t *scalars, const int32_t *__restrict__ cb,
                               const uint32_t *__restrict__ bcode, int L, int G,
                               int32_t *qs_leaf) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t == 0) scalars[kScalarValidQueries] = (int32_t)n_q;
    for (int64_t j = t; j < n_q; j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = sval[j];
        qs_key[j] = skey[j];
        qs_orig[j] = v;
        qs_leaf[j] = leaf_near(cb, bcode, L, G, skey[j]);
        if (v >= 0) {
            qs_x[j] = q_x[v];
            qs_y[j] = q_y[v];
            qs_id[j] = q_id[v];
        } else {
            qs_x[j] = 0.f;
            qs_y[j] = 0.f;
            qs_id[j] = -1;
        }
    }
}

void launch_queries_explicit(World &w, const Plan &p, const int32_t *q_id, const float *q_x,
                             const float *q_y, int64_t n_q, int32_t k, int32_t *out_ids,
                             float *out_d2, cudaStream_t s) {
    cudaMemsetAsync(w.hist, 0, sizeof(uint32_t) * 4 * 256, s);
    const int g = grid_for(n_q, 256, num_sms(w.device) * 4);
    k_query_keys_hist<<<g, 256, 0, s>>>(q_id, q_x, q_y, n_q, w.n, w.desc.x0, w.desc.y0, w.scale,
                                        p.L, p.passes, k, w.key[0], w.val[0], w.hist, out_ids,
                                        out_d2, w.err);
    radix_sort(w, n_q, p.passes, kCtrQuerySort, s);
    const int r = p.passes & 1;
    k_query_gather<<<grid_for(n_q, 256, num_sms(w.device) * 8), 256, 0, s>>>(
        w.key[r], w.val[r], n_q, q_id, q_x, q_y, w.qs_x, w.qs_y, w.qs_id, w.qs_orig, w.qs_key,
        w.scalars, w.cb, w.bcode, p.L, p.G, w.qs_leaf);
    w.launches += 2;
}

// ---------------------------------------------------------------------------
// Packets: at most 32 consecutive sorted queries inside one level-Gp cell,
// one packet per warp of the expansion (the paper's per-cell tasks).

// First sorted query of every level-Gp cell (qcs[c], c in [0, ncell]): each
// boundary between consecutive sorted queries fills the cells it crosses.
__global__ void k_query_cells(const uint32_t *__restrict__ qs_key, int32_t *scalars, int L,
                              int Gp, int64_t ncell, int64_t nq_cap, int32_t *qcs) {
    int32_t nv = scalars[kScalarValidQueries];
    if (nv < 0) nv = 0;
    if (nv > nq_cap) nv = (int32_t)nq_cap;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        scalars[kScalarPackets] = 0;
        scalars[kScalarPartialPackets] = 0;
        scalars[kScalarHandedBack] = 0;
    }
    const int sh = 2 * (L - Gp);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j <= nv;
         j += (int64_t)gridDim.x * blockDim.x) {
        int64_t c_here = j < nv ? (int64_t)((uint64_t)qs_key[j] >> sh) : ncell;
        if (c_here > ncell) c_here = ncell;
        const int64_t c_prev = j > 0 ? (int64_t)((uint64_t)qs_key[j - 1] >> sh) : -1;
        for (int64_t c = c_prev + 1; c <= c_here; ++c) qcs[c] = (int32_t)j;
    }
}

// Packets of a cell: its queries 32 at a time, the last one partial.  Full
// packets go to the front of the list and partial ones to the back (slots
// pk_cap - 1 down), so that a persistent expansion taking the full ones first
// ends on the cheaper partial ones.  Slots come from warp-aggregated atomic
// counters; the order of packets changes nothing in the rows.
__global__ void k_packets(const int32_t *__restrict__ qcs, int64_t ncell, int64_t pk_cap,
                          int32_t *scalars, int32_t *pk_start, int32_t *pk_len) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t start = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    // every lane of a warp runs the same number of rounds
    for (int64_t c0 = start - lane; c0 < ncell; c0 += stride) {
        const int64_t c = c0 + lane;
        int32_t s = 0, cnt = 0;
        if (c < ncell) {
            s = qcs[c];
            cnt = qcs[c + 1] - s;
            if (cnt < 0) cnt = 0;
        }
        const int32_t nfull = cnt >> 5;
        const bool part = (cnt & 31) != 0;
        int32_t inc = nfull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += y;
        }
        const unsigned pm = __ballot_sync(kFull, part);
        int32_t fbase = 0, pbase = 0;
        if (lane == 31 && inc > 0) fbase = atomicAdd(scalars + kScalarPackets, inc);
        if (lane == 0 && pm) pbase = atomicAdd(scalars + kScalarPartialPackets, __popc(pm));
        fbase = __shfl_sync(kFull, fbase, 31);
        pbase = __shfl_sync(kFull, pbase, 0);
        const int64_t f0 = (int64_t)fbase + inc - nfull;
        for (int32_t i = 0; i < nfull; ++i) {
            const int64_t o = f0 + i;
            if (o < pk_cap) {
                pk_start[o] = s + 32 * i;
                pk_len[o] = 32;
            }
        }
        if (part) {
            const int64_t o = pk_cap - 1 - ((int64_t)pbase + __popc(pm & ((1u << lane) - 1u)));
            if (o >= 0) {
                pk_start[o] = s + 32 * nfull;
                pk_len[o] = cnt & 31;
            }
        }
    }
}

void launch_query_cells(World &w, const Plan &p, int64_t n_q, cudaStream_t s) {
    const int64_t ncell = 1ll << (2 * p.Gp);
    k_query_cells<<<grid_for(n_q + 1, 256, num_sms(w.device) * 8), 256, 0, s>>>(
        w.qs_key, w.scalars, p.L, p.Gp, ncell, n_q, w.qcs);
    ++w.launches;
}

void launch_packets(World &w, const Plan &p, int64_t n_q, cudaStream_t s) {
    const int64_t ncell = 1ll << (2 * p.Gp);
    const int g = grid_for(ncell, 256, num_sms(w.device) * 16);
    launch_query_cells(w, p, n_q, s);
    k_packets<<<g, 256, 0, s>>>(w.qcs, ncell, packet_capacity(w), w.scalars, w.pk_start,
                                w.pk_len);
    ++w.launches;
}

// ---------------------------------------------------------------------------
// Index reuse (the paper's stage (i) skipped): on a tick that keeps the
// leaves, every object is put in a leaf of its level-G cell (the leaf whose
// code range holds its key, else the nearest one in Morton order; any leaf of
// the cell keeps the walk exact, since the walk reaches leaves through their
// cells and tests every leaf's box, recomputed each tick from its members),
// and a counting sort by leaf replaces the radix sort and the leaf split.
// While reuse is on, the leaf split gives every empty level-G cell an empty
// leaf, so an object always finds one; a cell without leaf (only if the plan
// changed underneath) makes the tick rebuild instead.

__global__ void k_reuse_assign(const float *__restrict__ px, const float *__restrict__ py,
                               int64_t n, float x0, float y0, float scale, int L, int G,
                               const int32_t *__restrict__ cb, const uint32_t *__restrict__ bcode,
                               int32_t *scalars, uint32_t *__restrict__ key_by_id,
                               int32_t *__restrict__ leaf_by_id, int32_t *lcnt) {
    if (scalars[kScalarRebuild] != 0) return;
    const int32_t m = scalars[kScalarLeaves];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t key = morton_key(px[i], py[i], x0, y0, scale, L);
        const uint32_t c = key >> (2 * (L - G));
        if (cb[c] >= cb[c + 1]) {  // no leaf in this cell: rebuild this tick
            atomicExch(scalars + kScalarRebuild, 1);
            return;
        }
        int32_t b = leaf_near(cb, bcode, L, G, key);
        b = b < 0 ? 0 : (b >= m ? m - 1 : b);
        key_by_id[i] = key;
        leaf_by_id[i] = b;
        atomicAdd(lcnt + b, 1);
    }
}

// Each object's place: the next free slot of its leaf (the order inside a
// leaf does not matter); perm[place] = object.
__global__ void k_reuse_rank(int64_t n, const int32_t *__restrict__ leaf_by_id,
                             const int32_t *__restrict__ bstart, int32_t *lcnt,
                             const int32_t *__restrict__ scalars, int32_t *__restrict__ perm,
                             int32_t *__restrict__ inv) {
    if (scalars[kScalarRebuild] != 0) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t b = leaf_by_id[i];
        int32_t pos = bstart[b] + atomicSub(lcnt + b, 1) - 1;  // leaves lcnt at 0
        pos = pos < 0 ? 0 : (pos >= n ? (int32_t)(n - 1) : pos);  // only after a timeout
        perm[pos] = (int32_t)i;
        inv[i] = pos;
    }
}

// The leaf-ordered store, gathered in place order (coalesced writes).
__global__ void k_reuse_gather(const float *__restrict__ px, const float *__restrict__ py,
                               int64_t n, const uint32_t *__restrict__ key_by_id,
                               const int32_t *__restrict__ leaf_by_id,
                               const int32_t *__restrict__ perm,
                               const int32_t *__restrict__ scalars, float *__restrict__ xs,
                               float *__restrict__ ys, int32_t *__restrict__ sid,
                               int32_t *__restrict__ obj_leaf, uint32_t *__restrict__ skey) {
    if (scalars[kScalarRebuild] != 0) return;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        int32_t i = perm[p];
        i = i < 0 || i >= n ? 0 : i;
        xs[p] = px[i];
        ys[p] = py[i];
        sid[p] = i;
        obj_leaf[p] = leaf_by_id[i];
        skey[p] = key_by_id[i];
    }
}

void launch_index_reuse(World &w, const Plan &p, cudaStream_t s) {
    // the sorted keys and the place order land where the radix sort leaves its
    // keys and ids; the other key and value buffers hold each object's key and
    // leaf meanwhile
    const int r = p.passes & 1;
    int32_t *lcnt = w.lcnt;
    // leaves: the objects' ones plus at most one empty leaf per level-G cell
    int64_t len = w.n + (1ll << (2 * p.G)) + 1;
    len = len < w.leaf_cap + 1 ? len : w.leaf_cap + 1;
    const int g = grid_for(w.n, 256, num_sms(w.device) * 8);
    cudaMemsetAsync(lcnt, 0, sizeof(int32_t) * (size_t)len, s);
    k_reuse_assign<<<g, 256, 0, s>>>(w.px, w.py, w.n, w.desc.x0, w.desc.y0, w.scale, p.L, p.G,
                                     w.cb, w.bcode, w.scalars, w.key[r ^ 1], w.val[r ^ 1], lcnt);
    scan_excl(w, lcnt, w.bstart, len, nullptr, kCtrReuseScan, s, nullptr,
              w.scalars + kScalarRebuild, w.scalars + kScalarLeaves);
    k_reuse_rank<<<g, 256, 0, s>>>(w.n, w.val[r ^ 1], w.bstart, lcnt, w.scalars, w.val[r],
                                   w.inv);
    k_reuse_gather<<<g, 256, 0, s>>>(w.px, w.py, w.n, w.key[r ^ 1], w.val[r ^ 1], w.val[r],
                                     w.scalars, w.xs, w.ys, w.sid, w.obj_leaf, w.key[r]);
    w.launches += 3;
}

void prepare_kernels() {
    static bool done[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || done[dev]) return;
    cudaFuncSetAttribute(k_leaves<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)leaves_smem(kMaxLeafCapacity));
    cudaFuncSetAttribute(k_leaves<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)leaves_smem(kMaxLeafCapacity));
    num_sms(dev);          // fill the per-device caches now: the query APIs
    prepare_expand(dev);   // must not run while a batch is being recorded
    prepare_expand_wide(dev);
    prepare_expand_gather(dev);
    prepare_expand_tile(dev);
    done[dev] = true;
}

int num_sms(int device) {
    static int cached[64] = {0};
    if (device < 0 || device >= 64) device = 0;
    if (!cached[device]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
        cached[device] = v > 0 ? v : 1;
    }
    return cached[device];
}

}  // namespace knnq

namespace knnq {

// Leaves of the last tick in the exported layout (level, own-level code,
// start, count) and the sorted object order.
__global__ void k_export_leaves(const int32_t *__restrict__ bstart,
                                const uint32_t *__restrict__ bcode,
                                const uint8_t *__restrict__ blevel, int64_t m, int L,
                                int32_t *level, uint32_t *z, int32_t *start, int32_t *count) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < m;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int lv = blevel[b];
        level[b] = lv;
        z[b] = (uint32_t)((uint64_t)bcode[b] >> (2 * (L - lv)));
        start[b] = bstart[b];
        count[b] = bstart[b + 1] - bstart[b];
    }
}

// Failure detection without a fault: one warp resolves the look-back of tile 1
// of a chain whose tile 0 never publishes -- its status word carries an older
// epoch than the one asked for (epochs advance by 64 per tick from 0, so
// 2^30 - 1 is never reached) -- and so waits exactly as a stalled tick's
// look-back would, until the poll limit (or the tick's abort flag): then the
// timeout bit and the abort flag are raised and the kernel returns.
__global__ void k_wait_runs_out(uint64_t *status, uint32_t *err) {
    lookback_warp_resolve(status, 1u, 0x3FFFFFFFu, 0u, err);
}

// Debug builds: evaluates one bounds check that fails (index n of an array of
// n objects); the check records the failure and the access is skipped.
// (A regular build compiles an empty body: there the check is the constant true.)
__global__ void k_bounds_check_probe(int64_t n, const float *xs, float *sink, uint32_t *err) {
#ifdef KNN_DEBUG
    if (threadIdx.x == 0 && blockIdx.x == 0 && KNN_IN_BOUNDS(n, 0, n, err)) sink[0] = xs[n];
#endif
}

void launch_bounds_check_probe(World &w, cudaStream_t s) {
    k_bounds_check_probe<<<1, 32, 0, s>>>(w.n, w.xs, w.xs, w.err);
    ++w.launches;
}

void launch_wait_runs_out(World &w, cudaStream_t s) {
    k_wait_runs_out<<<1, 32, 0, s>>>(w.status, w.err);
}

void launch_export_leaves(World &w, int64_t m, int32_t *level, uint32_t *z, int32_t *start,
                          int32_t *count, cudaStream_t s) {
    if (m <= 0) return;
    k_export_leaves<<<grid_for(m, 256, 4096), 256, 0, s>>>(w.bstart, w.bcode, w.blevel, m, w.L,
                                                          level, z, start, count);
}

}  // namespace knnq
