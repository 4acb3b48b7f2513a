// Device-side helpers shared by the index and expansion kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace knnq {

constexpr unsigned kFull = 0xFFFFFFFFu;

// Error bits recorded in the world's device error word.
enum : uint32_t {
    kErrBadUpdateId = 1u << 0,
    kErrNonFiniteUpdate = 1u << 1,
    kErrBadQuery = 1u << 2,
    kErrTimeout = 1u << 3,
    kErrDebugBounds = 1u << 4,  // a bounds check of a KNN_DEBUG build failed
};

// Device bounds checks of a debug build (compiled with -DKNN_DEBUG): an index
// outside [lo, hi) raises kErrDebugBounds in the error word and the access is
// skipped; nothing traps.  In a regular build the check is the constant true
// and costs nothing.  Use as: if (KNN_IN_BOUNDS(i, 0, n, err)) { access i }.
#ifdef KNN_DEBUG
__device__ __forceinline__ bool knn_in_bounds(int64_t i, int64_t lo, int64_t hi, uint32_t *err) {
    if (i >= lo && i < hi) return true;
    atomicOr(err, kErrDebugBounds);
    return false;
}
#define KNN_IN_BOUNDS(i, lo, hi, err) \
    knnq::knn_in_bounds((int64_t)(i), (int64_t)(lo), (int64_t)(hi), (err))
#else
#define KNN_IN_BOUNDS(i, lo, hi, err) true
#endif

// Bounded spins: a wait gives up after this many polls (each poll after the
// first few sleeps ~0.1-1 us), records kErrTimeout and continues; once the
// timeout bit is set every other wait gives up within 64 polls, so a broken
// tick ends in milliseconds.  Results are then invalid (the status says so)
// but every index stays clamped to its buffer.
constexpr uint32_t kSpinLimit = 1u << 16;

// ---------------------------------------------------------------------------
// Morton codes (Section 4.1.1): the level-L cell of a coordinate is
// floor((v - v0) * scale) with scale = 2^L / side, clamped to [0, 2^L - 1];
// x goes to the even bits, y to the odd bits.  Every operation is rounded on
// its own (the _rn intrinsics are never contracted).
__device__ __forceinline__ uint32_t cell_coord(float v, float v0, float scale, int L) {
    float t = __fmul_rn(__fsub_rn(v, v0), scale);
    float lim = (float)(1u << L);
    if (!(t >= 0.0f)) return 0u;
    if (t >= lim) return (1u << L) - 1u;
    return (uint32_t)t;
}

__device__ __forceinline__ uint32_t spread_bits(uint32_t v) {
    v &= 0xFFFFu;
    v = (v | (v << 8)) & 0x00FF00FFu;
    v = (v | (v << 4)) & 0x0F0F0F0Fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

__device__ __forceinline__ uint32_t interleave(uint32_t cx, uint32_t cy) {
    return spread_bits(cx) | (spread_bits(cy) << 1);
}

__device__ __forceinline__ uint32_t morton_key(float x, float y, float x0, float y0,
                                               float scale, int L) {
    return interleave(cell_coord(x, x0, scale, L), cell_coord(y, y0, scale, L));
}

// Number of leading 2-bit digits (quadtree levels) shared by two level-L codes.
__device__ __forceinline__ int common_levels(uint32_t a, uint32_t b, int L) {
    uint32_t d = a ^ b;
    if (d == 0u) return L;
    return (__clz(d) - (32 - 2 * L)) >> 1;
}

// ---------------------------------------------------------------------------
// Expansion helpers (Sections 4.2.1-4.2.2), shared by the packet kernel and
// the warp-per-query kernel for large k.

// key = (float bits of d^2) << 32 | (id + 1): for d >= 0 the unsigned order of
// keys is the lexicographic (d^2, id) order.  kPad (+inf, 0xFFFFFFFF) is above
// every real key and marks an empty slot; 0 is below every real key.
constexpr unsigned long long kPad = 0x7f800000FFFFFFFFull;

__device__ __forceinline__ int32_t key_id(unsigned long long key) {
    const uint32_t lo = (uint32_t)key;
    return lo == 0xFFFFFFFFu ? -1 : (int32_t)lo - 1;
}

// Sorted register lists of keys are merged with batches of kBatch keys by
// sorting networks (all lanes of a warp run the same compare-exchanges).
constexpr int kBatch = 8;

__device__ __forceinline__ void cmpx(unsigned long long &x, unsigned long long &y) {
    const bool s = y < x;
    const unsigned long long lo = s ? y : x;
    y = s ? x : y;
    x = lo;
}

// Sort 8 keys ascending (19 comparators, depth 6).
__device__ __forceinline__ void sort8(unsigned long long (&b)[kBatch]) {
    cmpx(b[0], b[2]); cmpx(b[1], b[3]); cmpx(b[4], b[6]); cmpx(b[5], b[7]);
    cmpx(b[0], b[4]); cmpx(b[1], b[5]); cmpx(b[2], b[6]); cmpx(b[3], b[7]);
    cmpx(b[0], b[1]); cmpx(b[2], b[3]); cmpx(b[4], b[5]); cmpx(b[6], b[7]);
    cmpx(b[2], b[4]); cmpx(b[3], b[5]);
    cmpx(b[1], b[4]); cmpx(b[3], b[6]);
    cmpx(b[1], b[2]); cmpx(b[3], b[4]); cmpx(b[5], b[6]);
}

// a (KC keys, ascending) := the KC smallest of a and b (8 keys, ascending):
// c_i = min(a_i, b_{KC-1-i}) is bitonic and holds them; a bitonic merger sorts it.
template <int KC>
__device__ __forceinline__ void merge_batch(unsigned long long (&a)[KC],
                                            const unsigned long long (&b)[kBatch]) {
#pragma unroll
    for (int i = (KC > kBatch ? KC - kBatch : 0); i < KC; ++i) {
        const unsigned long long v = b[KC - 1 - i];
        a[i] = v < a[i] ? v : a[i];
    }
#pragma unroll
    for (int span = KC / 2; span >= 1; span >>= 1) {
#pragma unroll
        for (int i = 0; i < KC; ++i)
            if ((i & span) == 0) cmpx(a[i], a[i + span]);
    }
}

// Two binary32 operations at once (sm_100 packed pairs): each half is rounded
// to nearest on its own, like the scalar operation.
__device__ __forceinline__ unsigned long long f2sub(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f2mul(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f2pack(float lo, float hi) {
    return ((unsigned long long)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}

// Level-G cell of a coordinate, with the same monotone rounding as the keys.
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
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Squared distance from (x, y) up to a box [x0, x1] x [y0, y1]: a lower bound
// of the squared distance to every point of the box, in the same rounding as
// the exact distances (round-to-nearest is monotone, so a point farther out
// never gets a smaller bound).
__device__ __forceinline__ float box_lb(float x0, float y0, float x1, float y1, float qx0,
                                        float qy0, float qx1, float qy1) {
    float dx = 0.f, dy = 0.f;
    if (qx1 < x0) dx = __fsub_rn(x0, qx1);
    else if (qx0 > x1) dx = __fsub_rn(qx0, x1);
    if (qy1 < y0) dy = __fsub_rn(y0, qy1);
    else if (qy0 > y1) dy = __fsub_rn(qy0, y1);
    return __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
}

// Ring of the level-G cells around a centre cell: ring 0 is the centre, ring
// r >= 1 the 8r cells at Chebyshev distance r.  Taking the rings in order and
// each ring in a fixed order numbers the cells: ring r >= 1 holds numbers
// 1 + 4r(r-1) .. 4r(r+1).  ring_of inverts that.
__device__ __forceinline__ int ring_of(int u) {
    if (u <= 0) return 0;
    int r = (int)(0.5f * (1.0f + sqrtf((float)u)));
    while (1 + 4 * r * (r + 1) <= u) ++r;
    while (r > 0 && 1 + 4 * r * (r - 1) > u) --r;
    return r;
}

// Cell (cx, cy) number u lies on, around the centre (ccx, ccy); r = ring_of(u).
// Ring r: the bottom row, the top row, then the left and right columns.
__device__ __forceinline__ void ring_cell(int u, int r, int ccx, int ccy, int &cx, int &cy) {
    const int t = r == 0 ? 0 : u - (1 + 4 * r * (r - 1));
    if (r == 0) { cx = ccx; cy = ccy; }
    else if (t < 2 * r + 1) { cx = ccx - r + t; cy = ccy - r; }
    else if (t < 4 * r + 2) { cx = ccx - r + (t - 2 * r - 1); cy = ccy + r; }
    else if (t < 6 * r + 1) { cx = ccx - r; cy = ccy - r + 1 + (t - 4 * r - 2); }
    else { cx = ccx + r; cy = ccy - r + 1 + (t - 6 * r - 1); }
}

// ---------------------------------------------------------------------------
// Decoupled look-back (single pass scans).  A status word packs
// [63:34] epoch (30 bits) | [33:32] flag | [31:0] value.  Every launch uses a
// fresh epoch (the tick's device-side epoch base plus the launch's index in
// the tick).  A world's status array is cleared once when its scratch is
// attached and sits at a fixed place afterwards, so words left by earlier
// launches carry older epochs and read as "not ready" without clearing (the
// 30-bit epoch repeats only after 2^24 ticks).  The allocation-free call, whose
// status words move with its sizes, clears them on every call.
constexpr uint32_t kFlagAgg = 1u, kFlagPrefix = 2u;

__device__ __forceinline__ uint64_t pack_status(uint32_t epoch, uint32_t flag, uint32_t v) {
    return ((uint64_t)(epoch & 0x3FFFFFFFu) << 34) | ((uint64_t)flag << 32) | (uint64_t)v;
}
__device__ __forceinline__ bool status_ready(uint64_t s, uint32_t epoch) {
    return (uint32_t)(s >> 34) == (epoch & 0x3FFFFFFFu) && ((s >> 32) & 3u) != 0u;
}
__device__ __forceinline__ uint32_t status_flag(uint64_t s) { return (uint32_t)(s >> 32) & 3u; }
__device__ __forceinline__ uint32_t status_value(uint64_t s) { return (uint32_t)s; }

__device__ __forceinline__ void st_status(uint64_t *p, uint64_t v) {
    *reinterpret_cast<volatile uint64_t *>(p) = v;
}
__device__ __forceinline__ uint64_t ld_status(const uint64_t *p) {
    return *reinterpret_cast<const volatile uint64_t *>(p);
}

// err[0] holds the sticky error bits the host reads; err[2] is this tick's
// abort flag (cleared by the host before every tick).
__device__ __forceinline__ bool ld_abort(const uint32_t *err) {
    return *reinterpret_cast<const volatile uint32_t *>(err + 2) != 0u;
}
__device__ __forceinline__ void raise_timeout(uint32_t *err) {
    atomicOr(err, kErrTimeout);
    atomicOr(err + 2, 1u);
}

__device__ __forceinline__ uint32_t warp_sum_u32(uint32_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Exclusive prefix of `agg` over all earlier tiles, called by one full warp,
// in two halves so that a tile can publish its aggregate as soon as it is
// known and do other work before it waits: lookback_warp_publish stores the
// aggregate (the inclusive prefix for tile 0); lookback_warp_resolve looks
// back 32 predecessors at a time, publishes the inclusive prefix and returns
// the exclusive prefix in all lanes.
__device__ __forceinline__ void lookback_warp_publish(uint64_t *status, uint32_t tile,
                                                      uint32_t epoch, uint32_t agg) {
    if ((threadIdx.x & 31) == 0)
        st_status(&status[tile], pack_status(epoch, tile == 0 ? kFlagPrefix : kFlagAgg, agg));
}

__device__ __forceinline__ uint32_t lookback_warp_resolve(uint64_t *status, uint32_t tile,
                                                          uint32_t epoch, uint32_t agg,
                                                          uint32_t *err) {
    const int lane = threadIdx.x & 31;
    if (tile == 0) return 0u;
    uint32_t excl = 0;
    int64_t t = (int64_t)tile - 1;
    uint32_t spins = 0;
    for (;;) {
        const int64_t idx = t - lane;
        uint64_t s = idx >= 0 ? ld_status(&status[idx]) : pack_status(epoch, kFlagPrefix, 0u);
        const bool ready = status_ready(s, epoch);
        const unsigned rm = __ballot_sync(kFull, ready);
        const unsigned pm = __ballot_sync(kFull, ready && status_flag(s) == kFlagPrefix);
        if (pm) {
            const int p = __ffs(pm) - 1;
            const unsigned need = p == 31 ? kFull : ((1u << (p + 1)) - 1u);
            if ((rm & need) == need) {
                excl += warp_sum_u32(lane <= p ? status_value(s) : 0u);
                break;
            }
        } else if (rm == kFull) {
            excl += warp_sum_u32(status_value(s));
            t -= 32;
            continue;
        }
        ++spins;
        const bool give_up = spins > kSpinLimit || ((spins & 63u) == 0u && ld_abort(err));
        if (__any_sync(kFull, give_up)) {
            if (lane == 0) raise_timeout(err);
            break;
        }
        if (spins > 8) __nanosleep(100);
    }
    if (lane == 0) st_status(&status[tile], pack_status(epoch, kFlagPrefix, excl + agg));
    return excl;
}

__device__ __forceinline__ uint32_t lookback_warp(uint64_t *status, uint32_t tile,
                                                  uint32_t epoch, uint32_t agg,
                                                  uint32_t *err) {
    lookback_warp_publish(status, tile, epoch, agg);
    return lookback_warp_resolve(status, tile, epoch, agg, err);
}

// Per-thread look-back over a strided status array (one digit of a radix pass
// per thread): status[t * stride].  Split in two so that a tile can publish its
// aggregate as soon as it is known and do other work before it waits:
// lookback_publish stores the aggregate (the inclusive prefix for tile 0);
// lookback_resolve reads the words of kAhead predecessors together and takes
// them in order -- a run of tiles that have published only their aggregates
// costs one memory round trip per kAhead tiles -- then publishes this tile's
// inclusive prefix and returns its exclusive prefix.
__device__ __forceinline__ void lookback_publish(uint64_t *status, uint32_t tile,
                                                 uint32_t stride, uint32_t epoch, uint32_t agg) {
    st_status(&status[(uint64_t)tile * stride],
              pack_status(epoch, tile == 0 ? kFlagPrefix : kFlagAgg, agg));
}

__device__ __forceinline__ uint32_t lookback_resolve(uint64_t *status, uint32_t tile,
                                                     uint32_t stride, uint32_t epoch,
                                                     uint32_t agg, uint32_t *err) {
    constexpr int kAhead = 8;
    if (tile == 0) return 0u;
    uint32_t excl = 0;
    bool done = false;
    for (int64_t t = (int64_t)tile - 1; t >= 0 && !done; t -= kAhead) {
        uint64_t s[kAhead];
#pragma unroll
        for (int i = 0; i < kAhead; ++i)
            s[i] = t - i >= 0 ? ld_status(&status[(uint64_t)(t - i) * stride])
                              : pack_status(epoch, kFlagPrefix, 0u);
#pragma unroll
        for (int i = 0; i < kAhead; ++i) {
            if (done) break;
            uint32_t spins = 0;
            while (!status_ready(s[i], epoch)) {
                ++spins;
                if (spins > kSpinLimit || ((spins & 63u) == 0u && ld_abort(err))) {
                    raise_timeout(err);
                    s[i] = pack_status(epoch, kFlagPrefix, 0u);
                    break;
                }
                if (spins > 8) __nanosleep(100);
                s[i] = ld_status(&status[(uint64_t)(t - i) * stride]);
            }
            excl += status_value(s[i]);
            if (status_flag(s[i]) == kFlagPrefix) done = true;
        }
    }
    st_status(&status[(uint64_t)tile * stride], pack_status(epoch, kFlagPrefix, excl + agg));
    return excl;
}

// Block-wide exclusive scan of one uint32 per thread for blockDim.x == 256.
// `tmp` needs 8 words of shared memory.  Returns the exclusive prefix; the
// block total is written to *total (shared) when non-null.
__device__ __forceinline__ uint32_t block_excl_scan_256(uint32_t v, uint32_t *tmp,
                                                        uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    uint32_t wpre = 0, all = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        uint32_t t = tmp[w];
        wpre += (w < warp) ? t : 0u;
        all += t;
    }
    if (total && threadIdx.x == 0) *total = all;
    __syncthreads();
    return wpre + x - v;
}

// Exclusive prefix of count(0) .. count(n - 1) into out[0 .. n - 1] and the
// total into out[n], by one block of exactly 1024 threads (all of them call
// it); n may exceed the block, the counts are taken 1024 at a time.
template <class Count>
__device__ void block_prefix_1024(int n, const Count &count, long long *out) {
    __shared__ long long wsum[32];
    __shared__ long long carry;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += 1024) {
        const int i = base + tid;
        const long long v = i < n ? count(i) : 0;
        long long x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            long long t = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(kFull, t, o);
                if (lane >= o) t += y;
            }
            wsum[lane] = t;
        }
        __syncthreads();
        const long long excl = carry + (wid > 0 ? wsum[wid - 1] : 0) + x - v;
        if (i < n) out[i] = excl;
        __syncthreads();  // every thread has read carry and wsum
        if (tid == 1023) carry = excl + v;
        __syncthreads();
    }
    if (tid == 0) out[n] = carry;
}

}  // namespace knnq
