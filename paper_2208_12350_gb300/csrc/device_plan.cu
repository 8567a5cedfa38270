// Device-side planning of a batch whose offsets live in device memory: the
// batch schedule (lane-group width of each pair, longest-first queues per
// width, warp shares) computed by small kernels on the launching stream, so
// that the one-shot call reads nothing back and never waits for the device.
//
// ADEPT's batch call is just its forward and reverse launches (Section
// III-B); the host planner of sw_plan_create first reads every length on
// the host.  Here the same rules run on the device, in this order:
//
//   1. classify   each pair's lengths from its offsets (bad offsets set a
//                 status bit and give the "no alignment" outputs, as do empty
//                 sequences, whose outputs are written here); its arithmetic
//                 route: the packed 16-bit form while min(n, m) is within the
//                 packed bound, else scaled int32 within its bound, else the
//                 plain kernel; the sum of the route's pair costs at the bulk
//                 lane-group width
//   2. keys       each group-route pair's width: the bulk width, or the
//                 narrowest wider one whose cost stays under the cap (a
//                 fraction of the mean load of a group), half width for a
//                 pair whose last strip would be at most half used (packed
//                 form with 32-bit profile words), and wide enough that the
//                 group's strip-boundary slot holds the pair; a 16-bit key
//                 (bucket of route and width, then the cost's logarithm,
//                 largest first) and the per-bucket pair counts and work
//   3. sort       a stable two-pass LSD radix sort of the keys (8-bit digits):
//                 per tile, per-warp digit counts by warp match; one scan of
//                 the (digit, tile) counts; a stable scatter that ranks each
//                 item among its tile's equal digits in index order.  The
//                 second scatter writes the pair records in schedule order.
//   4. tables     per route, one queue per width (widest first) over the
//                 sorted records, warps shared in proportion to class work,
//                 queue heads zeroed, and the plain kernel's ranges.
//
// The cost model is the host planner's: a pair on G lanes with R rows per
// lane takes ceil(n / GR) strips of m + G - 1 steps (in blocks of 4), plus a
// fixed charge per strip start times 32 / G (the warp builds the strip's
// profile with all its lanes), times 1.25 for the reverse pass.  Only the
// candidate search of the host planner (a simulated schedule of several
// bulk widths and caps) is left out: the bulk width and cap are the
// context's tuning, else 8 lanes and half the mean load.
#include <algorithm>
#include <climits>
#include <cstddef>
#include <cstring>

#include "device_plan.h"
#include "swgb.h"

namespace swgb {
namespace {

constexpr int kThreads = 256;  // planning kernels
constexpr int kWarps = kThreads / 32;
constexpr int kTile = 4096;  // items per radix tile (16 chunks of 32 per warp)
constexpr int kSeg = kTile / kWarps;
constexpr int kChunks = kSeg / 32;
constexpr int kDigits = 256;
constexpr int kScanThreads = 1024;

// Buckets of the sort key's top 4 bits.
constexpr int kBucketPlainShort = 10;  // plain kernel, n <= 256 (one row per thread)
constexpr int kBucketPlainLong = 11;   // plain kernel, longer queries
constexpr int kBucketNone = 12;        // nothing to align (written by classify)
constexpr int kNumBuckets = 13;
constexpr int kPlainShortMaxN = 256;

__host__ __device__ constexpr int bucket_of(int route, int lg) { return route * 5 + (5 - lg); }

// Workspace header (device), zeroed before each plan.
struct Header {
    unsigned long long total[2];                 // route cost sums at the bulk width
    unsigned long long work[kNumBuckets];        // class work (cost x G)
    int32_t count[kNumBuckets];                  // pairs per bucket
    int32_t plain_range[2][2];                   // {first, count}: short, long
    ClassInfo classes[2][kMaxClasses];           // per route, widest first
    int32_t counters[2][kMaxClasses];            // queue heads
};

__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Byte offsets of the workspace parts for n pairs; with guards, a guard
// region before every part and after the last (offsets in guard[]).
struct WsLayout {
    size_t hdr, counts1, counts2, keys0, keys1, vals1, pairs, scratch, total;
    size_t guard[9];
    int n_guards = 0;
};
__host__ WsLayout ws_layout(int64_t n, int64_t tiles, int64_t scratch_words, bool guards = false) {
    WsLayout L;
    size_t at = 0;
    auto take = [&](size_t bytes) {
        if (guards) {
            L.guard[L.n_guards++] = at;
            at += kGuardBytes;
        }
        const size_t o = at;
        at = align256(at + bytes);
        return o;
    };
    L.hdr = take(sizeof(Header));
    L.counts1 = take((size_t)kDigits * tiles * 4);
    L.counts2 = take((size_t)kDigits * tiles * 4);
    L.keys0 = take((size_t)n * 2);
    L.keys1 = take((size_t)n * 2);
    L.vals1 = take((size_t)n * 4);
    L.pairs = take((size_t)n * sizeof(PairInfo));
    L.scratch = take((size_t)scratch_words * 4);
    if (guards) {
        L.guard[L.n_guards++] = at;
        at += kGuardBytes;
    }
    L.total = at;
    return L;
}

struct PairView {
    int64_t q, r;
    int n, m;
    int route;  // 0 packed, 1 int32, 2 plain, 3 none
};

// Pair i's sequences: [qo[i], qe[i]) and [ro[i], re[i]), or CSR
// ([qo[i], qo[i + 1]) ...) when the end arrays are NULL.
struct Offsets {
    const int64_t *qo, *ro, *qe, *re;
};

__device__ __forceinline__ PairView view_pair(const DevicePlanShape &S, const Offsets &off, int i,
                                              bool *bad) {
    PairView v;
    const int64_t q0 = off.qo[i], r0 = off.ro[i];
    const int64_t q1 = off.qe ? off.qe[i] : off.qo[i + 1];
    const int64_t r1 = off.re ? off.re[i] : off.ro[i + 1];
    const int64_t n = q1 - q0, m = r1 - r0;
    *bad = q0 < 0 || r0 < 0 || n < 0 || m < 0 || n > SW_MAX_LEN || m > SW_MAX_LEN;
    v.q = q0;
    v.r = r0;
    v.n = *bad ? 0 : (int)n;
    v.m = *bad ? 0 : (int)m;
    const int mn = v.n < v.m ? v.n : v.m;
    if (v.n == 0 || v.m == 0)
        v.route = 3;
    else if (S.all_plain || v.n > kColBase || v.m > kColBase)
        v.route = 2;
    else if (S.route_on[0] && mn <= S.lim[0])
        v.route = 0;
    else if (S.route_on[1] && mn <= S.lim[1])
        v.route = 1;
    else
        v.route = 2;
    return v;
}

// Planner cost of a pair on 2^lg lanes (host planner's model, times 4).
__device__ __forceinline__ uint32_t pair_cost(int n, int m, int lg, int rows, int ov) {
    const int G = 1 << lg;
    const uint32_t strips = (uint32_t)((n + G * rows - 1) / (G * rows));
    const uint32_t cols = (uint32_t)((m + G - 1 + 3) / 4 * 4);
    return 5u * (strips * cols + strips * (uint32_t)ov * (uint32_t)(32 >> lg));
}

// Strip-boundary words per lane a pair needs on 2^lg lanes (0: one strip).
__device__ __forceinline__ int pair_slot_need(int n, int m, int lg, int rows) {
    const int G = 1 << lg, strip = G * rows;
    if (n <= strip && m <= strip) return 0;
    const int cols = n > m ? n : m;
    const int w = 2 * ((cols + 3) & ~3) + 4;
    return (((w + G - 1) / G) + 3) & ~3;
}

// log2 of c on 12 bits (7 bits of mantissa after the leading one): a
// monotone integer approximation, 0.5 % per step.
__device__ __forceinline__ uint32_t log_level(uint32_t c) {
    if (c == 0) return 0;
    const int msb = 31 - __clz(c);
    const uint32_t mant = msb >= 7 ? (c >> (msb - 7)) & 127u : (c << (7 - msb)) & 127u;
    return (uint32_t)msb * 128u + mant;
}

__device__ __forceinline__ void write_none(const Outputs &o, int id, bool ends_only) {
    o.score[id] = 0;
    o.qend[id] = -1;
    o.rend[id] = -1;
    if (!ends_only) {
        o.qstart[id] = -1;
        o.rstart[id] = -1;
    }
}

// 1. Routes, status, outputs of pairs with nothing to align, route cost sums.
__global__ void __launch_bounds__(kThreads) dp_classify(const DevicePlanShape S, const Offsets off,
                                                        Header *hdr, int32_t *status, Outputs o) {
    __shared__ unsigned long long tot[2];
    if (threadIdx.x < 2) tot[threadIdx.x] = 0;
    __syncthreads();
    unsigned long long my[2] = {0, 0};
    bool any_bad = false;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < S.n_pairs; i += gridDim.x * kThreads) {
        bool bad = false;
        const PairView v = view_pair(S, off, i, &bad);
        any_bad |= bad;
        if (v.route == 3)
            write_none(o, i, S.ends_only);
        else if (v.route < 2)
            my[v.route] += pair_cost(v.n, v.m, S.bulk_log2g, S.rows[v.route], S.strip_ov);
    }
    if (any_bad) atomicOr(status, kStatusBadOffsets);
    for (int r = 0; r < 2; ++r) {
        unsigned long long v = my[r];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&tot[r], v);
    }
    __syncthreads();
    if (threadIdx.x < 2 && tot[threadIdx.x]) atomicAdd(&hdr->total[threadIdx.x], tot[threadIdx.x]);
}

// The long-pair cap of a route, in pair-cost units: cap_fraction times the
// mean load of a bulk-width group (a cost above it takes wider groups).
__device__ __forceinline__ uint64_t route_cap(const DevicePlanShape &S, const Header *hdr,
                                              int route) {
    const double groups = (double)S.n_warps[route] * (double)(32 >> S.bulk_log2g);
    const double cap = S.cap_fraction * (double)hdr->total[route] / (groups > 1.0 ? groups : 1.0);
    return cap >= 1.8e19 ? ~0ull : (uint64_t)cap;  // cost > cap <=> cost > floor(cap)
}

// The width class of a group-route pair (log2 of its lane count), or -1
// when no group slot holds it (it then takes the plain kernel).
__device__ __forceinline__ int choose_lg(const DevicePlanShape &S, uint64_t cap, int n, int m,
                                         int route) {
    const int rows = S.rows[route], gn = S.bulk_log2g;
    // the narrowest width from gn up whose cost stays under the cap, else
    // the widest (32 lanes)
    int lg = gn;
    while (lg < 5 && (uint64_t)pair_cost(n, m, lg, rows, S.strip_ov) > cap) ++lg;
    if (S.half_tails[route] && lg == gn && gn > kMinLog2G) {
        const int h = rows << gn;
        if ((n + h / 2 - 1) / (h / 2) * (h / 2) < (n + h - 1) / h * h) lg = gn - 1;
    }
    while (lg < 5 && pair_slot_need(n, m, lg, rows) > S.slot_words) ++lg;
    return pair_slot_need(n, m, lg, rows) > S.slot_words ? -1 : lg;
}

// Per-warp digit counts of this tile's items (warp w: items [w kSeg, (w + 1) kSeg)).
template <class KeyFn>
__device__ __forceinline__ void tile_counts(int n, int shift, KeyFn key, uint32_t (*hist)[kDigits]) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = threadIdx.x; k < kWarps * kDigits; k += kThreads) hist[k / kDigits][k % kDigits] = 0;
    __syncthreads();
    const int base = blockIdx.x * kTile + warp * kSeg;
    for (int c = 0; c < kChunks; ++c) {
        const int i = base + c * 32 + lane;
        const bool valid = i < n;
        const unsigned live = __ballot_sync(0xffffffffu, valid);
        if (valid) {
            const uint32_t d = (key(i) >> shift) & (kDigits - 1);
            const unsigned peers = __match_any_sync(live, d);
            if (lane == __ffs(peers) - 1) hist[warp][d] += __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
}

// 2. Width classes, sort keys, per-bucket counts and work; digit counts of
// the first radix pass.
__global__ void __launch_bounds__(kThreads) dp_keys(const DevicePlanShape S, const Offsets off,
                                                    Header *hdr, uint16_t *keys0, uint32_t *counts1,
                                                    int tiles) {
    __shared__ uint32_t hist[kWarps][kDigits];
    __shared__ unsigned long long bwork[kNumBuckets];
    __shared__ int32_t bcount[kNumBuckets];
    __shared__ uint64_t cap[2];  // the routes' long-pair caps, computed once per block
    if (threadIdx.x < kNumBuckets) {
        bwork[threadIdx.x] = 0;
        bcount[threadIdx.x] = 0;
    }
    if (threadIdx.x < 2) cap[threadIdx.x] = route_cap(S, hdr, threadIdx.x);
    __syncthreads();
    const int lo = blockIdx.x * kTile, hi = min(S.n_pairs, lo + kTile);
    // per-thread bucket counts and work in registers (a select per bucket,
    // no shared-memory atomics per pair), reduced per warp after the loop
    uint32_t my_count[kNumBuckets];
    unsigned long long my_work[kNumBuckets];
#pragma unroll
    for (int b = 0; b < kNumBuckets; ++b) my_count[b] = 0, my_work[b] = 0;
    for (int i = lo + threadIdx.x; i < hi; i += kThreads) {
        bool bad = false;
        const PairView v = view_pair(S, off, i, &bad);
        int bucket = kBucketNone;
        uint32_t cost = 0;
        if (v.route < 2) {
            const int lg = choose_lg(S, cap[v.route], v.n, v.m, v.route);
            if (lg >= 0) {
                bucket = bucket_of(v.route, lg);
                cost = pair_cost(v.n, v.m, lg, S.rows[v.route], S.strip_ov);
                const unsigned long long w = (unsigned long long)cost << lg;
#pragma unroll
                for (int b = 0; b < kNumBuckets; ++b) my_work[b] += b == bucket ? w : 0ull;
            } else {
                bucket = v.n <= kPlainShortMaxN ? kBucketPlainShort : kBucketPlainLong;
            }
        } else if (v.route == 2) {
            bucket = v.n <= kPlainShortMaxN ? kBucketPlainShort : kBucketPlainLong;
        }
        if (bucket == kBucketPlainShort || bucket == kBucketPlainLong) {
            const uint64_t c = (uint64_t)v.n * (uint64_t)v.m;
            cost = c > 0xffffffffull ? 0xffffffffu : (uint32_t)c;
        }
#pragma unroll
        for (int b = 0; b < kNumBuckets; ++b) my_count[b] += b == bucket ? 1u : 0u;
        keys0[i] = (uint16_t)((bucket << 12) | (4095u - log_level(cost)));
    }
#pragma unroll
    for (int b = 0; b < kNumBuckets; ++b) {
        uint32_t c = my_count[b];
        unsigned long long w = my_work[b];
        for (int o = 16; o > 0; o >>= 1) {
            c += __shfl_xor_sync(0xffffffffu, c, o);
            w += __shfl_xor_sync(0xffffffffu, w, o);
        }
        if ((threadIdx.x & 31) == 0) {
            if (c) atomicAdd(&bcount[b], (int32_t)c);
            if (w) atomicAdd(&bwork[b], w);
        }
    }
    __syncthreads();
    if (threadIdx.x < kNumBuckets) {
        if (bcount[threadIdx.x]) atomicAdd(&hdr->count[threadIdx.x], bcount[threadIdx.x]);
        if (bwork[threadIdx.x]) atomicAdd(&hdr->work[threadIdx.x], bwork[threadIdx.x]);
    }
    // the keys this block wrote are visible to its own threads after the barrier
    __threadfence_block();
    tile_counts(S.n_pairs, 0, [&](int i) { return (uint32_t)keys0[i]; }, hist);
    for (int d = threadIdx.x; d < kDigits; d += kThreads) {
        uint32_t s = 0;
        for (int w = 0; w < kWarps; ++w) s += hist[w][d];
        counts1[(size_t)d * tiles + blockIdx.x] = s;
    }
}

// Exclusive scan of counts[0 .. len) in place (one block).
__device__ void block_exclusive_scan(uint32_t *counts, int len) {
    __shared__ uint32_t wsum[kScanThreads / 32];
    const int t = threadIdx.x;
    const int per = (len + kScanThreads - 1) / kScanThreads;
    const int b = t * per, e = min(len, b + per);
    uint32_t s = 0;
    for (int k = b; k < e; ++k) s += counts[k];
    // inclusive scan of the 1024 partial sums: warps, then warp totals
    uint32_t v = s;
    const int lane = t & 31, warp = t >> 5;
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t o = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += o;
    }
    if (lane == 31) wsum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = wsum[lane];
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t o = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += o;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    uint32_t run = v - s + (warp > 0 ? wsum[warp - 1] : 0);
    for (int k = b; k < e; ++k) {
        const uint32_t c = counts[k];
        counts[k] = run;
        run += c;
    }
}

// 3a. Scan of the first pass's (digit, tile) counts.
__global__ void __launch_bounds__(kScanThreads) dp_scan(uint32_t *counts, int len) {
    block_exclusive_scan(counts, len);
}

// Stable scatter of one radix pass: each item goes to base(digit, tile) +
// (equal digits of earlier warps of the tile) + (equal digits earlier in the
// warp's segment).
template <class KeyFn, class EmitFn>
__device__ __forceinline__ void tile_scatter(int n, int shift, int tiles, const uint32_t *offsets,
                                             KeyFn key, EmitFn emit, uint32_t (*hist)[kDigits]) {
    tile_counts(n, shift, key, hist);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = threadIdx.x; d < kDigits; d += kThreads) {
        uint32_t run = offsets[(size_t)d * tiles + blockIdx.x];
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t c = hist[w][d];
            hist[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
    const unsigned below = (1u << lane) - 1u;
    const int base = blockIdx.x * kTile + warp * kSeg;
    for (int c = 0; c < kChunks; ++c) {
        const int i = base + c * 32 + lane;
        const bool valid = i < n;
        const unsigned live = __ballot_sync(0xffffffffu, valid);
        unsigned peers = 0;
        uint32_t d = 0;
        if (valid) {
            const uint32_t k = key(i);
            d = (k >> shift) & (kDigits - 1);
            peers = __match_any_sync(live, d);
            emit(i, k, hist[warp][d] + __popc(peers & below));
        }
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) hist[warp][d] += __popc(peers);
        __syncwarp();
    }
}

// 3b. First pass (low 8 bits) to keys1/vals1; counts of the second pass.
__global__ void __launch_bounds__(kThreads) dp_scatter1(int n, int tiles, const uint16_t *keys0,
                                                        const uint32_t *offsets1, uint16_t *keys1,
                                                        uint32_t *vals1, uint32_t *counts2) {
    __shared__ uint32_t hist[kWarps][kDigits];
    tile_scatter(
        n, 0, tiles, offsets1, [&](int i) { return (uint32_t)keys0[i]; },
        [&](int i, uint32_t k, uint32_t pos) {
            keys1[pos] = (uint16_t)k;
            vals1[pos] = (uint32_t)i;
            atomicAdd(&counts2[(size_t)(k >> 8) * tiles + pos / kTile], 1u);
        },
        hist);
}

// 3c. Scan of the second pass's counts, then the class tables (one block).
__global__ void __launch_bounds__(kScanThreads) dp_scan_tables(const DevicePlanShape S,
                                                               uint32_t *counts, int len,
                                                               Header *hdr) {
    block_exclusive_scan(counts, len);
    if (threadIdx.x != 0) return;
    int first[kNumBuckets + 1];
    first[0] = 0;
    for (int b = 0; b < kNumBuckets; ++b) first[b + 1] = first[b] + hdr->count[b];
    for (int r = 0; r < 2; ++r) {
        // widths 32 .. 2 in order; warps in proportion to class work
        double wt = 0, work[5];
        int nonempty = 0;
        for (int c = 0; c < 5; ++c) {
            const int b = bucket_of(r, 5 - c);
            work[c] = hdr->count[b] ? (double)hdr->work[b] : 0.0;
            wt += work[c];
            nonempty += hdr->count[b] ? 1 : 0;
        }
        const int nw = S.n_warps[r];
        int warps[5], assigned = 0, big = -1;
        for (int c = 0; c < 5; ++c) {
            const int b = bucket_of(r, 5 - c);
            warps[c] = 0;
            if (!hdr->count[b]) continue;
            warps[c] = (int)floor((double)nw * work[c] / (wt > 1e-9 ? wt : 1e-9));
            if (warps[c] == 0 && nw >= nonempty) warps[c] = 1;
            assigned += warps[c];
            if (big < 0 || work[c] > work[big]) big = c;
        }
        if (big >= 0) {
            warps[big] += nw - assigned;
            if (warps[big] < 0) warps[big] = 0;
        }
        int wb = 0;
        for (int c = 0; c < 5; ++c) {
            const int b = bucket_of(r, 5 - c);
            ClassInfo ci;
            ci.first = first[b];
            ci.count = hdr->count[b];
            ci.log2g = 5 - c;
            ci.warp_begin = wb;
            wb += warps[c];
            hdr->classes[r][c] = ci;
            hdr->counters[r][c] = 0;
        }
        // classes after the last one with warps start no warp
        for (int c = 4; c >= 0 && warps[c] == 0; --c) hdr->classes[r][c].warp_begin = nw;
        hdr->classes[r][5] = ClassInfo{0, 0, 1, nw};
        hdr->counters[r][5] = 0;
    }
    hdr->plain_range[0][0] = first[kBucketPlainShort];
    hdr->plain_range[0][1] = hdr->count[kBucketPlainShort];
    hdr->plain_range[1][0] = first[kBucketPlainLong];
    hdr->plain_range[1][1] = hdr->count[kBucketPlainLong];
}

// 3d. Second pass (high 8 bits): the pair records in schedule order.
__global__ void __launch_bounds__(kThreads) dp_scatter2(const DevicePlanShape S, int tiles,
                                                        const uint16_t *keys1, const uint32_t *vals1,
                                                        const uint32_t *offsets2,
                                                        const Offsets off, PairInfo *pairs) {
    __shared__ uint32_t hist[kWarps][kDigits];
    tile_scatter(
        S.n_pairs, 8, tiles, offsets2, [&](int k) { return (uint32_t)keys1[k]; },
        [&](int k, uint32_t key, uint32_t pos) {
            if ((int)(key >> 12) >= kBucketNone) return;
            const int i = (int)vals1[k];
            bool bad = false;
            const PairView v = view_pair(S, off, i, &bad);
            pairs[pos] = PairInfo{v.q, v.r, -1, v.n, v.m, i, 0};
        },
        hist);
}

}  // namespace

size_t device_plan_workspace_bytes(const DevicePlanShape &S) {
    const int64_t tiles = std::max<int64_t>(1, ((int64_t)S.n_pairs + kTile - 1) / kTile);
    return ws_layout(S.n_pairs, tiles, S.scratch_words, S.guards != 0).total;
}

int device_plan_shape(int32_t n_pairs, const int8_t *mat, int32_t A, int32_t go, int32_t ge,
                      int32_t mode, int sm_count, int narrow_log2g, double cap_fraction,
                      int slot_words, DevicePlanShape *out, std::string *msg,
                      int min_pairs_per_warp) {
    DevicePlanShape S;
    std::memset(&S, 0, sizeof S);
    S.n_pairs = n_pairs;
    S.A = A;
    S.go = go;
    S.ge = ge;
    std::memcpy(S.mat, mat, (size_t)A * A);
    S.linear = go == ge;
    S.all_plain = mode == SW_MODE_PLAIN;
    S.bulk_log2g = narrow_log2g >= 0 ? std::max(narrow_log2g, kMinLog2G) : 3;
    S.cap_fraction = narrow_log2g >= 0 ? cap_fraction : 0.5;
    S.strip_ov = 18;  // the host planner's strip-start charge
    S.slot_words = slot_words;
    int smax = -128, smin = 127;
    for (int i = 0; i < A * A; ++i) {
        smax = std::max(smax, (int)mat[i]);
        smin = std::min(smin, (int)mat[i]);
    }
    const int sp = std::max(smax, 0);
    const int64_t per_block = (int64_t)kGroupWarps * std::max(1, min_pairs_per_warp);
    const int64_t want_grid = std::max<int64_t>(1, ((int64_t)n_pairs + per_block - 1) / per_block);
    // route 0: packed 16-bit form (32-bit profile words, else bytes)
    if (!S.all_plain && smin >= go && -go <= kMaxScaledGap && -ge <= kMaxScaledGap) {
        for (ProfileKind k : {ProfileKind::kPacked16, ProfileKind::kPacked16Bytes}) {
            const int scale = k == ProfileKind::kPacked16 ? 8 : 4;
            if ((int64_t)scale * -ge > 16384) continue;
            if (scale == 4 && smax - go > 31) continue;
            const int64_t room = 32767 / scale - sp + go;  // sp L <= room
            if (room < 0) continue;
            const int bps = group_blocks_per_sm(k, S.linear, A, nullptr);
            if (bps < 0) {
                if (msg) *msg = "occupancy query failed";
                return SW_ECUDA;
            }
            if (bps < 2) continue;
            S.route_on[0] = 1;
            S.kind[0] = (int)k;
            S.lim[0] = sp > 0 ? (int)std::min<int64_t>(room / sp, INT_MAX) : INT_MAX;
            S.grid[0] = (int)std::min<int64_t>((int64_t)bps * sm_count, want_grid);
            break;
        }
    }
    // route 1: scaled int32
    if (!S.all_plain && -go <= kMaxScaledGap && -ge <= kMaxScaledGap) {
        ProfileKind k = ProfileKind::kInt32;
        if (A > 4 && smax - go <= 127 && smin - go >= -127) k = ProfileKind::kInt8;
        const int bps = group_blocks_per_sm(k, S.linear, A, nullptr);
        if (bps < 0) {
            if (msg) *msg = "occupancy query failed";
            return SW_ECUDA;
        }
        if (bps > 0) {
            S.route_on[1] = 1;
            S.kind[1] = (int)k;
            S.lim[1] = sp > 0 ? kMaxScaledScore / sp : INT_MAX;
            S.grid[1] = (int)std::min<int64_t>((int64_t)bps * sm_count, want_grid);
        }
    }
    for (int r = 0; r < 2; ++r) {
        S.rows[r] = rows_of((ProfileKind)S.kind[r]);
        S.n_warps[r] = S.grid[r] * kGroupWarps;
        S.half_tails[r] = S.route_on[r] && S.kind[r] == (int)ProfileKind::kPacked16;
    }
    // group slots for the larger of the two grids (the kernels run one after
    // the other on the stream and share them)
    S.scratch_words = (int64_t)std::max(S.n_warps[0], S.n_warps[1]) * 32 * slot_words;
    S.plain_grid = std::max(1, sm_count * 4);
    *out = S;
    return SW_OK;
}

cudaError_t enqueue_device_plan(const DevicePlanShape &S, void *workspace, const int64_t *qo,
                                const int64_t *ro, const uint8_t *q, const uint8_t *r,
                                const Outputs &o, int32_t *status, cudaStream_t s,
                                const int64_t *qe, const int64_t *re) {
    const Offsets off{qo, ro, qe, re};
    if (S.n_pairs <= 0) return cudaSuccess;
    const int tiles = (int)std::max<int64_t>(1, ((int64_t)S.n_pairs + kTile - 1) / kTile);
    const WsLayout L = ws_layout(S.n_pairs, tiles, S.scratch_words, S.guards != 0);
    unsigned char *base = static_cast<unsigned char *>(workspace);
    Header *hdr = reinterpret_cast<Header *>(base + L.hdr);
    uint32_t *counts1 = reinterpret_cast<uint32_t *>(base + L.counts1);
    uint32_t *counts2 = reinterpret_cast<uint32_t *>(base + L.counts2);
    uint16_t *keys0 = reinterpret_cast<uint16_t *>(base + L.keys0);
    uint16_t *keys1 = reinterpret_cast<uint16_t *>(base + L.keys1);
    uint32_t *vals1 = reinterpret_cast<uint32_t *>(base + L.vals1);
    PairInfo *pairs = reinterpret_cast<PairInfo *>(base + L.pairs);
    uint32_t *scratch = reinterpret_cast<uint32_t *>(base + L.scratch);

    GuardList guards{};
    for (int k = 0; k < L.n_guards; ++k) {
        guards.ptr[k] = reinterpret_cast<uint32_t *>(base + L.guard[k]);
        guards.words[k] = (int32_t)(kGuardBytes / 4);
    }
    guards.n = L.n_guards;
    cudaError_t e = launch_guard_fill(guards, s);
    if (e != cudaSuccess) return e;
    // header and both count arrays start at zero (contiguous unless guarded)
    if (guards.n) {
        if ((e = cudaMemsetAsync(base + L.hdr, 0, sizeof(Header), s)) != cudaSuccess ||
            (e = cudaMemsetAsync(base + L.counts1, 0, (size_t)kDigits * tiles * 4, s)) !=
                cudaSuccess ||
            (e = cudaMemsetAsync(base + L.counts2, 0, (size_t)kDigits * tiles * 4, s)) !=
                cudaSuccess)
            return e;
    } else if ((e = cudaMemsetAsync(base, 0, L.keys0, s)) != cudaSuccess) {
        return e;
    }
    const int cgrid = (int)std::min<int64_t>(((int64_t)S.n_pairs + kThreads - 1) / kThreads, 1024);
    dp_classify<<<cgrid, kThreads, 0, s>>>(S, off, hdr, status, o);
    dp_keys<<<tiles, kThreads, 0, s>>>(S, off, hdr, keys0, counts1, tiles);
    dp_scan<<<1, kScanThreads, 0, s>>>(counts1, kDigits * tiles);
    dp_scatter1<<<tiles, kThreads, 0, s>>>(S.n_pairs, tiles, keys0, counts1, keys1, vals1, counts2);
    dp_scan_tables<<<1, kScanThreads, 0, s>>>(S, counts2, kDigits * tiles, hdr);
    dp_scatter2<<<tiles, kThreads, 0, s>>>(S, tiles, keys1, vals1, counts2, off, pairs);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;

    for (int rt = 0; rt < 2; ++rt) {
        if (!S.route_on[rt]) continue;
        GroupParams gp;
        std::memset(&gp, 0, sizeof gp);
        gp.q = q;
        gp.r = r;
        gp.pairs = pairs;
        // device addresses inside the header (no host access)
        gp.classes = reinterpret_cast<const ClassInfo *>(
            base + L.hdr + offsetof(Header, classes) + (size_t)rt * kMaxClasses * sizeof(ClassInfo));
        gp.n_classes = kMaxClasses;
        gp.counters = reinterpret_cast<int32_t *>(
            base + L.hdr + offsetof(Header, counters) + (size_t)rt * kMaxClasses * sizeof(int32_t));
        gp.n_warps = S.n_warps[rt];
        gp.scratch = scratch;
        gp.slot_words = S.slot_words;
        gp.status = status;
        gp.out = o;
        gp.alphabet = S.A;
        gp.gap_open = S.go;
        gp.gap_extend = S.ge;
        gp.ends_only = S.ends_only;
        std::memcpy(gp.mat, S.mat, (size_t)S.A * S.A);
        if ((e = launch_group(gp, (ProfileKind)S.kind[rt], S.linear, S.grid[rt], s)) != cudaSuccess)
            return e;
    }
    for (int k = 0; k < 2; ++k) {
        PlainParams pp;
        std::memset(&pp, 0, sizeof pp);
        pp.q = q;
        pp.r = r;
        pp.pairs = pairs;
        pp.range = reinterpret_cast<const int32_t *>(base + L.hdr + offsetof(Header, plain_range) +
                                                     (size_t)k * 2 * sizeof(int32_t));
        pp.status = status;
        pp.out = o;
        pp.alphabet = S.A;
        pp.gap_open = S.go;
        pp.gap_extend = S.ge;
        pp.ends_only = S.ends_only;
        std::memcpy(pp.mat, S.mat, (size_t)S.A * S.A);
        if ((e = launch_plain_range(pp, k == 0 ? kPlainShortMaxN : kPlainWideThreads,
                                    k == 0 ? 1 : kPlainMaxRows, S.plain_grid, s)) != cudaSuccess)
            return e;
    }
    // guards: every guard word still holds the pattern
    return launch_guard_check(guards, status, s);
}

}  // namespace swgb
