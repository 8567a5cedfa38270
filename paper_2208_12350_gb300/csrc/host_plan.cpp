// Host planning of a batch shared by every entry point: argument checks,
// profile width, which kernel each pair takes, the persistent kernel's
// class queues and grid, and the strip-boundary scratch layout.  The
// callers differ only in where they put the resulting tables (plan-owned
// allocations, the fixed module array, a serving arena).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "sw_internal.h"
#include "swgb.h"

namespace swgb {

static int plan_err(std::string *msg, int code, const char *fmt, long long a = 0, long long b = 0,
                    long long c = 0) {
    char buf[256];
    snprintf(buf, sizeof buf, fmt, a, b, c);
    if (msg) *msg = buf;
    return code;
}

// Planner cost of one strip start, in wavefront steps of the whole warp
// (the strip's profile build and its first staging wait).  A term per
// residue code (the build writes A + 1 profile columns) sent 20k protein
// pairs to wider groups, measured slower, so the cost is one constant.
// With branch-free steady-state staging (cheaper steps, so a strip start
// weighs more) 18 measured 0.6-0.8 % faster than 12 on 100k DNA and 20k
// protein pairs and no slower on 200k skewed pairs; 6 was 17 % slower there.
#ifndef SWGB_STRIP_OV_STEPS
#define SWGB_STRIP_OV_STEPS 18
#endif
static double strip_overhead_steps(int /*A*/) { return (double)SWGB_STRIP_OV_STEPS; }

static int smax_of(const int8_t *mat, int A, int *smin_out) {
    int smax = -128, smin = 127;
    for (int i = 0; i < A * A; ++i) {
        smax = std::max(smax, (int)mat[i]);
        smin = std::min(smin, (int)mat[i]);
    }
    if (smin_out) *smin_out = smin;
    return smax;
}

int check_batch(const int64_t *q_offsets, const int64_t *r_offsets, int32_t n_pairs,
                const int8_t *mat, int32_t A, int32_t go, int32_t ge, int64_t *q_bytes,
                int64_t *r_bytes, int64_t *max_scratch_words, std::string *msg) {
    if (n_pairs < 0) return plan_err(msg, SW_EINVAL, "n_pairs < 0");
    if (n_pairs > 0 && (!q_offsets || !r_offsets))
        return plan_err(msg, SW_EINVAL, "offsets are NULL");
    if (!mat) return plan_err(msg, SW_EINVAL, "score_matrix is NULL");
    if (A < 1 || A > SW_MAX_ALPHABET)
        return plan_err(msg, SW_EINVAL, "alphabet_size %lld not in [1, %lld]", A, SW_MAX_ALPHABET);
    if (ge > 0 || go > ge)
        return plan_err(msg, SW_EINVAL, "need gap_open <= gap_extend <= 0 (got %lld, %lld)", go,
                        ge);
    if (go < -SW_MAX_GAP) return plan_err(msg, SW_EINVAL, "|gap_open| above %lld", SW_MAX_GAP);
    const int smax = smax_of(mat, A, nullptr);
    int64_t words = 0;
    for (int32_t i = 0; i < n_pairs; ++i) {
        const int64_t a = q_offsets[i + 1] - q_offsets[i];
        const int64_t b = r_offsets[i + 1] - r_offsets[i];
        if (q_offsets[i] < 0 || r_offsets[i] < 0 || a < 0 || b < 0)
            return plan_err(msg, SW_ERANGE, "offsets of pair %lld negative or decreasing", i);
        if (a > SW_MAX_LEN || b > SW_MAX_LEN)
            return plan_err(msg, SW_ERANGE, "pair %lld has lengths (%lld, %lld) above SW_MAX_LEN", i,
                            a, b);
        if (max_scratch_words && a > 0 && b > 0 &&
            group_path_eligible((int)a, (int)b, smax, go, ge))
            words += pair_scratch_words((int)a, (int)b, 1 << kMinLog2G, kRows);
    }
    if (q_bytes) *q_bytes = n_pairs > 0 ? q_offsets[n_pairs] : 0;
    if (r_bytes) *r_bytes = n_pairs > 0 ? r_offsets[n_pairs] : 0;
    if (max_scratch_words) *max_scratch_words = words;
    return SW_OK;
}

int make_host_plan(const int64_t *q_offsets, const int64_t *r_offsets, int32_t n_pairs,
                   const int8_t *mat, int32_t A, int32_t go, int32_t ge, int32_t mode,
                   int sm_count, int narrow_log2g, double cap_fraction, HostPlan *out,
                   std::string *msg, int min_pairs_per_warp, int sample_cap,
                   bool allow_packed, BlocksPerSmFn blocks_per_sm, bool group_slots,
                   bool rows32, int blocks_cap) {
    *out = HostPlan();
    int rc = check_batch(q_offsets, r_offsets, n_pairs, mat, A, go, ge, nullptr, nullptr,
                         nullptr, msg);
    if (rc != SW_OK) return rc;
    if (mode != SW_MODE_AUTO && mode != SW_MODE_PLAIN && mode != SW_MODE_BATCHED)
        return plan_err(msg, SW_EINVAL, "unknown mode %lld", mode);
    if (mode == SW_MODE_AUTO) mode = SW_MODE_BATCHED;

    int smin = 0;
    const int smax = smax_of(mat, A, &smin);
    std::vector<int32_t> n(n_pairs), m(n_pairs);
    for (int32_t i = 0; i < n_pairs; ++i) {
        n[i] = (int32_t)(q_offsets[i + 1] - q_offsets[i]);
        m[i] = (int32_t)(r_offsets[i + 1] - r_offsets[i]);
    }
    out->linear = go == ge;
    out->q_bytes = n_pairs > 0 ? q_offsets[n_pairs] : 0;
    out->r_bytes = n_pairs > 0 ? r_offsets[n_pairs] : 0;
#ifndef SWGB_SMALL_ALPHABET_INT32
#define SWGB_SMALL_ALPHABET_INT32 1
#endif
#ifndef SWGB_PACKED16
#define SWGB_PACKED16 1
#endif
    // The packed 16-bit form takes the batch when every pair of the batched
    // path fits its bound (one kernel per batch).
    // Its profile of 32-bit words needs 4 bytes per row and residue code:
    // with large alphabets fewer than two blocks fit on an SM, and the byte
    // profile (scores scaled by 4) takes over where its bound holds.
    const bool try_packed = allow_packed && SWGB_PACKED16 && mode != SW_MODE_PLAIN && n_pairs > 0;
    bool packed8 = try_packed, packed4 = try_packed;
    for (int32_t i = 0; i < n_pairs && (packed8 || packed4); ++i)
        if (group_path_eligible(n[i], m[i], smax, go, ge)) {
            packed8 = packed8 && packed_eligible(n[i], m[i], smax, smin, go, ge, 8);
            packed4 = packed4 && packed_eligible(n[i], m[i], smax, smin, go, ge, 4);
        }
    for (ProfileKind k : {ProfileKind::kPacked16, ProfileKind::kPacked16Bytes}) {
        bool &ok = k == ProfileKind::kPacked16 ? packed8 : packed4;
        if (!ok) continue;
        const int b = blocks_per_sm(k, go == ge, A, nullptr);
        if (b < 0) return plan_err(msg, SW_ECUDA, "occupancy query failed");
        ok = b >= 2;
    }
    if (packed8 && rows32) {
        // the 32-rows-per-lane kernel, where two of its blocks fit an SM
        const int b = blocks_per_sm(ProfileKind::kPacked16R32, go == ge, A, nullptr);
        if (b < 0) return plan_err(msg, SW_ECUDA, "occupancy query failed");
        out->kind = b >= 2 ? ProfileKind::kPacked16R32 : ProfileKind::kPacked16;
    } else if (packed8)
        out->kind = ProfileKind::kPacked16;
    else if (packed4)
        out->kind = ProfileKind::kPacked16Bytes;
    else if (A <= 4 && SWGB_SMALL_ALPHABET_INT32)
        out->kind = ProfileKind::kInt32;
    else if (smax - go <= 127 && smin - go >= -127)
        out->kind = ProfileKind::kInt8;
    else
        out->kind = ProfileKind::kInt32;

    // The persistent kernel takes every eligible pair, unless its shared
    // memory for this alphabet and profile does not fit the device (int32
    // profiles of large alphabets): then every pair takes the plain kernel.
    bool group_fits = mode != SW_MODE_PLAIN;
    int bps = 0;
    if (group_fits) {
        bool any = false;
        for (int32_t i = 0; i < n_pairs && !any; ++i)
            any = group_path_eligible(n[i], m[i], smax, go, ge);
        if (any) {
            int smem = 0;
            bps = blocks_per_sm(out->kind, go == ge, A, &smem);
            if (bps < 0) return plan_err(msg, SW_ECUDA, "occupancy query failed");
            group_fits = bps > 0;
            if (blocks_cap > 0) bps = std::min(bps, blocks_cap);
        }
    }
    std::vector<PlanPair> gp;  // group-path pairs, id = index into gid
    std::vector<int32_t> gid;
    int plain_max_n = 0;
    for (int32_t i = 0; i < n_pairs; ++i) {
        if (!group_fits || !group_path_eligible(n[i], m[i], smax, go, ge)) {
            out->plain.push_back({q_offsets[i], r_offsets[i], -1, n[i], m[i], i, 0});
            plain_max_n = std::max(plain_max_n, n[i]);
        } else {
            gp.push_back({(int32_t)gid.size(), n[i], m[i]});
            gid.push_back(i);
        }
    }
    if (!gp.empty()) {
        const int64_t per_block = (int64_t)kGroupWarps * std::max(1, min_pairs_per_warp);
        const int64_t want = ((int64_t)gp.size() + per_block - 1) / per_block;
        out->grid = (int)std::min<int64_t>((int64_t)bps * sm_count, want);
        out->n_warps = out->grid * kGroupWarps;
    }
    const std::vector<PlannedClass> planned =
        plan_classes(gp, out->n_warps, narrow_log2g, cap_fraction, sample_cap,
                     out->kind == ProfileKind::kPacked16 || out->kind == ProfileKind::kPacked16R32,
                     rows_of(out->kind),
                     strip_overhead_steps(A));
    out->pairs.reserve(gp.size());
    int warp_begin = 0;
    for (const PlannedClass &pc : planned) {
        out->classes.push_back(
            {(int32_t)out->pairs.size(), (int32_t)pc.pairs.size(), pc.log2g, warp_begin});
        warp_begin += pc.warps;
        const int G = 1 << pc.log2g;
        for (int32_t k : pc.pairs) {
            const int32_t i = gid[k];
            PairInfo pi{q_offsets[i], r_offsets[i], -1, n[i], m[i], i, 0};
            if (n[i] > 0 && m[i] > 0) {
                if (group_slots) {
                    out->slot_words = std::max(out->slot_words,
                                               pair_slot_words(n[i], m[i], G, rows_of(out->kind)));
                } else {
                    const int64_t w = pair_scratch_words(n[i], m[i], G, rows_of(out->kind));
                    if (w > 0) {
                        pi.scratch = out->scratch_words;
                        out->scratch_words += w;
                    }
                }
            }
            out->pairs.push_back(pi);
        }
    }
    // one slot per lane of every warp of the launch
    if (group_slots) out->scratch_words = (int64_t)out->n_warps * 32 * out->slot_words;
    if (!out->plain.empty()) {
        if (plain_max_n <= 1024) {
            out->plain_threads = std::max(32, ((plain_max_n + 31) / 32) * 32);
            out->plain_kmax = 1;
        } else {
            out->plain_threads = kPlainWideThreads;
            out->plain_kmax = kPlainMaxRows;
        }
    }
    return SW_OK;
}

cudaError_t enqueue_plan(const HostPlan &hp, const DeviceTables &t, const uint8_t *q,
                         const uint8_t *r, const Outputs &o, const int8_t *mat, int A, int go,
                         int ge, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    if (!hp.pairs.empty()) {
        e = cudaMemsetAsync(t.counters, 0, kMaxClasses * sizeof(int32_t), s);
        if (e != cudaSuccess) return e;
        GroupParams gp;
        std::memset(&gp, 0, sizeof gp);
        gp.q = q;
        gp.r = r;
        gp.pairs = t.pairs;
        gp.classes = t.classes;
        gp.n_classes = (int32_t)hp.classes.size();
        gp.counters = t.counters;
        gp.n_warps = hp.n_warps;
        gp.scratch = t.scratch;
        gp.slot_words = hp.slot_words;
        gp.status = t.status;
        gp.out = o;
        gp.alphabet = A;
        gp.gap_open = go;
        gp.gap_extend = ge;
        gp.ends_only = hp.ends_only ? 1 : 0;
        std::memcpy(gp.mat, mat, (size_t)A * A);
        e = launch_group(gp, hp.kind, hp.linear, hp.grid, s);
        if (e != cudaSuccess) return e;
    }
    if (!hp.plain.empty()) {
        PlainParams pp;
        std::memset(&pp, 0, sizeof pp);
        pp.q = q;
        pp.r = r;
        pp.pairs = t.plain;
        pp.n_pairs = (int32_t)hp.plain.size();
        pp.status = t.status;
        pp.out = o;
        pp.alphabet = A;
        pp.gap_open = go;
        pp.gap_extend = ge;
        pp.ends_only = hp.ends_only ? 1 : 0;
        std::memcpy(pp.mat, mat, (size_t)A * A);
        e = launch_plain(pp, hp.plain_threads, hp.plain_kmax, s);
    }
    return e;
}

// Occupancy of the group kernel estimated from its shared memory alone (the
// host-only preview has no device to ask): 228 KB per SM with 1 KB reserved
// per block, 227 KB at most per block, and the blocks the registers allow
// (the launch bounds' minimum).
static int estimate_blocks_per_sm(ProfileKind kind, bool, int alphabet, int *smem_bytes) {
    const size_t bytes = group_smem_bytes(kind, alphabet);
    if (smem_bytes) *smem_bytes = (int)bytes;
    constexpr size_t kSmemPerSm = 233472, kReservedPerBlock = 1024, kMaxPerBlock = 232448;
    if (bytes > kMaxPerBlock) return 0;
    const int by_smem = (int)(kSmemPerSm / (bytes + kReservedPerBlock));
    const int by_regs = kind == ProfileKind::kPacked16R32 ? 2 : kGroupMinBlocks;
    return std::min(by_smem, by_regs);
}

}  // namespace swgb

extern "C" int sw_plan_preview(const int64_t *q_offsets, const int64_t *r_offsets,
                               int32_t n_pairs, const int8_t *score_matrix,
                               int32_t alphabet_size, int32_t gap_open, int32_t gap_extend,
                               int32_t mode, uint32_t flags, int32_t sm_count,
                               int32_t narrow_log2g, double cap_fraction, int32_t *out_kind,
                               int32_t *pair_log2g, int32_t *pair_rank) {
    using namespace swgb;
    if (!out_kind || (n_pairs > 0 && (!pair_log2g || !pair_rank)) || sm_count < 1 ||
        narrow_log2g < -1 || narrow_log2g > 5 || !(cap_fraction > 0))
        return set_error(SW_EINVAL, "sw_plan_preview: bad argument");
    HostPlan hp;
    std::string msg;
    const int rc = make_host_plan(q_offsets, r_offsets, n_pairs, score_matrix, alphabet_size,
                                  gap_open, gap_extend, mode, sm_count, narrow_log2g,
                                  cap_fraction, &hp, &msg, 1, 8192,
                                  (flags & SW_PLAN_NO_S16X2) == 0, estimate_blocks_per_sm, false,
                                  (flags & SW_PLAN_ROWS32) != 0);
    if (rc != SW_OK) return set_error(rc, ("sw_plan_preview: " + msg).c_str());
    *out_kind = (int32_t)hp.kind;
    for (int32_t i = 0; i < n_pairs; ++i) pair_log2g[i] = pair_rank[i] = -1;
    for (const ClassInfo &c : hp.classes)
        for (int32_t k = 0; k < c.count; ++k) {
            const int32_t id = hp.pairs[(size_t)(c.first + k)].id;
            pair_log2g[id] = c.log2g;
            pair_rank[id] = k;
        }
    for (size_t k = 0; k < hp.plain.size(); ++k) pair_rank[hp.plain[k].id] = (int32_t)k;
    return SW_OK;
}
