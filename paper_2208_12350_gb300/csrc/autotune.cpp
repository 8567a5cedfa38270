// sw_autotune: measured choice of the batched path's tuning for a batch.
//
// The planner (plan.cpp) picks lane-group widths from a cost model.  The
// autotuner measures instead: it runs the batch under each candidate tuning
// - bulk lane-group width G in {2, 4, 8, 16, 32} x long-pair cap in {0.25, 0.5, 1,
// none}, plus the planner's own choice, for each kernel form the batch
// allows (the packed 16-bit form with 16 or with 32 rows per lane, and the
// scaled int32 form) - keeps the fastest, sets it on the context and
// records it in a JSON cache keyed by the GPU (name, SM count) and a
// signature of the batch (pair count, length sums, maxima and length
// histograms, scoring), so the next run of the same kind of batch skips the
// measurement.  Every form is a kernel instantiation built into the library
// (no rebuild); the winner is then timed with one resident block per SM
// fewer (2 instead of 3 for 16 rows per lane).  Steps per staging block are
// fixed per form (8; 4 measured 9 % slower on 100k DNA pairs).
#include <cuda_runtime.h>
#include <unistd.h>

#include <algorithm>
#include <cinttypes>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "sw_internal.h"
#include "swgb.h"

namespace swgb {
namespace {

uint64_t fnv1a(uint64_t h, const void *data, size_t n) {
    const unsigned char *p = static_cast<const unsigned char *>(data);
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

// Part of every cache key: a tuning measured on another kernel build is not
// reused.  Changed whenever the batched kernel's code changes.
constexpr char kKernelRevision[] = "group-kernel-r14 H+go / transposed reverse / linear / score tables / warp-built profiles / packed 16-bit / half-width tails / paired end-key chain / strip-start cost 18 / branch-free staging / group slots / forms / bulk widths to 32";

std::string batch_key(const char *gpu, int sms, const int64_t *qo, const int64_t *ro, int n_pairs,
                      const int8_t *mat, int A, int go, int ge) {
    uint64_t h = 1469598103934665603ull;
    h = fnv1a(h, kKernelRevision, sizeof kKernelRevision - 1);
    h = fnv1a(h, gpu, std::strlen(gpu));
    h = fnv1a(h, &sms, sizeof sms);
    h = fnv1a(h, &n_pairs, sizeof n_pairs);
    h = fnv1a(h, &A, sizeof A);
    h = fnv1a(h, &go, sizeof go);
    h = fnv1a(h, &ge, sizeof ge);
    h = fnv1a(h, mat, (size_t)A * A);
    int64_t sum_n = 0, sum_m = 0, max_n = 0, max_m = 0;
    double sum_nm = 0;
    int64_t hist_n[32] = {0}, hist_m[32] = {0};
    for (int i = 0; i < n_pairs; ++i) {
        const int64_t n = qo[i + 1] - qo[i], m = ro[i + 1] - ro[i];
        sum_n += n;
        sum_m += m;
        sum_nm += (double)n * (double)m;
        max_n = std::max(max_n, n);
        max_m = std::max(max_m, m);
        hist_n[std::min<int64_t>(31, n / 64)]++;
        hist_m[std::min<int64_t>(31, m / 256)]++;
    }
    h = fnv1a(h, &sum_n, sizeof sum_n);
    h = fnv1a(h, &sum_m, sizeof sum_m);
    h = fnv1a(h, &sum_nm, sizeof sum_nm);
    h = fnv1a(h, &max_n, sizeof max_n);
    h = fnv1a(h, &max_m, sizeof max_m);
    h = fnv1a(h, hist_n, sizeof hist_n);
    h = fnv1a(h, hist_m, sizeof hist_m);
    char buf[32];
    snprintf(buf, sizeof buf, "%016" PRIx64, h);
    return buf;
}

struct Entry {
    std::string key;
    int log2g = -1;
    double frac = 0.5, ms = 0;
    int arith = -1, rows = 16;  // kernel form (sw_ctx_set_form)
    int blocks = 0;             // resident blocks per SM (0: as many as fit)
};

// The cache file is a JSON object {"entries": [ {...}, ... ]} with one
// entry per line, as this file writes it.
std::vector<Entry> read_cache(const char *path) {
    std::vector<Entry> out;
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {
        const size_t k = line.find("\"key\": \"");
        if (k == std::string::npos) continue;
        Entry e;
        const size_t k0 = k + 8, k1 = line.find('"', k0);
        if (k1 == std::string::npos) continue;
        e.key = line.substr(k0, k1 - k0);
        auto num = [&](const char *name, double &v) {
            const size_t p = line.find(name);
            if (p != std::string::npos) v = std::atof(line.c_str() + p + std::strlen(name));
        };
        double lg = -1, ar = -1, rw = 16, bl = 0;
        num("\"narrow_log2g\": ", lg);
        num("\"cap_fraction\": ", e.frac);
        num("\"ms\": ", e.ms);
        num("\"arith\": ", ar);
        num("\"rows\": ", rw);
        num("\"blocks_per_sm\": ", bl);
        e.log2g = (int)lg;
        e.arith = (int)ar;
        e.rows = (int)rw;
        e.blocks = (int)bl;
        out.push_back(e);
    }
    return out;
}

bool write_cache(const char *path, const std::vector<Entry> &entries, const char *gpu, int sms) {
    // a temporary file of this process's own, renamed over the cache: several
    // processes tuning at once (one per GPU) never interleave their lines,
    // and a reader sees one whole file or the other
    const std::string tmp = std::string(path) + ".tmp." + std::to_string((long long)getpid());
    std::ofstream f(tmp);
    if (!f) return false;
    f << "{\"gpu\": \"" << gpu << "\", \"sms\": " << sms << ", \"entries\": [\n";
    for (size_t i = 0; i < entries.size(); ++i) {
        char buf[256];
        snprintf(buf, sizeof buf,
                 "  {\"key\": \"%s\", \"narrow_log2g\": %d, \"cap_fraction\": %.17g, "
                 "\"arith\": %d, \"rows\": %d, \"blocks_per_sm\": %d, \"ms\": %.17g}%s\n",
                 entries[i].key.c_str(), entries[i].log2g, entries[i].frac, entries[i].arith,
                 entries[i].rows, entries[i].blocks, entries[i].ms,
                 i + 1 < entries.size() ? "," : "");
        f << buf;
    }
    f << "]}\n";
    f.close();
    return std::rename(tmp.c_str(), path) == 0;
}

}  // namespace
}  // namespace swgb

using namespace swgb;

extern "C" int sw_autotune_ex(sw_ctx *ctx, const int64_t *q_offsets, const int64_t *r_offsets,
                              int32_t n_pairs, const int8_t *score_matrix, int32_t alphabet_size,
                              int32_t gap_open, int32_t gap_extend, const uint8_t *q_seqs,
                              const uint8_t *r_seqs, int32_t *out, uint32_t flags,
                              const char *cache_path, void *stream, int32_t *chosen_log2g,
                              double *chosen_frac, double *chosen_ms) {
    if (!ctx || n_pairs <= 0 || !q_offsets || !r_offsets || !score_matrix || !q_seqs || !r_seqs ||
        !out)
        return set_error(SW_EINVAL, "sw_autotune: bad argument");
    // the candidates run the kernels the timed plans will run: the same
    // arithmetic form and passes (the inputs here are one byte per residue)
    flags &= SW_PLAN_ENDS_ONLY | SW_PLAN_NO_S16X2 | SW_PLAN_PAIR_SCRATCH;
    char gpu[256];
    int32_t sms = 0;
    sw_ctx_sm_count(ctx, &sms);
    {
        int dev = 0;
        cudaDeviceProp prop;
        cudaGetDevice(&dev);
        if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
            return set_error(SW_ECUDA, "sw_autotune: device properties");
        snprintf(gpu, sizeof gpu, "%s", prop.name);
    }
    std::string key = batch_key(gpu, sms, q_offsets, r_offsets, n_pairs, score_matrix,
                                alphabet_size, gap_open, gap_extend);
    if (flags) key += "/flags" + std::to_string(flags);
    std::vector<Entry> cache;
    if (cache_path && *cache_path) {
        cache = read_cache(cache_path);
        for (const Entry &e : cache)
            if (e.key == key) {
                // an entry the context does not accept (a damaged or foreign
                // file) is measured again, as if it were absent
                int rc = sw_ctx_set_tuning(ctx, e.log2g, e.frac);
                if (rc == SW_OK) rc = sw_ctx_set_form(ctx, e.arith, e.rows, e.blocks);
                if (rc != SW_OK) break;
                if (chosen_log2g) *chosen_log2g = e.log2g;
                if (chosen_frac) *chosen_frac = e.frac;
                if (chosen_ms) *chosen_ms = e.ms;
                return SW_OK;
            }
    }
    struct Cand {
        int lg;
        double frac;
        int arith, rows;
        int blocks = 0;
    };
    // the kernel forms this batch allows, from host-only plans: the default
    // plan's; where that is a packed form, also the scaled int32 form; where
    // it is the packed form with 32-bit profile words and two blocks of the
    // 32-rows kernel fit an SM, also 32 rows per lane
    std::vector<std::pair<int, int>> forms = {{-1, 16}};
    {
        auto kind_of = [&](bool rows32, ProfileKind *k) -> int {
            HostPlan hp;
            std::string msg;
            const int rc = make_host_plan(q_offsets, r_offsets, n_pairs, score_matrix,
                                          alphabet_size, gap_open, gap_extend, SW_MODE_BATCHED,
                                          sms, -1, 0.5, &hp, &msg, 1, 8192,
                                          (flags & SW_PLAN_NO_S16X2) == 0, group_blocks_per_sm,
                                          (flags & SW_PLAN_PAIR_SCRATCH) == 0, rows32);
            if (rc != SW_OK) return set_error(rc, ("sw_autotune: " + msg).c_str());
            *k = hp.kind;
            return SW_OK;
        };
        ProfileKind k16 = ProfileKind::kInt32, k32 = ProfileKind::kInt32;
        int rc0 = kind_of(false, &k16);
        if (rc0 == SW_OK) rc0 = kind_of(true, &k32);
        if (rc0 != SW_OK) return rc0;
        if (k32 == ProfileKind::kPacked16R32) forms.push_back({1, 32});
        if (k16 == ProfileKind::kPacked16 || k16 == ProfileKind::kPacked16Bytes)
            forms.push_back({0, 16});
    }
    std::vector<Cand> cands;
    for (const auto &f : forms) {
        cands.push_back({-1, 0.5, f.first, f.second});
        // bulk widths up to 32 lanes: small batches (and the tail of large
        // ones) finish sooner on wide groups, which cut a pair's serial sweep
        for (int lg = kMinLog2G; lg <= 5; ++lg)
            for (double fr : {0.25, 0.5, 1.0, 1e9}) cands.push_back({lg, fr, f.first, f.second});
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return set_error(SW_ECUDA, "sw_autotune: event creation failed");
    const int64_t n = n_pairs;
    Cand best{-1, 0.5, -1, 16};
    double best_ms = 1e30;
    int rc = SW_OK;
    auto time_cand = [&](const Cand &c) {
        if ((rc = sw_ctx_set_tuning(ctx, c.lg, c.frac)) != SW_OK) return;
        if ((rc = sw_ctx_set_form(ctx, c.arith, c.rows, c.blocks)) != SW_OK) return;
        sw_plan *plan = nullptr;
        rc = sw_plan_create(ctx, q_offsets, r_offsets, n_pairs, score_matrix, alphabet_size,
                            gap_open, gap_extend, SW_MODE_BATCHED, flags, &plan);
        if (rc != SW_OK) return;
        float total = 0.f;
        for (int it = 0; it < 3 && rc == SW_OK; ++it) {
            cudaEventRecord(e0, s);
            rc = sw_plan_execute(plan, q_seqs, r_seqs, out, out + n, out + 2 * n, out + 3 * n,
                                 out + 4 * n, stream);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) rc = set_error(SW_ECUDA, "sw_autotune: run");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (it > 0) total += ms;  // first run warms up
        }
        sw_plan_destroy(plan);
        if (rc != SW_OK) return;
        const double ms = total / 2.0;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    };
    for (const Cand &c : cands) {
        time_cand(c);
        if (rc != SW_OK) break;
    }
    // then the winner with one block per SM fewer than fit (16 rows per lane:
    // 3 fit), which leaves each warp more of the SM's issue slots
    if (rc == SW_OK && best.rows == 16) {
        Cand c = best;
        c.blocks = 2;
        time_cand(c);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != SW_OK) return rc;
    if ((rc = sw_ctx_set_tuning(ctx, best.lg, best.frac)) != SW_OK) return rc;
    if ((rc = sw_ctx_set_form(ctx, best.arith, best.rows, best.blocks)) != SW_OK) return rc;
    if (chosen_log2g) *chosen_log2g = best.lg;
    if (chosen_frac) *chosen_frac = best.frac;
    if (chosen_ms) *chosen_ms = best_ms;
    if (cache_path && *cache_path) {
        cache.erase(std::remove_if(cache.begin(), cache.end(),
                                   [&](const Entry &e) { return e.key == key; }),
                    cache.end());
        cache.push_back({key, best.lg, best.frac, best_ms, best.arith, best.rows, best.blocks});
        if (!write_cache(cache_path, cache, gpu, sms))
            return set_error(SW_EINVAL, "sw_autotune: cannot write the cache file");
    }
    return SW_OK;
}

extern "C" int sw_autotune(sw_ctx *ctx, const int64_t *q_offsets, const int64_t *r_offsets,
                           int32_t n_pairs, const int8_t *score_matrix, int32_t alphabet_size,
                           int32_t gap_open, int32_t gap_extend, const uint8_t *q_seqs,
                           const uint8_t *r_seqs, int32_t *out, const char *cache_path,
                           void *stream, int32_t *chosen_log2g, double *chosen_frac,
                           double *chosen_ms) {
    return sw_autotune_ex(ctx, q_offsets, r_offsets, n_pairs, score_matrix, alphabet_size,
                          gap_open, gap_extend, q_seqs, r_seqs, out, 0u, cache_path, stream,
                          chosen_log2g, chosen_frac, chosen_ms);
}
