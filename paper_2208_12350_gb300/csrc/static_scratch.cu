// sw_align_batch_static: the batched alignment path without any device
// allocation, for callers that cannot call cudaMalloc.
//
// Some callers cannot allocate device memory on demand: a framework whose
// caching allocator already owns the device's memory budget, a fixed-size
// memory arena in an embedded or multi-tenant deployment, or a latency-
// critical serving loop that must not stall on the implicit device
// synchronisation of cudaMalloc/cudaFree.  This entry point runs the same
// persistent kernel (and, for pairs beyond its score bound, the same plain
// kernel) as sw_plan_execute, but every device table and all of the
// kernel's scratch - the per-class queue heads, the pair tables and the
// strip-boundary words of queries longer than one strip - live in one
// file-scope __device__ array of fixed size.  The caller passes the input
// sequences and the outputs, as for the other entry points.
//
// The array is a module global: every GPU that loads this part of the
// library holds it until the process exits.  Host code cannot use the
// array's name as a device address; on the first call on a device the entry
// point resolves the array's address with cudaGetSymbolAddress while that
// device is current, and passes that address to the kernels.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "sw_internal.h"
#include "swgb.h"

namespace swgb {
namespace {

constexpr int64_t kStaticMaxPairs = SW_STATIC_MAX_PAIRS;
constexpr int64_t kStaticMaxBoundaryWords = SW_STATIC_MAX_BOUNDARY_WORDS;

// Byte layout of the array.
constexpr size_t kOffCounters = 0;    // kMaxClasses queue heads + status word
constexpr size_t kOffStatus = 64;
constexpr size_t kOffClasses = 256;   // kMaxClasses ClassInfo
constexpr size_t kOffPairs = 512;     // group-path PairInfo table
constexpr size_t kOffPlain = kOffPairs + kStaticMaxPairs * sizeof(PairInfo);
constexpr size_t kOffBoundary = kOffPlain + kStaticMaxPairs * sizeof(PairInfo);
constexpr size_t kStaticBytes = kOffBoundary + kStaticMaxBoundaryWords * sizeof(uint32_t);
static_assert(kOffBoundary % 256 == 0, "boundary words must stay 256-byte aligned");
static_assert(kMaxClasses * sizeof(ClassInfo) <= kOffPairs - kOffClasses, "class table");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

std::mutex g_static_mu;
std::vector<unsigned char *> g_static_addr;  // device address per device, once resolved

int err(int code, const char *fmt, ...) {
    char buf[384];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return set_error(code, buf);
}

// Device address of the array on the current device (resolved once per device).
int static_address(int dev, unsigned char **out) {
    std::lock_guard<std::mutex> lk(g_static_mu);
    if ((int)g_static_addr.size() <= dev) g_static_addr.resize(dev + 1, nullptr);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            return err(SW_ECUDA, "sw_align_batch_static: cudaGetSymbolAddress: %s",
                       cudaGetErrorString(e));
        g_static_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_static_addr[dev];
    return SW_OK;
}

}  // namespace
}  // namespace swgb

using namespace swgb;

extern "C" int sw_align_batch_static(const uint8_t *q_seqs, const int64_t *q_offsets,
                                     const uint8_t *r_seqs, const int64_t *r_offsets,
                                     int32_t n_pairs, const int8_t *score_matrix,
                                     int32_t alphabet_size, int32_t gap_open,
                                     int32_t gap_extend, int32_t *out_score, int32_t *out_qend,
                                     int32_t *out_rend, int32_t *out_qstart,
                                     int32_t *out_rstart, void *stream) {
    if (n_pairs < 0) return err(SW_EINVAL, "sw_align_batch_static: n_pairs < 0");
    if (n_pairs == 0) return SW_OK;
    if (n_pairs > kStaticMaxPairs)
        return err(SW_ERANGE,
                   "sw_align_batch_static: %d pairs exceed the fixed limit of %lld per call; "
                   "split the batch",
                   n_pairs, (long long)kStaticMaxPairs);
    if (!q_offsets || !r_offsets || !score_matrix || !q_seqs || !r_seqs || !out_score ||
        !out_qend || !out_rend || !out_qstart || !out_rstart)
        return err(SW_EINVAL, "sw_align_batch_static: NULL pointer argument");
    if (alphabet_size < 1 || alphabet_size > SW_MAX_ALPHABET)
        return err(SW_EINVAL, "sw_align_batch_static: alphabet_size %d not in [1, %d]",
                   alphabet_size, SW_MAX_ALPHABET);
    if (gap_extend > 0 || gap_open > gap_extend || gap_open < -SW_MAX_GAP)
        return err(SW_EINVAL, "sw_align_batch_static: need -%d <= gap_open <= gap_extend <= 0",
                   SW_MAX_GAP);
    const int A = alphabet_size;
    int smax = -128, smin = 127;
    for (int i = 0; i < A * A; ++i) {
        smax = std::max(smax, (int)score_matrix[i]);
        smin = std::min(smin, (int)score_matrix[i]);
    }
    std::vector<int32_t> n(n_pairs), m(n_pairs);
    for (int32_t i = 0; i < n_pairs; ++i) {
        const int64_t a = q_offsets[i + 1] - q_offsets[i];
        const int64_t b = r_offsets[i + 1] - r_offsets[i];
        if (q_offsets[i] < 0 || r_offsets[i] < 0 || a < 0 || b < 0)
            return err(SW_ERANGE, "sw_align_batch_static: offsets of pair %d negative or decreasing",
                       i);
        if (a > SW_MAX_LEN || b > SW_MAX_LEN)
            return err(SW_ERANGE, "sw_align_batch_static: pair %d has lengths (%lld, %lld) > %d", i,
                       (long long)a, (long long)b, SW_MAX_LEN);
        n[i] = (int32_t)a;
        m[i] = (int32_t)b;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return err(SW_ECUDA, "sw_align_batch_static: no device");
    unsigned char *base = nullptr;
    int rc = static_address(dev, &base);
    if (rc != SW_OK) return rc;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return err(SW_ECUDA, "sw_align_batch_static: cannot read the SM count");

    ProfileKind kind = ProfileKind::kInt32;
    if (A > 4 && smax - gap_open <= 127 && smin - gap_open >= -127) kind = ProfileKind::kInt8;

    std::vector<PlanPair> gp;
    std::vector<int32_t> gid;
    std::vector<PairInfo> plain;
    int plain_max_n = 0;
    for (int32_t i = 0; i < n_pairs; ++i) {
        const bool scaled = group_path_eligible(n[i], m[i], smax, gap_open, gap_extend);
        if (!scaled) {
            plain.push_back({q_offsets[i], r_offsets[i], -1, n[i], m[i], i, 0});
            plain_max_n = std::max(plain_max_n, n[i]);
        } else {
            gp.push_back({(int32_t)gid.size(), n[i], m[i]});
            gid.push_back(i);
        }
    }
    int grid = 0, n_warps = 0;
    if (!gp.empty()) {
        int smem = 0;
        const int bps = group_blocks_per_sm(kind, A, &smem);
        if (bps <= 0) return err(SW_ECUDA, "sw_align_batch_static: group kernel does not fit");
        const int64_t want = ((int64_t)gp.size() + kGroupWarps - 1) / kGroupWarps;
        grid = (int)std::min<int64_t>((int64_t)bps * sms, want);
        n_warps = grid * kGroupWarps;
    }
    const std::vector<PlannedClass> planned = plan_classes(gp, n_warps, -1, 0.5);
    std::vector<PairInfo> pairs;
    std::vector<ClassInfo> classes;
    pairs.reserve(gp.size());
    int64_t words = 0;
    int warp_begin = 0;
    for (const PlannedClass &pc : planned) {
        classes.push_back({(int32_t)pairs.size(), (int32_t)pc.pairs.size(), pc.log2g, warp_begin});
        warp_begin += pc.warps;
        const int G = 1 << pc.log2g;
        for (int32_t k : pc.pairs) {
            const int32_t i = gid[k];
            PairInfo pi{q_offsets[i], r_offsets[i], -1, n[i], m[i], i, 0};
            if (n[i] > G * kRows && m[i] > 0) {
                pi.scratch = words;
                words += boundary_words(m[i]);
            }
            pairs.push_back(pi);
        }
    }
    if (words > kStaticMaxBoundaryWords)
        return err(SW_ERANGE,
                   "sw_align_batch_static: the batch needs %lld strip-boundary words, above the "
                   "fixed limit of %lld; split the batch",
                   (long long)words, (long long)kStaticMaxBoundaryWords);

    cudaStream_t s = (cudaStream_t)stream;
    int32_t *counters = reinterpret_cast<int32_t *>(base + kOffCounters);
    int32_t *status = reinterpret_cast<int32_t *>(base + kOffStatus);
    ClassInfo *d_classes = reinterpret_cast<ClassInfo *>(base + kOffClasses);
    PairInfo *d_pairs = reinterpret_cast<PairInfo *>(base + kOffPairs);
    PairInfo *d_plain = reinterpret_cast<PairInfo *>(base + kOffPlain);
    uint32_t *d_bnd = reinterpret_cast<uint32_t *>(base + kOffBoundary);
    // queue heads and the status word must start at zero on every call
    cudaError_t e = cudaMemsetAsync(base + kOffCounters, 0, kOffClasses - kOffCounters, s);
    if (e == cudaSuccess && !classes.empty())
        e = cudaMemcpyAsync(d_classes, classes.data(), classes.size() * sizeof(ClassInfo),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !pairs.empty())
        e = cudaMemcpyAsync(d_pairs, pairs.data(), pairs.size() * sizeof(PairInfo),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !plain.empty())
        e = cudaMemcpyAsync(d_plain, plain.data(), plain.size() * sizeof(PairInfo),
                            cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess)
        return err(SW_ECUDA, "sw_align_batch_static: table copy: %s", cudaGetErrorString(e));
    const Outputs o{out_score, out_qend, out_rend, out_qstart, out_rstart};
    if (!pairs.empty()) {
        GroupParams g;
        std::memset(&g, 0, sizeof g);
        g.q = q_seqs;
        g.r = r_seqs;
        g.pairs = d_pairs;
        g.classes = d_classes;
        g.n_classes = (int32_t)classes.size();
        g.counters = counters;
        g.n_warps = n_warps;
        g.scratch = d_bnd;
        g.status = status;
        g.out = o;
        g.alphabet = A;
        g.gap_open = gap_open;
        g.gap_extend = gap_extend;
        std::memcpy(g.mat, score_matrix, (size_t)A * A);
        e = launch_group(g, kind, grid, s);
        if (e != cudaSuccess)
            return err(SW_ECUDA, "sw_align_batch_static: launch: %s", cudaGetErrorString(e));
    }
    if (!plain.empty()) {
        PlainParams pp;
        std::memset(&pp, 0, sizeof pp);
        pp.q = q_seqs;
        pp.r = r_seqs;
        pp.pairs = d_plain;
        pp.n_pairs = (int32_t)plain.size();
        pp.status = status;
        pp.out = o;
        pp.alphabet = A;
        pp.gap_open = gap_open;
        pp.gap_extend = gap_extend;
        std::memcpy(pp.mat, score_matrix, (size_t)A * A);
        const bool wide = plain_max_n > 1024;
        e = launch_plain(pp, wide ? kPlainWideThreads : std::max(32, (plain_max_n + 31) / 32 * 32),
                         wide ? kPlainMaxRows : 1, s);
        if (e != cudaSuccess)
            return err(SW_ECUDA, "sw_align_batch_static: launch: %s", cudaGetErrorString(e));
    }
    return SW_OK;
}
