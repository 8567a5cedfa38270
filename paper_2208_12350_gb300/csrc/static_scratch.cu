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
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return err(SW_ECUDA, "sw_align_batch_static: no device");
    {
        // the pair tables are copied from host memory that is freed when the
        // call returns, so a captured copy would read freed memory on replay
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess)
            return err(SW_ECUDA, "sw_align_batch_static: cudaStreamIsCapturing failed");
        if (cs != cudaStreamCaptureStatusNone)
            return err(SW_EINVAL, "sw_align_batch_static: the stream is being captured; "
                                  "this call cannot be captured into a CUDA graph");
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return err(SW_ECUDA, "sw_align_batch_static: cannot read the SM count");
    HostPlan hp;
    std::string msg;
    int rc = make_host_plan(q_offsets, r_offsets, n_pairs, score_matrix, alphabet_size, gap_open,
                            gap_extend, SW_MODE_AUTO, sms, -1, 0.5, &hp, &msg);
    if (rc != SW_OK) return err(rc, "sw_align_batch_static: %s", msg.c_str());
    if (hp.scratch_words > kStaticMaxBoundaryWords)
        return err(SW_ERANGE,
                   "sw_align_batch_static: the batch needs %lld strip-boundary words, above the "
                   "fixed limit of %lld; split the batch",
                   (long long)hp.scratch_words, (long long)kStaticMaxBoundaryWords);
    unsigned char *base = nullptr;
    rc = static_address(dev, &base);
    if (rc != SW_OK) return rc;

    cudaStream_t s = (cudaStream_t)stream;
    DeviceTables t;
    t.counters = reinterpret_cast<int32_t *>(base + kOffCounters);
    t.status = reinterpret_cast<int32_t *>(base + kOffStatus);
    t.classes = reinterpret_cast<ClassInfo *>(base + kOffClasses);
    t.pairs = reinterpret_cast<PairInfo *>(base + kOffPairs);
    t.plain = reinterpret_cast<PairInfo *>(base + kOffPlain);
    t.scratch = reinterpret_cast<uint32_t *>(base + kOffBoundary);
    // enqueue_plan zeroes the queue heads itself; the status word (zero at
    // load) collects the bits of every call until sw_static_status reads it
    cudaError_t e = cudaSuccess;
    if (!hp.classes.empty())
        e = cudaMemcpyAsync(const_cast<ClassInfo *>(t.classes), hp.classes.data(),
                            hp.classes.size() * sizeof(ClassInfo), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !hp.pairs.empty())
        e = cudaMemcpyAsync(const_cast<PairInfo *>(t.pairs), hp.pairs.data(),
                            hp.pairs.size() * sizeof(PairInfo), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !hp.plain.empty())
        e = cudaMemcpyAsync(const_cast<PairInfo *>(t.plain), hp.plain.data(),
                            hp.plain.size() * sizeof(PairInfo), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess)
        return err(SW_ECUDA, "sw_align_batch_static: table copy: %s", cudaGetErrorString(e));
    const Outputs o{out_score, out_qend, out_rend, out_qstart, out_rstart};
    e = enqueue_plan(hp, t, q_seqs, r_seqs, o, score_matrix, alphabet_size, gap_open, gap_extend,
                     s);
    if (e != cudaSuccess)
        return err(SW_ECUDA, "sw_align_batch_static: launch: %s", cudaGetErrorString(e));
    return SW_OK;
}

// The status word the kernels of sw_align_batch_static set (bit 0: a reverse
// pass did not reproduce its forward score), read after the stream's work and
// cleared; nothing is allocated (the copy lands in the caller's host word).
extern "C" int sw_static_status(int32_t *status, void *stream) {
    if (!status) return err(SW_EINVAL, "sw_static_status: status is NULL");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return err(SW_ECUDA, "sw_static_status: no device");
    unsigned char *base = nullptr;
    int rc = static_address(dev, &base);
    if (rc != SW_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    int32_t word = 0;
    cudaError_t e = cudaMemcpyAsync(&word, base + kOffStatus, sizeof word, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + kOffStatus, 0, sizeof(int32_t), s);
    if (e != cudaSuccess)
        return err(SW_ECUDA, "sw_static_status: %s", cudaGetErrorString(e));
    *status = word;
    return SW_OK;
}
