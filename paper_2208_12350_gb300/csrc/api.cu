// C ABI of the library: argument checks, host-side planning of a batch,
// launch sequencing and CUDA-graph replay.  Declarations and the contract
// of each entry point are in include/swgb.h.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "device_plan.h"
#include "sw_internal.h"
#include "swgb.h"

using namespace swgb;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define SW_CUDA_TRY(call)                                                          \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess)                                                     \
            return fail(SW_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));       \
    } while (0)

// Makes a device current for a scope and restores the previous one.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

namespace swgb {
// Records a failure message for sw_last_error() from other translation units.
int set_error(int code, const char *msg) {
    g_last_error = msg;
    return code;
}
}  // namespace swgb

struct sw_ctx {
    int device = 0;
    int sm_count = 0;
    char name[256] = {0};
    int32_t *d_status = nullptr;
    int narrow_log2g = -1;      // planner override: bulk lane-group width (log2), -1 = auto
    double cap_fraction = 0.5;  // planner override: long-pair cap (used with narrow_log2g)
    int form_arith = -1;        // batched kernel form: -1 auto, 0 scaled int32, 1 packed 16-bit
    int form_rows = 16;         // packed form with 32-bit profile words: 16 or 32 rows per lane
    int form_blocks = 0;        // resident blocks per SM of the batched kernel (0: as many as fit)
    // the device reads host memory through the host's page tables over a
    // coherent link (NVLink-C2C on Grace): pinned host inputs are read in
    // place (host_in_place), unless the caller asked for copies
    bool host_in_place_ok = false;
    bool host_in_place = false;
    std::mutex mu;
    std::vector<std::pair<sw_plan *, cudaEvent_t>> retired;
    // stream-ordered workspaces of the one-shot calls (created on first use;
    // keeps freed memory for the next call instead of returning it)
    cudaMemPool_t pool = nullptr;
    bool guards = false;  // guard regions around one-shot workspace parts
    // page-locked staging for host tables uploaded by asynchronous calls,
    // reused once the event of its last upload has completed
    void *pinned = nullptr;
    size_t pinned_cap = 0;
    cudaEvent_t pinned_ev = nullptr;
    std::mutex pinned_mu;
};

namespace swgb {
int ctx_device(const ::sw_ctx *ctx) { return ctx->device; }
}  // namespace swgb

struct sw_plan {
    sw_ctx *ctx = nullptr;
    int32_t n_pairs = 0;
    int A = 0, go = 0, ge = 0, mode = 0;
    uint32_t flags = 0;
    int8_t mat[kMaxAlphabet * kMaxAlphabet] = {0};
    HostPlan hp;        // tables (host copies) and launch shapes
    DeviceTables dev;   // the same tables on the device
    PairInfo *d_pairs = nullptr, *d_plain = nullptr;
    ClassInfo *d_classes = nullptr;
    int32_t *d_counter = nullptr;
    uint32_t *d_scratch = nullptr;
    // host-buffer execution: staging copies of the inputs and outputs
    uint8_t *d_q = nullptr, *d_r = nullptr;
    // packed plans: the inputs expanded to one byte per residue
    uint8_t *d_unq = nullptr, *d_unr = nullptr;
    int32_t *d_out = nullptr;
    // graph replay
    cudaGraphExec_t gexec = nullptr;
    const void *gkey[8] = {nullptr};
    // every device allocation (the pointers above are views into them), and
    // with SW_PLAN_GUARDS the guard regions around them
    std::vector<void *> raw;
    GuardList guards{};
};

static void plan_free(sw_plan *p) {
    if (!p) return;
    DeviceGuard g(p->ctx ? p->ctx->device : 0);
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    for (void *a : p->raw) cudaFree(a);
    delete p;
}

// A device buffer of `bytes` for plan p; with SW_PLAN_GUARDS, between two
// guard regions filled with the guard pattern.
static int plan_alloc(sw_plan *p, void **out, size_t bytes, const char *what) {
    *out = nullptr;
    const bool guarded = (p->flags & SW_PLAN_GUARDS) != 0;
    const size_t body = (bytes + 255) & ~(size_t)255;
    void *raw = nullptr;
    if (cudaMalloc(&raw, guarded ? body + 2 * kGuardBytes : std::max<size_t>(bytes, 1)) !=
        cudaSuccess) {
        cudaGetLastError();
        return fail(SW_ENOMEM, "sw_plan: allocation of %zu bytes (%s) failed", bytes, what);
    }
    p->raw.push_back(raw);
    if (!guarded) {
        *out = raw;
        return SW_OK;
    }
    unsigned char *b = static_cast<unsigned char *>(raw);
    if (p->guards.n + 2 > kMaxGuards) return fail(SW_EINVAL, "sw_plan: too many guarded buffers");
    SW_CUDA_TRY(cudaMemset(b, 0xA5, kGuardBytes));
    SW_CUDA_TRY(cudaMemset(b + kGuardBytes + body, 0xA5, kGuardBytes));
    for (unsigned char *g : {b, b + kGuardBytes + body}) {
        p->guards.ptr[p->guards.n] = reinterpret_cast<uint32_t *>(g);
        p->guards.words[p->guards.n] = (int32_t)(kGuardBytes / 4);
        ++p->guards.n;
    }
    *out = b + kGuardBytes;
    return SW_OK;
}

template <class T>
static int plan_upload(sw_plan *p, T **dst, const std::vector<T> &src, const char *what) {
    *dst = nullptr;
    if (src.empty()) return SW_OK;
    void *d = nullptr;
    const int rc = plan_alloc(p, &d, src.size() * sizeof(T), what);
    if (rc != SW_OK) return rc;
    *dst = static_cast<T *>(d);
    SW_CUDA_TRY(cudaMemcpy(d, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    return SW_OK;
}

static void reap_retired(sw_ctx *ctx, bool wait) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto &v = ctx->retired;
    for (size_t i = 0; i < v.size();) {
        cudaError_t q = wait ? cudaEventSynchronize(v[i].second) : cudaEventQuery(v[i].second);
        if (q == cudaSuccess || (q != cudaErrorNotReady)) {
            cudaEventDestroy(v[i].second);
            plan_free(v[i].first);
            v[i] = v.back();
            v.pop_back();
        } else {
            ++i;
        }
    }
    cudaGetLastError();  // clear a cudaErrorNotReady left by the query
}

extern "C" {

const char *sw_last_error(void) { return g_last_error.c_str(); }

int sw_ctx_create(int32_t device, sw_ctx **out) {
    if (!out) return fail(SW_EINVAL, "sw_ctx_create: out is NULL");
    *out = nullptr;
    int count = 0;
    SW_CUDA_TRY(cudaGetDeviceCount(&count));
    if (device < 0 || device >= count)
        return fail(SW_EINVAL, "sw_ctx_create: device %d not in [0, %d)", device, count);
    DeviceGuard g(device);
    if (!g.ok) return fail(SW_ECUDA, "cudaSetDevice(%d) failed", device);
    auto *ctx = new sw_ctx();
    ctx->device = device;
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) {
        delete ctx;
        return fail(SW_ECUDA, "cudaGetDeviceProperties: %s", cudaGetErrorString(e));
    }
    ctx->sm_count = prop.multiProcessorCount;
    snprintf(ctx->name, sizeof ctx->name, "%s", prop.name);
    int ats = 0;
    if (cudaDeviceGetAttribute(&ats, cudaDevAttrPageableMemoryAccessUsesHostPageTables, device) !=
        cudaSuccess) {
        cudaGetLastError();
        ats = 0;
    }
    ctx->host_in_place_ok = ats != 0;
    ctx->host_in_place = ctx->host_in_place_ok;
    if (cudaMalloc(&ctx->d_status, sizeof(int32_t)) != cudaSuccess ||
        cudaMemset(ctx->d_status, 0, sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(ctx->d_status);
        delete ctx;
        return fail(SW_ENOMEM, "sw_ctx_create: status word allocation failed");
    }
    *out = ctx;
    return SW_OK;
}

int sw_ctx_destroy(sw_ctx *ctx) {
    if (!ctx) return SW_OK;
    reap_retired(ctx, true);
    {
        DeviceGuard g(ctx->device);
        cudaFree(ctx->d_status);
        // outstanding one-shot workspaces are released when their frees complete
        if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
        if (ctx->pinned_ev) {
            cudaEventSynchronize(ctx->pinned_ev);
            cudaEventDestroy(ctx->pinned_ev);
        }
        cudaFreeHost(ctx->pinned);
    }
    delete ctx;
    return SW_OK;
}

int sw_ctx_sm_count(const sw_ctx *ctx, int32_t *out) {
    if (!ctx || !out) return fail(SW_EINVAL, "sw_ctx_sm_count: NULL argument");
    *out = ctx->sm_count;
    return SW_OK;
}

int sw_ctx_status(sw_ctx *ctx, int32_t *status) {
    if (!ctx || !status) return fail(SW_EINVAL, "sw_ctx_status: NULL argument");
    DeviceGuard g(ctx->device);
    SW_CUDA_TRY(cudaDeviceSynchronize());
    SW_CUDA_TRY(cudaMemcpy(status, ctx->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost));
    SW_CUDA_TRY(cudaMemset(ctx->d_status, 0, sizeof(int32_t)));
    return SW_OK;
}

int sw_ctx_set_form(sw_ctx *ctx, int32_t arith, int32_t rows, int32_t blocks_per_sm) {
    if (!ctx || arith < -1 || arith > 1 || (rows != 16 && rows != 32) || blocks_per_sm < 0 ||
        blocks_per_sm > 32)
        return fail(SW_EINVAL, "sw_ctx_set_form: bad argument");
    ctx->form_arith = arith;
    ctx->form_rows = rows;
    ctx->form_blocks = blocks_per_sm;
    return SW_OK;
}

int sw_ctx_get_tuning(const sw_ctx *ctx, int32_t *narrow_log2g, double *cap_fraction,
                      int32_t *arith, int32_t *rows, int32_t *blocks_per_sm) {
    if (!ctx) return fail(SW_EINVAL, "sw_ctx_get_tuning: ctx is NULL");
    if (narrow_log2g) *narrow_log2g = ctx->narrow_log2g;
    if (cap_fraction) *cap_fraction = ctx->cap_fraction;
    if (arith) *arith = ctx->form_arith;
    if (rows) *rows = ctx->form_rows;
    if (blocks_per_sm) *blocks_per_sm = ctx->form_blocks;
    return SW_OK;
}

int sw_ctx_set_guards(sw_ctx *ctx, int32_t on) {
    if (!ctx || (on != 0 && on != 1)) return fail(SW_EINVAL, "sw_ctx_set_guards: bad argument");
    ctx->guards = on != 0;
    return SW_OK;
}

int sw_ctx_set_tuning(sw_ctx *ctx, int32_t narrow_log2g, double cap_fraction) {
    if (!ctx || narrow_log2g < -1 || narrow_log2g > 5 || !(cap_fraction > 0))
        return fail(SW_EINVAL, "sw_ctx_set_tuning: bad argument");
    ctx->narrow_log2g = narrow_log2g;
    ctx->cap_fraction = cap_fraction;
    return SW_OK;
}

int sw_plan_create(sw_ctx *ctx, const int64_t *q_offsets, const int64_t *r_offsets,
                   int32_t n_pairs, const int8_t *score_matrix, int32_t alphabet_size,
                   int32_t gap_open, int32_t gap_extend, int32_t mode, uint32_t flags,
                   sw_plan **out) {
    if (!out) return fail(SW_EINVAL, "sw_plan_create: out is NULL");
    *out = nullptr;
    if (!ctx) return fail(SW_EINVAL, "sw_plan_create: ctx is NULL");
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(SW_ECUDA, "cudaSetDevice(%d) failed", ctx->device);
    reap_retired(ctx, false);
    auto *p = new sw_plan();
    p->ctx = ctx;
    p->flags = flags;
    std::string msg;
    int rc = make_host_plan(q_offsets, r_offsets, n_pairs, score_matrix, alphabet_size, gap_open,
                            gap_extend, mode, ctx->sm_count, ctx->narrow_log2g, ctx->cap_fraction,
                            &p->hp, &msg, 1, 8192,
                            (flags & SW_PLAN_NO_S16X2) == 0 && ctx->form_arith != 0,
                            group_blocks_per_sm, (flags & SW_PLAN_PAIR_SCRATCH) == 0,
                            (flags & SW_PLAN_ROWS32) != 0 || ctx->form_rows == 32,
                            ctx->form_blocks);
    if (rc != SW_OK) {
        delete p;
        return fail(rc, "sw_plan_create: %s", msg.c_str());
    }
    p->ctx = ctx;
    p->n_pairs = n_pairs;
    p->A = alphabet_size;
    p->go = gap_open;
    p->ge = gap_extend;
    p->mode = mode == SW_MODE_AUTO ? SW_MODE_BATCHED : mode;
    p->flags = flags;
    p->hp.ends_only = (flags & SW_PLAN_ENDS_ONLY) != 0;
    if (flags & SW_PLAN_PACKED_2BIT) {
        if (alphabet_size > 4) {
            plan_free(p);
            return fail(SW_EINVAL, "sw_plan_create: SW_PLAN_PACKED_2BIT needs alphabet_size <= 4");
        }
        void *uq = nullptr, *ur = nullptr;
        if ((rc = plan_alloc(p, &uq, (size_t)std::max<int64_t>(p->hp.q_bytes, 4), "inputs")) ||
            (rc = plan_alloc(p, &ur, (size_t)std::max<int64_t>(p->hp.r_bytes, 4), "inputs"))) {
            plan_free(p);
            return rc;
        }
        p->d_unq = static_cast<uint8_t *>(uq);
        p->d_unr = static_cast<uint8_t *>(ur);
    }
    std::memcpy(p->mat, score_matrix, (size_t)alphabet_size * alphabet_size);
    if ((rc = plan_upload(p, &p->d_pairs, p->hp.pairs, "pair table")) ||
        (rc = plan_upload(p, &p->d_classes, p->hp.classes, "class table")) ||
        (rc = plan_upload(p, &p->d_plain, p->hp.plain, "plain table"))) {
        plan_free(p);
        return rc;
    }
    void *cnt = nullptr, *scr = nullptr;
    if ((rc = plan_alloc(p, &cnt, kMaxClasses * sizeof(int32_t), "queue heads")) ||
        (p->hp.scratch_words > 0 &&
         (rc = plan_alloc(p, &scr, p->hp.scratch_words * sizeof(uint32_t), "scratch")))) {
        plan_free(p);
        return rc;
    }
    p->d_counter = static_cast<int32_t *>(cnt);
    p->d_scratch = static_cast<uint32_t *>(scr);
    p->dev.pairs = p->d_pairs;
    p->dev.classes = p->d_classes;
    p->dev.plain = p->d_plain;
    p->dev.counters = p->d_counter;
    p->dev.scratch = p->d_scratch;
    p->dev.status = ctx->d_status;
    *out = p;
    return SW_OK;
}

static int enqueue(sw_plan *p, const uint8_t *q, const uint8_t *r, const Outputs &o,
                   cudaStream_t s) {
    if (p->flags & SW_PLAN_PACKED_2BIT) {
        SW_CUDA_TRY(enqueue_unpack_2bit(q, p->hp.q_bytes, p->d_unq, p->ctx->sm_count, s));
        SW_CUDA_TRY(enqueue_unpack_2bit(r, p->hp.r_bytes, p->d_unr, p->ctx->sm_count, s));
        q = p->d_unq;
        r = p->d_unr;
    }
    SW_CUDA_TRY(enqueue_plan(p->hp, p->dev, q, r, o, p->mat, p->A, p->go, p->ge, s));
    // SW_PLAN_GUARDS: every guard word still holds the pattern
    if (p->guards.n) SW_CUDA_TRY(launch_guard_check(p->guards, p->ctx->d_status, s));
    return SW_OK;
}

int sw_plan_execute(sw_plan *p, const uint8_t *q_seqs, const uint8_t *r_seqs,
                    int32_t *out_score, int32_t *out_qend, int32_t *out_rend,
                    int32_t *out_qstart, int32_t *out_rstart, void *stream) {
    if (!p) return fail(SW_EINVAL, "sw_plan_execute: plan is NULL");
    if (p->n_pairs == 0) return SW_OK;
    if (!q_seqs || !r_seqs || !out_score || !out_qend || !out_rend ||
        (!p->hp.ends_only && (!out_qstart || !out_rstart)))
        return fail(SW_EINVAL, "sw_plan_execute: NULL device pointer");
    DeviceGuard g(p->ctx->device);
    if (!g.ok) return fail(SW_ECUDA, "cudaSetDevice(%d) failed", p->ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const Outputs o{out_score, out_qend, out_rend, out_qstart, out_rstart};
    const bool graph = (p->flags & SW_PLAN_GRAPH) && s != nullptr;
    if (!graph) return enqueue(p, q_seqs, r_seqs, o, s);
    const void *key[8] = {q_seqs, r_seqs, out_score, out_qend, out_rend, out_qstart, out_rstart,
                          stream};
    if (!p->gexec || std::memcmp(key, p->gkey, sizeof key) != 0) {
        if (p->gexec) {
            cudaGraphExecDestroy(p->gexec);
            p->gexec = nullptr;
        }
        SW_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        const int rc = enqueue(p, q_seqs, r_seqs, o, s);
        cudaGraph_t graph_obj = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(s, &graph_obj);
        if (rc != SW_OK) {
            if (graph_obj) cudaGraphDestroy(graph_obj);
            return rc;
        }
        if (ec != cudaSuccess) return fail(SW_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(ec));
        const cudaError_t ei = cudaGraphInstantiate(&p->gexec, graph_obj, 0);
        cudaGraphDestroy(graph_obj);
        if (ei != cudaSuccess) {
            p->gexec = nullptr;
            return fail(SW_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ei));
        }
        std::memcpy(p->gkey, key, sizeof key);
    }
    SW_CUDA_TRY(cudaGraphLaunch(p->gexec, s));
    return SW_OK;
}

// The device address of a pinned (page-locked, registered) host buffer when
// the context reads host inputs in place, else NULL.
static const uint8_t *host_view(const sw_ctx *ctx, const uint8_t *h) {
    if (!ctx->host_in_place || !h) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    return static_cast<const uint8_t *>(a.devicePointer);
}

int sw_ctx_host_in_place(const sw_ctx *ctx, int32_t *yes) {
    if (!ctx || !yes) return fail(SW_EINVAL, "sw_ctx_host_in_place: NULL argument");
    *yes = ctx->host_in_place ? 1 : 0;
    return SW_OK;
}

int sw_ctx_set_host_in_place(sw_ctx *ctx, int32_t enable) {
    if (!ctx || (enable != 0 && enable != 1))
        return fail(SW_EINVAL, "sw_ctx_set_host_in_place: bad argument");
    ctx->host_in_place = enable != 0 && ctx->host_in_place_ok;
    return SW_OK;
}

int sw_plan_execute_host(sw_plan *p, const uint8_t *q_seqs, const uint8_t *r_seqs,
                         int32_t *out_host, void *stream) {
    if (!p) return fail(SW_EINVAL, "sw_plan_execute_host: plan is NULL");
    if (p->n_pairs == 0) return SW_OK;
    if ((p->hp.q_bytes > 0 && !q_seqs) || (p->hp.r_bytes > 0 && !r_seqs) || !out_host)
        return fail(SW_EINVAL, "sw_plan_execute_host: NULL host pointer");
    DeviceGuard g(p->ctx->device);
    if (!g.ok) return fail(SW_ECUDA, "cudaSetDevice(%d) failed", p->ctx->device);
    // packed plans take a quarter of the bytes (four residues per byte)
    const bool packed = (p->flags & SW_PLAN_PACKED_2BIT) != 0;
    const int64_t qb = packed ? (p->hp.q_bytes + 3) / 4 : p->hp.q_bytes;
    const int64_t rb = packed ? (p->hp.r_bytes + 3) / 4 : p->hp.r_bytes;
    if (!p->d_out) {
        void *dq = nullptr, *dr = nullptr, *dout = nullptr;
        int rc0;
        if ((rc0 = plan_alloc(p, &dq, (size_t)std::max<int64_t>(qb, 1), "staging")) ||
            (rc0 = plan_alloc(p, &dr, (size_t)std::max<int64_t>(rb, 1), "staging")) ||
            (rc0 = plan_alloc(p, &dout, (size_t)5 * p->n_pairs * sizeof(int32_t), "staging")))
            return rc0;
        p->d_q = static_cast<uint8_t *>(dq);
        p->d_r = static_cast<uint8_t *>(dr);
        p->d_out = static_cast<int32_t *>(dout);
    }
    cudaStream_t s = (cudaStream_t)stream;
    // Pinned host inputs on a coherent host link are read by the kernels in
    // place (each residue crosses the link once, during the alignment);
    // otherwise they are copied into the plan's staging buffers first.
    const uint8_t *q_in = host_view(p->ctx, q_seqs), *r_in = host_view(p->ctx, r_seqs);
    if (!q_in || !r_in) {
        if (qb > 0) SW_CUDA_TRY(cudaMemcpyAsync(p->d_q, q_seqs, qb, cudaMemcpyHostToDevice, s));
        if (rb > 0) SW_CUDA_TRY(cudaMemcpyAsync(p->d_r, r_seqs, rb, cudaMemcpyHostToDevice, s));
        q_in = p->d_q;
        r_in = p->d_r;
    }
    const int64_t n = p->n_pairs;
    int rc = sw_plan_execute(p, q_in, r_in, p->d_out, p->d_out + n, p->d_out + 2 * n,
                             p->d_out + 3 * n, p->d_out + 4 * n, stream);
    if (rc != SW_OK) return rc;
    // with SW_PLAN_ENDS_ONLY the start rows are not computed and not copied
    const int rows = p->hp.ends_only ? 3 : 5;
    SW_CUDA_TRY(cudaMemcpyAsync(out_host, p->d_out, (size_t)rows * n * sizeof(int32_t),
                                cudaMemcpyDeviceToHost, s));
    SW_CUDA_TRY(cudaStreamSynchronize(s));
    return SW_OK;
}

int sw_plan_info(const sw_plan *p, int32_t *n_group_pairs, int32_t *n_plain, int32_t *launches,
                 int64_t *scratch_bytes) {
    if (!p) return fail(SW_EINVAL, "sw_plan_info: plan is NULL");
    if (n_group_pairs) *n_group_pairs = (int32_t)p->hp.pairs.size();
    if (n_plain) *n_plain = (int32_t)p->hp.plain.size();
    if (launches)
        *launches = (p->hp.pairs.empty() ? 0 : 1) + (p->hp.plain.empty() ? 0 : 1) +
                    ((p->flags & SW_PLAN_PACKED_2BIT) ? 2 : 0);
    if (scratch_bytes) *scratch_bytes = p->hp.scratch_words * (int64_t)sizeof(uint32_t);
    return SW_OK;
}

int sw_plan_arith(const sw_plan *p, int32_t *arith) {
    if (!p || !arith) return fail(SW_EINVAL, "sw_plan_arith: NULL argument");
    *arith = (!p->hp.pairs.empty() && is_packed(p->hp.kind)) ? SW_ARITH_S16X2 : SW_ARITH_S32;
    return SW_OK;
}

int sw_plan_rows(const sw_plan *p, int32_t *rows) {
    if (!p || !rows) return fail(SW_EINVAL, "sw_plan_rows: NULL argument");
    *rows = rows_of(p->hp.kind);
    return SW_OK;
}

int sw_plan_poison_guard(sw_plan *p, int32_t region) {
    if (!p || region < 0 || region >= p->guards.n)
        return fail(SW_EINVAL, "sw_plan_poison_guard: no guard region %d", region);
    DeviceGuard g(p->ctx->device);
    const uint32_t word = ~kGuardWord;
    SW_CUDA_TRY(cudaDeviceSynchronize());
    SW_CUDA_TRY(cudaMemcpy(p->guards.ptr[region] + p->guards.words[region] / 2, &word,
                           sizeof word, cudaMemcpyHostToDevice));
    return SW_OK;
}

int sw_plan_destroy(sw_plan *p) {
    plan_free(p);
    return SW_OK;
}

// The context's pool of one-shot workspaces (created on first use).
static int ctx_pool(sw_ctx *ctx, cudaMemPool_t *out) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!ctx->pool) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = ctx->device;
        cudaMemPool_t pool = nullptr;
        SW_CUDA_TRY(cudaMemPoolCreate(&pool, &props));
        uint64_t keep = UINT64_MAX;
        const cudaError_t e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return fail(SW_ECUDA, "cudaMemPoolSetAttribute: %s", cudaGetErrorString(e));
        }
        ctx->pool = pool;
    }
    *out = ctx->pool;
    return SW_OK;
}

int sw_align_batch_ex(sw_ctx *ctx, const uint8_t *q_seqs, const int64_t *q_offsets,
                      const uint8_t *r_seqs, const int64_t *r_offsets, int32_t n_pairs,
                      const int8_t *score_matrix, int32_t alphabet_size, int32_t gap_open,
                      int32_t gap_extend, int32_t mode, int32_t *out_score, int32_t *out_qend,
                      int32_t *out_rend, int32_t *out_qstart, int32_t *out_rstart,
                      void *stream) {
    if (!ctx) return fail(SW_EINVAL, "sw_align_batch_ex: ctx is NULL");
    if (n_pairs < 0) return fail(SW_EINVAL, "sw_align_batch_ex: n_pairs < 0");
    if (n_pairs == 0) return SW_OK;
    if (!q_offsets || !r_offsets) return fail(SW_EINVAL, "sw_align_batch_ex: offsets are NULL");
    if (!q_seqs || !r_seqs || !out_score || !out_qend || !out_rend || !out_qstart || !out_rstart)
        return fail(SW_EINVAL, "sw_align_batch_ex: NULL device pointer");
    if (!score_matrix) return fail(SW_EINVAL, "sw_align_batch_ex: score_matrix is NULL");
    if (alphabet_size < 1 || alphabet_size > SW_MAX_ALPHABET)
        return fail(SW_EINVAL, "sw_align_batch_ex: alphabet_size %d not in [1, %d]", alphabet_size,
                    SW_MAX_ALPHABET);
    if (gap_extend > 0 || gap_open > gap_extend || gap_open < -SW_MAX_GAP)
        return fail(SW_EINVAL, "sw_align_batch_ex: need -%d <= gap_open <= gap_extend <= 0",
                    SW_MAX_GAP);
    if (mode != SW_MODE_AUTO && mode != SW_MODE_PLAIN && mode != SW_MODE_BATCHED)
        return fail(SW_EINVAL, "sw_align_batch_ex: unknown mode %d", mode);
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(SW_ECUDA, "cudaSetDevice(%d) failed", ctx->device);
    if (ctx->host_in_place) {
        // page-locked host inputs are read in place (their device view)
        auto view = [&](const void *h) -> const void * {
            const uint8_t *d = host_view(ctx, static_cast<const uint8_t *>(h));
            return d ? static_cast<const void *>(d) : h;
        };
        q_seqs = static_cast<const uint8_t *>(view(q_seqs));
        r_seqs = static_cast<const uint8_t *>(view(r_seqs));
        q_offsets = static_cast<const int64_t *>(view(q_offsets));
        r_offsets = static_cast<const int64_t *>(view(r_offsets));
    }
    reap_retired(ctx, false);
    DevicePlanShape shape;
    std::string msg;
    int rc = device_plan_shape(n_pairs, score_matrix, alphabet_size, gap_open, gap_extend, mode,
                               ctx->sm_count, ctx->narrow_log2g, ctx->cap_fraction,
                               kOneShotSlotWords, &shape, &msg);
    if (rc != SW_OK) return fail(rc, "sw_align_batch_ex: %s", msg.c_str());
    shape.guards = ctx->guards ? 1 : 0;
    cudaMemPool_t pool = nullptr;
    if ((rc = ctx_pool(ctx, &pool)) != SW_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    void *ws = nullptr;
    const size_t bytes = device_plan_workspace_bytes(shape);
    if (cudaMallocFromPoolAsync(&ws, bytes, pool, s) != cudaSuccess) {
        cudaGetLastError();
        return fail(SW_ENOMEM, "sw_align_batch_ex: workspace of %zu bytes", bytes);
    }
    const Outputs o{out_score, out_qend, out_rend, out_qstart, out_rstart};
    const cudaError_t e =
        enqueue_device_plan(shape, ws, q_offsets, r_offsets, q_seqs, r_seqs, o, ctx->d_status, s);
    // stream-ordered: released after the kernels that use it, also on failure
    cudaFreeAsync(ws, s);
    if (e != cudaSuccess) return fail(SW_ECUDA, "sw_align_batch_ex: %s", cudaGetErrorString(e));
    return SW_OK;
}

static std::mutex g_default_mu;
static std::vector<sw_ctx *> g_default_ctx;

int sw_default_ctx(int32_t device, sw_ctx **out) {
    if (!out) return fail(SW_EINVAL, "sw_default_ctx: out is NULL");
    *out = nullptr;
    int count = 0;
    SW_CUDA_TRY(cudaGetDeviceCount(&count));
    if (device < 0 || device >= count)
        return fail(SW_EINVAL, "sw_default_ctx: device %d not in [0, %d)", device, count);
    std::lock_guard<std::mutex> lk(g_default_mu);
    if ((int)g_default_ctx.size() <= device) g_default_ctx.resize(device + 1, nullptr);
    if (!g_default_ctx[device]) {
        const int rc = sw_ctx_create(device, &g_default_ctx[device]);
        if (rc != SW_OK) return rc;
    }
    *out = g_default_ctx[device];
    return SW_OK;
}

int sw_align_batch(const uint8_t *q_seqs, const int64_t *q_offsets, const uint8_t *r_seqs,
                   const int64_t *r_offsets, int32_t n_pairs, const int8_t *score_matrix,
                   int32_t alphabet_size, int32_t gap_open, int32_t gap_extend,
                   int32_t *out_score, int32_t *out_qend, int32_t *out_rend,
                   int32_t *out_qstart, int32_t *out_rstart, void *stream) {
    int dev = 0;
    SW_CUDA_TRY(cudaGetDevice(&dev));
    sw_ctx *ctx = nullptr;
    const int rc = sw_default_ctx(dev, &ctx);
    if (rc != SW_OK) return rc;
    return sw_align_batch_ex(ctx, q_seqs, q_offsets, r_seqs, r_offsets, n_pairs, score_matrix,
                             alphabet_size, gap_open, gap_extend, SW_MODE_AUTO, out_score,
                             out_qend, out_rend, out_qstart, out_rstart, stream);
}

int sw_check_residues(const uint8_t *seqs, int64_t n, int32_t alphabet_size, int64_t *bad_count,
                      void *stream) {
    if (n < 0 || !bad_count || (n > 0 && !seqs))
        return fail(SW_EINVAL, "sw_check_residues: bad argument");
    if (alphabet_size < 1 || alphabet_size > SW_MAX_ALPHABET)
        return fail(SW_EINVAL, "sw_check_residues: bad alphabet size");
    SW_CUDA_TRY(launch_check_residues(seqs, n, alphabet_size,
                                      reinterpret_cast<unsigned long long *>(bad_count),
                                      (cudaStream_t)stream));
    return SW_OK;
}

}  // extern "C"

namespace swgb {
// Stream-ordered device memory from the context's workspace pool (released
// with cudaFreeAsync on the same stream).
int ctx_alloc_async(sw_ctx *ctx, size_t bytes, cudaStream_t s, void **out) {
    *out = nullptr;
    cudaMemPool_t pool = nullptr;
    const int rc = ctx_pool(ctx, &pool);
    if (rc != SW_OK) return rc;
    if (cudaMallocFromPoolAsync(out, std::max<size_t>(bytes, 256), pool, s) != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
        return set_error(SW_ENOMEM, "workspace allocation from the context's pool failed");
    }
    return SW_OK;
}

// Copies `bytes` of host data to device memory `dst` on stream s through the
// context's page-locked staging buffer (asynchronous DMA; the buffer is
// reused only after its previous upload has completed).
int ctx_pinned_acquire(sw_ctx *ctx, size_t bytes, void **host) {
    ctx->pinned_mu.lock();
    if (ctx->pinned_ev) {
        if (cudaEventSynchronize(ctx->pinned_ev) != cudaSuccess) {
            ctx->pinned_mu.unlock();
            return set_error(SW_ECUDA, "staging event wait failed");
        }
    } else if (cudaEventCreateWithFlags(&ctx->pinned_ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        ctx->pinned_mu.unlock();
        return set_error(SW_ECUDA, "staging event creation failed");
    }
    if (ctx->pinned_cap < bytes) {
        cudaFreeHost(ctx->pinned);
        ctx->pinned = nullptr;
        ctx->pinned_cap = 0;
        const size_t cap = std::max(bytes, (size_t)1 << 20);
        if (cudaMallocHost(&ctx->pinned, cap) != cudaSuccess) {
            cudaGetLastError();
            ctx->pinned_mu.unlock();
            return set_error(SW_ENOMEM, "page-locked staging allocation failed");
        }
        ctx->pinned_cap = cap;
    }
    *host = ctx->pinned;
    return SW_OK;
}

int ctx_pinned_commit(sw_ctx *ctx, void *dst, size_t bytes, cudaStream_t s) {
    int rc = SW_OK;
    if (bytes > 0 &&
        (cudaMemcpyAsync(dst, ctx->pinned, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
         cudaEventRecord(ctx->pinned_ev, s) != cudaSuccess)) {
        cudaGetLastError();
        rc = set_error(SW_ECUDA, "staged upload failed");
    }
    ctx->pinned_mu.unlock();
    return rc;
}

void ctx_pinned_release(sw_ctx *ctx) { ctx->pinned_mu.unlock(); }

int ctx_upload_async(sw_ctx *ctx, void *dst, const void *src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return SW_OK;
    void *host = nullptr;
    const int rc = ctx_pinned_acquire(ctx, bytes, &host);
    if (rc != SW_OK) return rc;
    std::memcpy(host, src, bytes);
    return ctx_pinned_commit(ctx, dst, bytes, s);
}
}  // namespace swgb
