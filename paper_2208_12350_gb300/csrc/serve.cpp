// Serving loop: continuous batching of alignment requests.
//
// A request is a batch of pairs: either given on the host (sw_server_submit
// checks it and copies its sequences into a pinned staging pool) or a range
// of pairs of a resident pool (sw_server_add_pool uploads a batch once into
// the device budget; sw_server_submit_pool names a pair range of it, so only
// offsets and results move).  A worker thread turns the queue into
// launches: whenever a stream slot is free it takes the oldest queued
// request together with the later queued requests from the same source (the
// same pool, or staged sequences with the same scoring), up to a cap on
// pairs and cells and to what the device arena has left, and runs them as
// one batch (pairs are independent, so a pair's results do not depend on
// its batch mates) on the slot's stream: the merged offsets and any staged
// sequences copied into one arena block, the device planner's kernels (the
// one-shot call's: routes, lane-group widths, longest-first radix sort,
// queue tables) and the alignment kernels, then each request's outputs
// copied back into its staging area.  The host does no planning: it only
// sizes the grid, for latency (up to one warp per pair) on an idle GPU and
// for throughput (sixteen pairs per warp) while other launches run.  Under
// heavy load the queue grows between launches, so each launch takes many
// requests and runs at the batched kernel's throughput.  Launches are
// enqueued by eight helper threads; when a launch's completion event fires
// the worker frees its arena block and slot and wakes the waiters.
//
// Every wait is bounded: sw_server_wait and the submit calls take a timeout
// and return SW_ETIMEOUT instead of blocking forever.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "device_plan.h"
#include "sw_internal.h"
#include "swgb.h"

namespace swgb {
namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// First-fit allocator over [0, size) in kAlign units.
class Arena {
  public:
    explicit Arena(size_t size) : size_(size) { free_[0] = size; }
    bool alloc(size_t n, size_t *off) {
        n = align_up(std::max<size_t>(n, 1));
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n, at = it->first + n;
                free_.erase(it);
                if (rest) free_[at] = rest;
                used_ += n;
                peak_ = std::max(peak_, used_);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n) {
        n = align_up(std::max<size_t>(n, 1));
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }
    size_t size() const { return size_; }
    size_t largest_free() const {
        size_t b = 0;
        for (const auto &f : free_) b = std::max(b, f.second);
        return b;
    }

  private:
    size_t size_, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
};

// Caps on one launch: enough pairs to fill the GPU many times over, few
// enough cells that a small request merged into it still returns quickly.
constexpr int64_t kLaunchMaxPairs = 1 << 18;
constexpr double kLaunchMaxCells = 4e9;

struct Request {
    int64_t id = 0;
    int n_pairs = 0;
    int A = 0, go = 0, ge = 0;
    int8_t mat[kMaxAlphabet * kMaxAlphabet] = {0};
    std::vector<int64_t> q_off, r_off;  // the request's own CSR offsets
    int64_t q_bytes = 0, r_bytes = 0;
    double cells = 0;
    // staging pool layout: q | r | out (5 x n_pairs int32)
    size_t stage_off = 0, st_q = 0, st_r = 0, st_out = 0, st_total = 0;
    bool done = false;
    int status = SW_OK;
    int64_t done_ns = 0;  // CLOCK_MONOTONIC when the worker saw it finish
    // resident-pool request: pairs [first, first + n_pairs) of pool `pool`
    // (-1: the request's own sequences, staged at submission)
    int pool = -1;
    int64_t first = 0;
    int64_t lmax = 0;  // longest sequence of the request's pairs
};

bool same_scoring(const Request &a, const Request &b) {
    return a.A == b.A && a.go == b.go && a.ge == b.ge &&
           std::memcmp(a.mat, b.mat, (size_t)a.A * a.A) == 0;
}

// Requests that one launch can merge: the same resident pool, or both with
// staged sequences and the same scoring.
bool same_source(const Request &a, const Request &b) {
    return a.pool == b.pool && (a.pool >= 0 || same_scoring(a, b));
}

// A batch of pairs kept on the device for the server's lifetime, in one
// arena block (query residues, then reference residues); requests name
// pair ranges of it and move only offsets and results.
struct Pool {
    int A = 0, go = 0, ge = 0;
    int8_t mat[kMaxAlphabet * kMaxAlphabet] = {0};
    size_t dev_off = 0, dev_bytes = 0;
    size_t r_at = 0;                    // reference residues' offset in the block
    std::vector<int64_t> q_off, r_off;  // n_pairs + 1 each, from the block's q / r start
    int64_t n_pairs = 0;
};

// Byte layout of one launch's arena block: staged sequences, the pairs'
// start (and, for pool launches, end) offsets, the device planner's
// workspace (tables, sort buffers, strip-boundary slots) and the outputs.
struct Layout {
    size_t q = 0, r = 0, qo = 0, ro = 0, qe = 0, re = 0, ws = 0, out = 0, total = 0;
    size_t offsets_bytes = 0;  // the offset arrays, contiguous from qo
};

Layout layout_of(const DevicePlanShape &shape, int64_t n_pairs, size_t q_bytes, size_t r_bytes,
                 bool pooled) {
    Layout L;
    size_t at = 0;
    auto take = [&](size_t bytes) {
        const size_t o = at;
        at = align_up(at + bytes);
        return o;
    };
    L.q = take(q_bytes);
    L.r = take(r_bytes);
    const size_t arr = (size_t)(n_pairs + 1) * sizeof(int64_t);
    L.qo = take(arr);
    L.ro = take(arr);
    if (pooled) {
        L.qe = take(arr);
        L.re = take(arr);
    }
    L.offsets_bytes = at - L.qo;
    L.ws = take(device_plan_workspace_bytes(shape));
    L.out = take((size_t)5 * n_pairs * sizeof(int32_t));
    L.total = at;
    return L;
}

// Launches are planned on the device; the host only sizes the grid and the
// strip-boundary slots: up to one warp per pair on an idle GPU (latency:
// the planner then gives pairs wide groups, so slots sized for 32-lane
// groups of the launch's longest sequence), sixteen pairs per warp while
// other launches run (throughput: slots for 2-lane groups, at most the
// one-shot call's).  A pair whose need exceeds the slots takes wider groups.
int launch_shape(const Request &head, int64_t n_pairs, int64_t lmax, int sms, bool gpu_busy,
                 DevicePlanShape *shape, std::string *msg) {
    const int64_t bw = 2 * ((lmax + 3) & ~(int64_t)3) + 4;
    const int G = gpu_busy ? 2 : 32;
    const int64_t slot = std::min<int64_t>(((bw + G - 1) / G + 3) & ~(int64_t)3, kOneShotSlotWords);
    return device_plan_shape((int32_t)n_pairs, head.mat, head.A, head.go, head.ge, SW_MODE_AUTO,
                             sms, -1, 0.5, (int)slot, shape, msg, gpu_busy ? (32 >> kMinLog2G) : 1);
}

struct Launch {
    std::vector<std::shared_ptr<Request>> reqs;
    size_t dev_off = 0, dev_bytes = 0;
    int slot = -1;
    bool gpu_busy = false;  // other launches were on the GPU when it was formed
    bool enqueued = false;  // its work and completion event are on the stream
};

// Helper threads: a launch's host work (staging copies, table uploads and
// the enqueue of its kernels) runs on these, several launches at once,
// while the worker keeps admitting and retiring.
constexpr int kPlanners = 8;

}  // namespace
}  // namespace swgb

using namespace swgb;

struct sw_server {
    sw_ctx *ctx = nullptr;
    int device = 0, sms = 0;
    unsigned char *d_arena = nullptr, *h_pool = nullptr;
    int32_t *d_status = nullptr;
    std::unique_ptr<Arena> arena, staging;  // device budget, pinned staging pool
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    std::vector<std::unique_ptr<Launch>> slots;  // in flight, by slot
    std::vector<unsigned char *> h_tables;       // pinned per-slot offset buffers
    std::vector<size_t> h_tables_cap;
    std::vector<std::unique_ptr<Pool>> pools;   // resident pools, by id
    std::deque<std::shared_ptr<Request>> queue;  // oldest first
    std::unordered_map<int64_t, std::shared_ptr<Request>> all;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_space;
    std::thread worker;
    std::vector<std::thread> planners;
    std::deque<Launch *> plan_queue;   // formed, waiting for a planner
    std::condition_variable cv_plan;
    bool stop = false, stop_planners = false;
    int64_t next_id = 1, completed = 0, launches = 0, pairs_launched = 0;
    double plan_ms = 0;  // host time spent planning launches
    std::string worker_error;
};

// Pops the requests of the next launch from the queue (the oldest request
// and later ones from the same source - the same resident pool, or staged
// sequences with the same scoring - within the caps and the arena's
// largest free block) and returns the block size the launch needs.
// Caller holds the mutex.
static std::vector<std::shared_ptr<Request>> take_batch(sw_server *S, bool gpu_busy,
                                                        size_t *bytes_out) {
    std::vector<std::shared_ptr<Request>> out;
    const size_t room = S->arena->largest_free();
    size_t bytes = 0, qb = 0, rb = 0;
    int64_t pairs = 0, lmax = 0;
    double cells = 0;
    for (auto it = S->queue.begin(); it != S->queue.end();) {
        const auto &r = *it;
        if (!out.empty() && !same_source(*out.front(), *r)) {
            ++it;
            continue;
        }
        if (!out.empty() && (pairs + r->n_pairs > kLaunchMaxPairs ||
                             cells + r->cells > kLaunchMaxCells))
            break;
        DevicePlanShape shape;
        std::string msg;
        const Request &head = out.empty() ? *r : *out.front();
        if (launch_shape(head, pairs + r->n_pairs, std::max(lmax, r->lmax), S->sms, gpu_busy,
                         &shape, &msg) != SW_OK)
            break;
        const size_t b = layout_of(shape, pairs + r->n_pairs, qb + (size_t)r->q_bytes,
                                   rb + (size_t)r->r_bytes, r->pool >= 0)
                             .total;
        if (b > room) break;
        bytes = b;
        lmax = std::max(lmax, r->lmax);
        pairs += r->n_pairs;
        qb += (size_t)r->q_bytes;
        rb += (size_t)r->r_bytes;
        cells += r->cells;
        out.push_back(r);
        it = S->queue.erase(it);
    }
    *bytes_out = bytes;
    return out;
}

static void fail_launch(sw_server *S, Launch &L, cudaError_t e, int slot) {
    S->worker_error = cudaGetErrorString(e);
    for (auto &r : L.reqs) r->status = SW_ECUDA;
    cudaStreamSynchronize(S->streams[slot]);
    cudaGetLastError();
    cudaEventRecord(S->events[slot], S->streams[slot]);
}

// Plans and enqueues one launch on the slot's stream: the merged offsets go
// up through the slot's pinned buffer, staged sequences from the staging
// pool (a pool launch reads its pool's resident sequences instead), then the
// device planner and the alignment kernels run on the stream, and each
// request's outputs come back with one strided copy.  Called with the mutex
// released: only this thread touches the slot and the launch.
static void start_launch(sw_server *S, Launch &L, int slot, bool gpu_busy) {
    cudaStream_t s = S->streams[slot];
    const Request &head = *L.reqs.front();
    const Pool *pool = head.pool >= 0 ? S->pools[(size_t)head.pool].get() : nullptr;
    const auto t_plan = std::chrono::steady_clock::now();
    int64_t n = 0, lmax = 0;
    size_t qb_total = 0, rb_total = 0;
    for (auto &r : L.reqs) {
        n += r->n_pairs;
        lmax = std::max(lmax, r->lmax);
        qb_total += (size_t)r->q_bytes;
        rb_total += (size_t)r->r_bytes;
    }
    DevicePlanShape shape;
    std::string msg;
    int rc = launch_shape(head, n, lmax, S->sms, gpu_busy, &shape, &msg);
    const Layout Lay = layout_of(shape, n, qb_total, rb_total, pool != nullptr);
    if (rc != SW_OK || Lay.total > L.dev_bytes) {
        // cannot happen for a launch sized by take_batch; fail loudly
        S->worker_error = rc != SW_OK ? msg : "launch exceeds its arena block";
        for (auto &r : L.reqs) r->status = rc != SW_OK ? rc : SW_ENOMEM;
        cudaEventRecord(S->events[slot], s);
        return;
    }
    // the offsets, built in the slot's pinned buffer (the slot is idle, so
    // the buffer's previous contents are no longer being copied)
    const size_t tb = Lay.offsets_bytes;
    if (S->h_tables_cap[slot] < tb) {
        cudaFreeHost(S->h_tables[slot]);
        S->h_tables[slot] = nullptr;
        S->h_tables_cap[slot] = 0;
        if (cudaMallocHost(&S->h_tables[slot], std::max(tb, (size_t)1 << 20)) != cudaSuccess) {
            cudaGetLastError();
            S->worker_error = "cannot allocate pinned offset buffer";
            for (auto &r : L.reqs) r->status = SW_ENOMEM;
            cudaEventRecord(S->events[slot], s);
            return;
        }
        S->h_tables_cap[slot] = std::max(tb, (size_t)1 << 20);
    }
    unsigned char *ht = S->h_tables[slot];
    int64_t *qo = reinterpret_cast<int64_t *>(ht);
    int64_t *ro = reinterpret_cast<int64_t *>(ht + (Lay.ro - Lay.qo));
    int64_t *qe = pool ? reinterpret_cast<int64_t *>(ht + (Lay.qe - Lay.qo)) : nullptr;
    int64_t *re = pool ? reinterpret_cast<int64_t *>(ht + (Lay.re - Lay.qo)) : nullptr;
    {
        int64_t k = 0, qb = 0, rb = 0;
        for (auto &r : L.reqs) {
            for (int i = 0; i < r->n_pairs; ++i, ++k) {
                if (pool) {
                    const int64_t p = r->first + i;
                    qo[k] = pool->q_off[(size_t)p];
                    qe[k] = pool->q_off[(size_t)p + 1];
                    ro[k] = pool->r_off[(size_t)p];
                    re[k] = pool->r_off[(size_t)p + 1];
                } else {
                    qo[k] = qb + r->q_off[i];
                    ro[k] = rb + r->r_off[i];
                }
            }
            qb += r->q_bytes;
            rb += r->r_bytes;
        }
        qo[n] = pool ? 0 : qb;
        ro[n] = pool ? 0 : rb;
    }
    unsigned char *d = S->d_arena + L.dev_off;
    cudaError_t e = cudaSuccess;
    if (!pool) {
        size_t qb = 0, rb = 0;
        for (auto &r : L.reqs) {
            const unsigned char *h = S->h_pool + r->stage_off;
            if (e == cudaSuccess && r->q_bytes)
                e = cudaMemcpyAsync(d + Lay.q + qb, h + r->st_q, (size_t)r->q_bytes,
                                    cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess && r->r_bytes)
                e = cudaMemcpyAsync(d + Lay.r + rb, h + r->st_r, (size_t)r->r_bytes,
                                    cudaMemcpyHostToDevice, s);
            qb += (size_t)r->q_bytes;
            rb += (size_t)r->r_bytes;
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + Lay.qo, ht, tb, cudaMemcpyHostToDevice, s);
    const uint8_t *qbase = pool ? S->d_arena + pool->dev_off : d + Lay.q;
    const uint8_t *rbase = pool ? S->d_arena + pool->dev_off + pool->r_at : d + Lay.r;
    int32_t *o = reinterpret_cast<int32_t *>(d + Lay.out);
    const Outputs outs{o, o + n, o + 2 * n, o + 3 * n, o + 4 * n};
    if (e == cudaSuccess)
        e = enqueue_device_plan(shape, d + Lay.ws, reinterpret_cast<const int64_t *>(d + Lay.qo),
                                reinterpret_cast<const int64_t *>(d + Lay.ro), qbase, rbase, outs,
                                S->d_status, s,
                                pool ? reinterpret_cast<const int64_t *>(d + Lay.qe) : nullptr,
                                pool ? reinterpret_cast<const int64_t *>(d + Lay.re) : nullptr);
    {
        const double ms = std::chrono::duration<double, std::milli>(
                              std::chrono::steady_clock::now() - t_plan).count();
        std::lock_guard<std::mutex> g(S->mu);
        S->plan_ms += ms;
        S->pairs_launched += n;
    }
    {
        // each request's 5 output rows: one strided copy into its staging area
        int64_t first = 0;
        for (auto &r : L.reqs) {
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(S->h_pool + r->stage_off + r->st_out,
                                      (size_t)r->n_pairs * sizeof(int32_t), o + first,
                                      (size_t)n * sizeof(int32_t),
                                      (size_t)r->n_pairs * sizeof(int32_t), 5,
                                      cudaMemcpyDeviceToHost, s);
            first += r->n_pairs;
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(S->events[slot], s);
    if (e != cudaSuccess) fail_launch(S, L, e, slot);
}

static void worker_loop(sw_server *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        bool progressed = false;
        // ---- completions
        for (size_t k = 0; k < S->slots.size(); ++k) {
            auto &L = S->slots[k];
            if (!L || !L->enqueued) continue;
            const cudaError_t q = cudaEventQuery(S->events[k]);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) {
                S->worker_error = cudaGetErrorString(q);
                for (auto &r : L->reqs) r->status = SW_ECUDA;
            }
            S->arena->release(L->dev_off, L->dev_bytes);
            const int64_t now = std::chrono::duration_cast<std::chrono::nanoseconds>(
                                    std::chrono::steady_clock::now().time_since_epoch())
                                    .count();
            for (auto &r : L->reqs) {
                r->done_ns = now;
                r->done = true;
                ++S->completed;
            }
            L.reset();
            progressed = true;
        }
        if (progressed) {
            S->cv_done.notify_all();
            S->cv_space.notify_all();
        }
        // ---- launches, oldest request first
        while (!S->queue.empty()) {
            int slot = -1;
            bool busy = false;
            for (size_t k = 0; k < S->slots.size(); ++k) {
                if (S->slots[k])
                    busy = true;
                else if (slot < 0)
                    slot = (int)k;
            }
            if (slot < 0) break;
            size_t bytes = 0;
            std::vector<std::shared_ptr<Request>> reqs = take_batch(S, busy, &bytes);
            if (reqs.empty()) break;  // wait for memory to free up
            size_t off = 0;
            if (!S->arena->alloc(bytes, &off)) {  // cannot fail: checked above
                for (auto it = reqs.rbegin(); it != reqs.rend(); ++it) S->queue.push_front(*it);
                break;
            }
            auto L = std::make_unique<Launch>();
            L->reqs = std::move(reqs);
            L->dev_off = off;
            L->dev_bytes = bytes;
            L->slot = slot;
            L->gpu_busy = busy;
            S->plan_queue.push_back(L.get());
            S->slots[slot] = std::move(L);
            ++S->launches;
            S->cv_plan.notify_one();
            progressed = true;
        }
        if (S->stop && S->queue.empty()) {
            bool inflight = false;
            for (auto &L : S->slots) inflight |= (bool)L;
            if (!inflight) break;
        }
        // ---- sleep until new work or a short poll interval for completions
        bool inflight = false;
        for (auto &L : S->slots) inflight |= (bool)L;
        if (!progressed) {
            if (inflight)
                S->cv_work.wait_for(lk, std::chrono::microseconds(20));
            else
                S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
        }
    }
}

static void planner_loop(sw_server *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        S->cv_plan.wait(lk, [&] { return S->stop_planners || !S->plan_queue.empty(); });
        if (S->plan_queue.empty()) break;  // stopping, nothing left
        Launch *L = S->plan_queue.front();
        S->plan_queue.pop_front();
        lk.unlock();
        start_launch(S, *L, L->slot, L->gpu_busy);  // the slot's stream is this launch's alone
        lk.lock();
        L->enqueued = true;
        S->cv_work.notify_one();
    }
}

// Whether a launch of this request alone fits the arena (less the pools).
static bool fits_budget(sw_server *S, const Request &req) {
    DevicePlanShape shape;
    std::string msg;
    if (launch_shape(req, req.n_pairs, req.lmax, S->sms, false, &shape, &msg) != SW_OK) return false;
    const size_t need = layout_of(shape, req.n_pairs, (size_t)req.q_bytes, (size_t)req.r_bytes,
                                  req.pool >= 0)
                            .total;
    size_t pooled = 0;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (auto &p : S->pools) pooled += p->dev_bytes;
    }
    return need + pooled <= S->arena->size();
}

extern "C" {

int sw_server_create(sw_ctx *ctx, int64_t budget_bytes, int32_t streams, int64_t staging_bytes,
                     sw_server **out) {
    if (!out || !ctx || budget_bytes < (1 << 20) || streams < 1 || streams > 64 ||
        staging_bytes < (1 << 20))
        return set_error(SW_EINVAL, "sw_server_create: bad argument");
    *out = nullptr;
    auto *S = new sw_server();
    S->ctx = ctx;
    int dev = 0;
    cudaGetDevice(&dev);
    S->device = dev;
    sw_ctx_sm_count(ctx, &S->sms);
    if (cudaMalloc(&S->d_arena, (size_t)budget_bytes) != cudaSuccess ||
        cudaMalloc(&S->d_status, sizeof(int32_t)) != cudaSuccess ||
        cudaMallocHost(&S->h_pool, (size_t)staging_bytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(S->d_arena);
        cudaFree(S->d_status);
        cudaFreeHost(S->h_pool);
        delete S;
        return set_error(SW_ENOMEM, "sw_server_create: cannot allocate the arena or staging pool");
    }
    cudaMemset(S->d_status, 0, sizeof(int32_t));
    S->arena.reset(new Arena((size_t)budget_bytes));
    S->staging.reset(new Arena((size_t)staging_bytes));
    S->streams.resize(streams);
    S->events.resize(streams);
    S->slots.resize(streams);
    S->h_tables.assign(streams, nullptr);
    S->h_tables_cap.assign(streams, 0);
    for (int k = 0; k < streams; ++k) {
        cudaStreamCreateWithFlags(&S->streams[k], cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&S->events[k], cudaEventDisableTiming);
    }
    S->worker = std::thread(worker_loop, S);
    for (int k = 0; k < kPlanners; ++k) S->planners.emplace_back(planner_loop, S);
    *out = S;
    return SW_OK;
}

int sw_server_submit(sw_server *S, const uint8_t *q_seqs, const int64_t *q_offsets,
                     const uint8_t *r_seqs, const int64_t *r_offsets, int32_t n_pairs,
                     const int8_t *score_matrix, int32_t alphabet_size, int32_t gap_open,
                     int32_t gap_extend, int32_t timeout_ms, int64_t *request_id) {
    if (!S || !request_id || n_pairs < 1)
        return set_error(SW_EINVAL, "sw_server_submit: bad argument");
    auto req = std::make_shared<Request>();
    std::string msg;
    int64_t scratch_words = 0;
    int rc = check_batch(q_offsets, r_offsets, n_pairs, score_matrix, alphabet_size, gap_open,
                         gap_extend, &req->q_bytes, &req->r_bytes, &scratch_words, &msg);
    if (rc != SW_OK) return set_error(rc, ("sw_server_submit: " + msg).c_str());
    if ((req->q_bytes > 0 && !q_seqs) || (req->r_bytes > 0 && !r_seqs))
        return set_error(SW_EINVAL, "sw_server_submit: NULL sequences");
    req->n_pairs = n_pairs;
    req->A = alphabet_size;
    req->go = gap_open;
    req->ge = gap_extend;
    std::memcpy(req->mat, score_matrix, (size_t)alphabet_size * alphabet_size);
    // offsets relative to the request's own first residue
    req->q_off.resize((size_t)n_pairs + 1);
    req->r_off.resize((size_t)n_pairs + 1);
    for (int32_t i = 0; i <= n_pairs; ++i) {
        req->q_off[i] = q_offsets[i] - q_offsets[0];
        req->r_off[i] = r_offsets[i] - r_offsets[0];
    }
    req->q_bytes -= q_offsets[0];
    req->r_bytes -= r_offsets[0];
    for (int32_t i = 0; i < n_pairs; ++i) {
        const int64_t a = req->q_off[i + 1] - req->q_off[i], b = req->r_off[i + 1] - req->r_off[i];
        req->cells += (double)a * (double)b;
        req->lmax = std::max(req->lmax, std::max(a, b));
    }
    (void)scratch_words;
    if (!fits_budget(S, *req))
        return set_error(SW_EBUDGET, "sw_server_submit: request needs more device memory than the "
                                     "server's whole budget");
    req->st_q = 0;
    req->st_r = align_up((size_t)req->q_bytes);
    req->st_out = req->st_r + align_up((size_t)req->r_bytes);
    req->st_total = req->st_out + (size_t)5 * n_pairs * sizeof(int32_t);
    if (req->st_total > S->staging->size())
        return set_error(SW_EBUDGET, "sw_server_submit: request larger than the staging pool");
    std::unique_lock<std::mutex> lk(S->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
    while (!S->staging->alloc(req->st_total, &req->stage_off)) {
        if (S->cv_space.wait_until(lk, deadline) == std::cv_status::timeout) {
            if (!S->staging->alloc(req->st_total, &req->stage_off))
                return set_error(SW_ETIMEOUT,
                                 "sw_server_submit: staging pool full until the timeout");
            break;
        }
    }
    lk.unlock();
    unsigned char *h = S->h_pool + req->stage_off;
    if (req->q_bytes) std::memcpy(h + req->st_q, q_seqs + q_offsets[0], (size_t)req->q_bytes);
    if (req->r_bytes) std::memcpy(h + req->st_r, r_seqs + r_offsets[0], (size_t)req->r_bytes);
    lk.lock();
    req->id = S->next_id++;
    *request_id = req->id;
    S->all[req->id] = req;
    S->queue.push_back(req);
    S->cv_work.notify_one();
    return SW_OK;
}

int sw_server_add_pool(sw_server *S, const uint8_t *q_seqs, const int64_t *q_offsets,
                       const uint8_t *r_seqs, const int64_t *r_offsets, int32_t n_pairs,
                       const int8_t *score_matrix, int32_t alphabet_size, int32_t gap_open,
                       int32_t gap_extend, int32_t *pool_id) {
    if (!S || !pool_id || n_pairs < 1) return set_error(SW_EINVAL, "sw_server_add_pool: bad argument");
    std::string msg;
    int64_t qb = 0, rb = 0, scratch_words = 0;
    int rc = check_batch(q_offsets, r_offsets, n_pairs, score_matrix, alphabet_size, gap_open,
                         gap_extend, &qb, &rb, &scratch_words, &msg);
    if (rc != SW_OK) return set_error(rc, ("sw_server_add_pool: " + msg).c_str());
    if ((qb > q_offsets[0] && !q_seqs) || (rb > r_offsets[0] && !r_seqs))
        return set_error(SW_EINVAL, "sw_server_add_pool: NULL sequences");
    auto P = std::make_unique<Pool>();
    P->A = alphabet_size;
    P->go = gap_open;
    P->ge = gap_extend;
    std::memcpy(P->mat, score_matrix, (size_t)alphabet_size * alphabet_size);
    P->n_pairs = n_pairs;
    P->q_off.resize((size_t)n_pairs + 1);
    P->r_off.resize((size_t)n_pairs + 1);
    for (int32_t i = 0; i <= n_pairs; ++i) {
        P->q_off[i] = q_offsets[i] - q_offsets[0];
        P->r_off[i] = r_offsets[i] - r_offsets[0];
    }
    const size_t qn = (size_t)(qb - q_offsets[0]), rn = (size_t)(rb - r_offsets[0]);
    P->r_at = align_up(qn);
    P->dev_bytes = P->r_at + align_up(rn);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (!S->arena->alloc(P->dev_bytes, &P->dev_off))
            return set_error(SW_EBUDGET, "sw_server_add_pool: the pool does not fit the free budget");
    }
    unsigned char *d = S->d_arena + P->dev_off;
    cudaError_t e = cudaSuccess;
    if (qn) e = cudaMemcpy(d, q_seqs + q_offsets[0], qn, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && rn) e = cudaMemcpy(d + P->r_at, r_seqs + r_offsets[0], rn, cudaMemcpyHostToDevice);
    std::lock_guard<std::mutex> lk(S->mu);
    if (e != cudaSuccess) {
        S->arena->release(P->dev_off, P->dev_bytes);
        return set_error(SW_ECUDA, "sw_server_add_pool: copy to the device failed");
    }
    *pool_id = (int32_t)S->pools.size();
    S->pools.push_back(std::move(P));
    return SW_OK;
}

int sw_server_submit_pool(sw_server *S, int32_t pool_id, int64_t first_pair, int32_t n_pairs,
                          int32_t timeout_ms, int64_t *request_id) {
    if (!S || !request_id || n_pairs < 1) return set_error(SW_EINVAL, "sw_server_submit_pool: bad argument");
    auto req = std::make_shared<Request>();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (pool_id < 0 || pool_id >= (int32_t)S->pools.size())
            return set_error(SW_EINVAL, "sw_server_submit_pool: unknown pool");
        const Pool &P = *S->pools[(size_t)pool_id];
        if (first_pair < 0 || first_pair + n_pairs > P.n_pairs)
            return set_error(SW_ERANGE, "sw_server_submit_pool: pair range outside the pool");
        req->A = P.A;
        req->go = P.go;
        req->ge = P.ge;
        std::memcpy(req->mat, P.mat, sizeof P.mat);
        for (int64_t p = first_pair; p < first_pair + n_pairs; ++p) {
            const int64_t a = P.q_off[(size_t)p + 1] - P.q_off[(size_t)p];
            const int64_t b = P.r_off[(size_t)p + 1] - P.r_off[(size_t)p];
            req->cells += (double)a * (double)b;
            req->lmax = std::max(req->lmax, std::max(a, b));
        }
    }
    req->pool = pool_id;
    req->first = first_pair;
    req->n_pairs = n_pairs;
    req->st_q = req->st_r = req->st_out = 0;  // only the outputs are staged
    req->st_total = (size_t)5 * n_pairs * sizeof(int32_t);
    if (!fits_budget(S, *req))
        return set_error(SW_EBUDGET, "sw_server_submit_pool: request needs more device memory "
                                     "than the server's budget leaves");
    if (req->st_total > S->staging->size())
        return set_error(SW_EBUDGET, "sw_server_submit_pool: request larger than the staging pool");
    std::unique_lock<std::mutex> lk(S->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
    while (!S->staging->alloc(req->st_total, &req->stage_off)) {
        if (S->cv_space.wait_until(lk, deadline) == std::cv_status::timeout) {
            if (!S->staging->alloc(req->st_total, &req->stage_off))
                return set_error(SW_ETIMEOUT,
                                 "sw_server_submit_pool: staging pool full until the timeout");
            break;
        }
    }
    req->id = S->next_id++;
    *request_id = req->id;
    S->all[req->id] = req;
    S->queue.push_back(req);
    S->cv_work.notify_one();
    return SW_OK;
}

int sw_server_poll(sw_server *S, int64_t request_id, int32_t *done) {
    if (!S || !done) return set_error(SW_EINVAL, "sw_server_poll: bad argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(request_id);
    if (it == S->all.end()) return set_error(SW_EINVAL, "sw_server_poll: unknown request");
    *done = it->second->done ? 1 : 0;
    return SW_OK;
}

int sw_server_wait(sw_server *S, int64_t request_id, int32_t timeout_ms, int32_t *out_host,
                   int64_t *done_ns) {
    if (!S || !out_host) return set_error(SW_EINVAL, "sw_server_wait: bad argument");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(request_id);
    if (it == S->all.end()) return set_error(SW_EINVAL, "sw_server_wait: unknown request");
    auto req = it->second;
    const bool ok = S->cv_done.wait_for(lk, std::chrono::milliseconds(std::max(0, timeout_ms)),
                                         [&] { return req->done; });
    if (!ok) return set_error(SW_ETIMEOUT, "sw_server_wait: request not done before the timeout");
    const int status = req->status;
    if (status == SW_OK) {
        std::memcpy(out_host, S->h_pool + req->stage_off + req->st_out,
                    (size_t)5 * req->n_pairs * sizeof(int32_t));
        if (done_ns) *done_ns = req->done_ns;
    }
    S->staging->release(req->stage_off, req->st_total);
    S->all.erase(it);
    S->cv_space.notify_all();
    if (status != SW_OK)
        return set_error(status, ("sw_server_wait: " + S->worker_error).c_str());
    return SW_OK;
}

int sw_server_stats(sw_server *S, int64_t *completed, int64_t *in_flight, int64_t *queued,
                    int64_t *device_bytes_in_use, int64_t *device_bytes_peak) {
    if (!S) return set_error(SW_EINVAL, "sw_server_stats: bad argument");
    std::lock_guard<std::mutex> lk(S->mu);
    int64_t inflight = 0;
    for (auto &L : S->slots)
        if (L) inflight += (int64_t)L->reqs.size();
    if (completed) *completed = S->completed;
    if (in_flight) *in_flight = inflight;
    if (queued) *queued = (int64_t)S->queue.size();
    if (device_bytes_in_use) *device_bytes_in_use = (int64_t)S->arena->used();
    if (device_bytes_peak) *device_bytes_peak = (int64_t)S->arena->peak();
    return SW_OK;
}

int sw_server_launches(sw_server *S, int64_t *launches, int64_t *pairs_launched,
                       double *plan_ms) {
    if (!S) return set_error(SW_EINVAL, "sw_server_launches: bad argument");
    std::lock_guard<std::mutex> lk(S->mu);
    if (launches) *launches = S->launches;
    if (pairs_launched) *pairs_launched = S->pairs_launched;
    if (plan_ms) *plan_ms = S->plan_ms;
    return SW_OK;
}

int sw_server_destroy(sw_server *S) {
    if (!S) return SW_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();  // returns once every launch retired
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop_planners = true;
        S->cv_plan.notify_all();
    }
    for (auto &th : S->planners)
        if (th.joinable()) th.join();
    cudaSetDevice(S->device);
    for (size_t k = 0; k < S->streams.size(); ++k) {
        cudaStreamSynchronize(S->streams[k]);
        cudaStreamDestroy(S->streams[k]);
        cudaEventDestroy(S->events[k]);
        cudaFreeHost(S->h_tables[k]);
    }
    cudaFree(S->d_arena);
    cudaFree(S->d_status);
    cudaFreeHost(S->h_pool);
    delete S;
    return SW_OK;
}

}  // extern "C"
