// Serving loop: continuous batching of alignment requests.
//
// A request is a batch of pairs on the host.  sw_server_submit checks it,
// copies its sequences into a pinned staging pool and queues it.  A worker
// thread turns the queue into launches: whenever a stream slot is free it
// takes the oldest queued request together with the later queued requests
// that share its scoring (matrix and gap costs), up to a cap on pairs and
// cells and to what the device arena has left, plans them as one batch
// (pairs are independent, so a pair's results do not depend on its batch
// mates) and runs that batch on the slot's stream: sequences copied into
// one arena block, the persistent kernel, each request's outputs copied
// back into its staging area.  The arena is one device allocation of the
// server's memory budget, made at creation.  Under light load a launch
// holds one request and is planned for latency (up to one warp per pair);
// while other launches are in flight it is planned to fill lane groups
// instead, and under heavy load the queue grows between launches, so each
// launch takes many requests and runs at the batched kernel's throughput.
// Forming a launch is the worker's; planning and enqueueing it (milliseconds
// of host work for tens of thousands of pairs) is done by one of eight
// planner threads, so launches are planned in parallel.  When a launch's
// completion event fires the worker frees its arena block and slot and
// wakes the waiters.
//
// Every wait is bounded: sw_server_wait and sw_server_submit take a timeout
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
// The worker plans every launch itself, so its schedule simulation looks at
// fewer pairs than a one-off plan's.
constexpr int kLaunchPlanSample = 1024;

struct Request {
    int64_t id = 0;
    int n_pairs = 0;
    int A = 0, go = 0, ge = 0;
    int8_t mat[kMaxAlphabet * kMaxAlphabet] = {0};
    std::vector<int64_t> q_off, r_off;  // the request's own CSR offsets
    int64_t q_bytes = 0, r_bytes = 0;
    double cells = 0;
    size_t dev_bound = 0;  // device bytes the request can add to a launch
    // staging pool layout: q | r | out (5 x n_pairs int32)
    size_t stage_off = 0, st_q = 0, st_r = 0, st_out = 0, st_total = 0;
    bool done = false;
    int status = SW_OK;
    int64_t done_ns = 0;  // CLOCK_MONOTONIC when the worker saw it finish
};

bool same_scoring(const Request &a, const Request &b) {
    return a.A == b.A && a.go == b.go && a.ge == b.ge &&
           std::memcmp(a.mat, b.mat, (size_t)a.A * a.A) == 0;
}

// Byte layout of one launch's arena block.
struct Layout {
    size_t q = 0, r = 0, pairs = 0, classes = 0, plain = 0, counters = 0, scratch = 0, out = 0,
           tables_end = 0, total = 0;
};

Layout layout_of(const HostPlan &hp, int64_t n_pairs) {
    Layout L;
    size_t at = 0;
    auto take = [&](size_t bytes) {
        const size_t o = at;
        at = align_up(at + bytes);
        return o;
    };
    L.q = take((size_t)hp.q_bytes);
    L.r = take((size_t)hp.r_bytes);
    L.pairs = take(hp.pairs.size() * sizeof(PairInfo));
    L.classes = take(hp.classes.size() * sizeof(ClassInfo));
    L.plain = take(hp.plain.size() * sizeof(PairInfo));
    L.tables_end = at;
    L.counters = take(kMaxClasses * sizeof(int32_t));
    L.scratch = take((size_t)hp.scratch_words * sizeof(uint32_t));
    L.out = take((size_t)5 * n_pairs * sizeof(int32_t));
    L.total = at;
    return L;
}

// Upper bound on what a request adds to a launch's block: its sequences,
// pair records, worst-case strip scratch, outputs and alignment slack.  The
// classes table and counters (fixed, small) are covered by kLaunchFixed.
size_t request_bound(int64_t q_bytes, int64_t r_bytes, int64_t n_pairs, int64_t scratch_words) {
    return (size_t)q_bytes + (size_t)r_bytes + (size_t)n_pairs * sizeof(PairInfo) +
           (size_t)scratch_words * sizeof(uint32_t) + (size_t)n_pairs * 5 * sizeof(int32_t) +
           8 * kAlign;
}
constexpr size_t kLaunchFixed = 8 * kAlign + kMaxClasses * (sizeof(ClassInfo) + sizeof(int32_t));

struct Launch {
    std::vector<std::shared_ptr<Request>> reqs;
    size_t dev_off = 0, dev_bytes = 0;
    int slot = -1;
    bool gpu_busy = false;  // other launches were on the GPU when it was formed
    bool enqueued = false;  // its work and completion event are on the stream
};

// Planner threads: a launch's host planning takes milliseconds for tens of
// thousands of pairs, so several launches are planned and enqueued at once
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
    std::unique_ptr<Arena> arena, pool;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    std::vector<std::unique_ptr<Launch>> slots;  // in flight, by slot
    std::vector<unsigned char *> h_tables;       // pinned per-slot table buffers
    std::vector<size_t> h_tables_cap;
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
// and later ones with the same scoring, within the caps and the arena's
// largest free block).  Caller holds the mutex.
static std::vector<std::shared_ptr<Request>> take_batch(sw_server *S) {
    std::vector<std::shared_ptr<Request>> out;
    const size_t room = S->arena->largest_free();
    size_t bytes = kLaunchFixed;
    int64_t pairs = 0;
    double cells = 0;
    for (auto it = S->queue.begin(); it != S->queue.end();) {
        const auto &r = *it;
        if (!out.empty() && !same_scoring(*out.front(), *r)) {
            ++it;
            continue;
        }
        if (bytes + r->dev_bound > room) break;
        if (!out.empty() && (pairs + r->n_pairs > kLaunchMaxPairs ||
                             cells + r->cells > kLaunchMaxCells))
            break;
        bytes += r->dev_bound;
        pairs += r->n_pairs;
        cells += r->cells;
        out.push_back(r);
        it = S->queue.erase(it);
    }
    return out;
}

static void fail_launch(sw_server *S, Launch &L, cudaError_t e, int slot) {
    S->worker_error = cudaGetErrorString(e);
    for (auto &r : L.reqs) r->status = SW_ECUDA;
    cudaStreamSynchronize(S->streams[slot]);
    cudaGetLastError();
    cudaEventRecord(S->events[slot], S->streams[slot]);
}

// Plans and enqueues one launch on the slot's stream.  Called with the
// mutex released: only the worker touches the slot and the launch.
static void start_launch(sw_server *S, Launch &L, int slot, bool gpu_busy) {
    cudaStream_t s = S->streams[slot];
    const Request &head = *L.reqs.front();
    // merged CSR offsets: the requests' sequences one after another
    int64_t n = 0;
    for (auto &r : L.reqs) n += r->n_pairs;
    std::vector<int64_t> qo((size_t)n + 1), ro((size_t)n + 1);
    {
        int64_t k = 0, qb = 0, rb = 0;
        for (auto &r : L.reqs) {
            for (int i = 0; i < r->n_pairs; ++i, ++k) {
                qo[k] = qb + r->q_off[i];
                ro[k] = rb + r->r_off[i];
            }
            qb += r->q_bytes;
            rb += r->r_bytes;
        }
        qo[n] = qb;
        ro[n] = rb;
    }
    HostPlan hp;
    std::string msg;
    const auto t_plan = std::chrono::steady_clock::now();
    int rc = make_host_plan(qo.data(), ro.data(), (int32_t)n, head.mat, head.A, head.go, head.ge,
                            SW_MODE_AUTO, S->sms, -1, 0.5, &hp, &msg,
                            gpu_busy ? (32 >> kMinLog2G) : 1, kLaunchPlanSample);
    const Layout Lay = layout_of(hp, n);
    {
        const double ms = std::chrono::duration<double, std::milli>(
                              std::chrono::steady_clock::now() - t_plan).count();
        std::lock_guard<std::mutex> g(S->mu);
        S->plan_ms += ms;
        S->pairs_launched += n;
    }
    if (rc != SW_OK || Lay.total > L.dev_bytes) {
        // cannot happen for checked requests within their bound; fail loudly
        S->worker_error = rc != SW_OK ? msg : "launch exceeds its arena block";
        for (auto &r : L.reqs) r->status = rc != SW_OK ? rc : SW_ENOMEM;
        cudaEventRecord(S->events[slot], s);
        return;
    }
    unsigned char *d = S->d_arena + L.dev_off;
    // tables through a pinned per-slot buffer (the slot is idle, so the
    // buffer's previous contents are no longer being copied)
    const size_t tb = Lay.tables_end - Lay.pairs;
    if (S->h_tables_cap[slot] < tb) {
        cudaFreeHost(S->h_tables[slot]);
        S->h_tables[slot] = nullptr;
        S->h_tables_cap[slot] = 0;
        if (cudaMallocHost(&S->h_tables[slot], std::max(tb, (size_t)1 << 20)) != cudaSuccess) {
            cudaGetLastError();
            S->worker_error = "cannot allocate pinned table buffer";
            for (auto &r : L.reqs) r->status = SW_ENOMEM;
            cudaEventRecord(S->events[slot], s);
            return;
        }
        S->h_tables_cap[slot] = std::max(tb, (size_t)1 << 20);
    }
    unsigned char *ht = S->h_tables[slot];
    if (!hp.pairs.empty())
        std::memcpy(ht + (Lay.pairs - Lay.pairs), hp.pairs.data(), hp.pairs.size() * sizeof(PairInfo));
    if (!hp.classes.empty())
        std::memcpy(ht + (Lay.classes - Lay.pairs), hp.classes.data(),
                    hp.classes.size() * sizeof(ClassInfo));
    if (!hp.plain.empty())
        std::memcpy(ht + (Lay.plain - Lay.pairs), hp.plain.data(), hp.plain.size() * sizeof(PairInfo));
    cudaError_t e = cudaSuccess;
    {
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
    if (e == cudaSuccess && tb)
        e = cudaMemcpyAsync(d + Lay.pairs, ht, tb, cudaMemcpyHostToDevice, s);
    DeviceTables t;
    t.pairs = reinterpret_cast<const PairInfo *>(d + Lay.pairs);
    t.classes = reinterpret_cast<const ClassInfo *>(d + Lay.classes);
    t.plain = reinterpret_cast<const PairInfo *>(d + Lay.plain);
    t.counters = reinterpret_cast<int32_t *>(d + Lay.counters);
    t.scratch = reinterpret_cast<uint32_t *>(d + Lay.scratch);
    t.status = S->d_status;
    int32_t *o = reinterpret_cast<int32_t *>(d + Lay.out);
    const Outputs outs{o, o + n, o + 2 * n, o + 3 * n, o + 4 * n};
    if (e == cudaSuccess)
        e = enqueue_plan(hp, t, d + Lay.q, d + Lay.r, outs, head.mat, head.A, head.go, head.ge, s);
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
            std::vector<std::shared_ptr<Request>> reqs = take_batch(S);
            if (reqs.empty()) break;  // wait for memory to free up
            size_t bytes = kLaunchFixed;
            for (auto &r : reqs) bytes += r->dev_bound;
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
    S->pool.reset(new Arena((size_t)staging_bytes));
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
    for (int32_t i = 0; i < n_pairs; ++i)
        req->cells += (double)(req->q_off[i + 1] - req->q_off[i]) *
                      (double)(req->r_off[i + 1] - req->r_off[i]);
    req->dev_bound = request_bound(req->q_bytes, req->r_bytes, n_pairs, scratch_words);
    if (req->dev_bound + kLaunchFixed > S->arena->size())
        return set_error(SW_EBUDGET, "sw_server_submit: request needs more device memory than the "
                                     "server's whole budget");
    req->st_q = 0;
    req->st_r = align_up((size_t)req->q_bytes);
    req->st_out = req->st_r + align_up((size_t)req->r_bytes);
    req->st_total = req->st_out + (size_t)5 * n_pairs * sizeof(int32_t);
    if (req->st_total > S->pool->size())
        return set_error(SW_EBUDGET, "sw_server_submit: request larger than the staging pool");
    std::unique_lock<std::mutex> lk(S->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
    while (!S->pool->alloc(req->st_total, &req->stage_off)) {
        if (S->cv_space.wait_until(lk, deadline) == std::cv_status::timeout) {
            if (!S->pool->alloc(req->st_total, &req->stage_off))
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
    S->pool->release(req->stage_off, req->st_total);
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
