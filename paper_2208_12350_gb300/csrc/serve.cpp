// Serving loop: continuous batching of alignment requests.
//
// A request is a batch of pairs on the host.  sw_server_submit plans it at
// once (host planning, as sw_plan_create), copies its sequences and device
// tables into a pinned staging pool and queues it.  A worker thread admits
// queued requests in arrival order as soon as a stream slot is free and the
// request's device bytes (sequences, tables, strip scratch, outputs) fit in
// the server's device arena, whose size is the memory budget given at
// creation: one allocation, made once, holds every admitted request's data
// while it is on the GPU.  An admitted request's copies and kernels run on
// its slot's stream, so requests that arrive while others are running
// overlap with them on the device.  When its completion event fires, the
// worker releases its arena block and slot and wakes the waiters.  Results
// are identical to running the request alone: the same kernels see the same
// inputs.
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

  private:
    size_t size_, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
};

// Byte layout of one request, identical in the staging pool and the arena.
struct Layout {
    size_t q = 0, r = 0, pairs = 0, classes = 0, plain = 0, counters = 0, scratch = 0, out = 0,
           total = 0;
};

Layout layout_of(const HostPlan &hp, int n_pairs) {
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
    L.counters = take(kMaxClasses * sizeof(int32_t));
    L.scratch = take((size_t)hp.scratch_words * sizeof(uint32_t));
    L.out = take((size_t)5 * n_pairs * sizeof(int32_t));
    L.total = at;
    return L;
}

struct Request {
    int64_t id = 0;
    int n_pairs = 0;
    int A = 0, go = 0, ge = 0;
    int8_t mat[kMaxAlphabet * kMaxAlphabet] = {0};
    HostPlan hp;
    Layout L;
    size_t stage_off = 0;  // in the pinned pool
    size_t dev_off = 0;    // in the device arena
    int slot = -1;
    bool done = false;
    int status = SW_OK;
};

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
    std::vector<std::shared_ptr<Request>> slots;  // in flight, by slot
    std::deque<std::shared_ptr<Request>> queue;   // admitted in this order
    std::unordered_map<int64_t, std::shared_ptr<Request>> all;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_space;
    std::thread worker;
    bool stop = false;
    int64_t next_id = 1, completed = 0;
    std::string worker_error;
};

static void worker_loop(sw_server *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        bool progressed = false;
        // ---- completions
        for (size_t k = 0; k < S->slots.size(); ++k) {
            auto &req = S->slots[k];
            if (!req) continue;
            const cudaError_t q = cudaEventQuery(S->events[k]);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) {
                req->status = SW_ECUDA;
                S->worker_error = cudaGetErrorString(q);
            }
            S->arena->release(req->dev_off, req->L.total);
            req->done = true;
            req->slot = -1;
            ++S->completed;
            req.reset();
            progressed = true;
        }
        if (progressed) {
            S->cv_done.notify_all();
            S->cv_space.notify_all();
        }
        // ---- admissions, in arrival order
        while (!S->queue.empty()) {
            int slot = -1;
            for (size_t k = 0; k < S->slots.size(); ++k)
                if (!S->slots[k]) {
                    slot = (int)k;
                    break;
                }
            if (slot < 0) break;
            auto req = S->queue.front();
            size_t off = 0;
            if (!S->arena->alloc(req->L.total, &off)) break;  // wait for memory to free up
            S->queue.pop_front();
            req->dev_off = off;
            req->slot = slot;
            S->slots[slot] = req;
            cudaStream_t s = S->streams[slot];
            unsigned char *d = S->d_arena + off;
            const unsigned char *h = S->h_pool + req->stage_off;
            const Layout &L = req->L;
            // sequences and tables in one copy (they are contiguous)
            cudaError_t e = cudaMemcpyAsync(d, h, L.counters, cudaMemcpyHostToDevice, s);
            DeviceTables t;
            t.pairs = reinterpret_cast<const PairInfo *>(d + L.pairs);
            t.classes = reinterpret_cast<const ClassInfo *>(d + L.classes);
            t.plain = reinterpret_cast<const PairInfo *>(d + L.plain);
            t.counters = reinterpret_cast<int32_t *>(d + L.counters);
            t.scratch = reinterpret_cast<uint32_t *>(d + L.scratch);
            t.status = S->d_status;
            int32_t *o = reinterpret_cast<int32_t *>(d + L.out);
            const int64_t n = req->n_pairs;
            const Outputs outs{o, o + n, o + 2 * n, o + 3 * n, o + 4 * n};
            if (e == cudaSuccess)
                e = enqueue_plan(req->hp, t, d + L.q, d + L.r, outs, req->mat, req->A, req->go,
                                 req->ge, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(S->h_pool + req->stage_off + L.out, o, 5 * n * sizeof(int32_t),
                                    cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaEventRecord(S->events[slot], s);
            if (e != cudaSuccess) {
                req->status = SW_ECUDA;
                S->worker_error = cudaGetErrorString(e);
                cudaStreamSynchronize(s);
                cudaGetLastError();
                cudaEventRecord(S->events[slot], s);
            }
            progressed = true;
        }
        if (S->stop && S->queue.empty()) {
            bool busy = false;
            for (auto &r : S->slots) busy |= (bool)r;
            if (!busy) break;
        }
        // ---- sleep until new work or a short poll interval for completions
        bool inflight = false;
        for (auto &r : S->slots) inflight |= (bool)r;
        if (!progressed) {
            if (inflight)
                S->cv_work.wait_for(lk, std::chrono::microseconds(20));
            else
                S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
        }
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
    for (int k = 0; k < streams; ++k) {
        cudaStreamCreateWithFlags(&S->streams[k], cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&S->events[k], cudaEventDisableTiming);
    }
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return SW_OK;
}

int sw_server_submit(sw_server *S, const uint8_t *q_seqs, const int64_t *q_offsets,
                     const uint8_t *r_seqs, const int64_t *r_offsets, int32_t n_pairs,
                     const int8_t *score_matrix, int32_t alphabet_size, int32_t gap_open,
                     int32_t gap_extend, int32_t timeout_ms, int64_t *request_id) {
    if (!S || !request_id || n_pairs < 1) return set_error(SW_EINVAL, "sw_server_submit: bad argument");
    auto req = std::make_shared<Request>();
    std::string msg;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != S->device) cudaSetDevice(S->device);
    int rc = make_host_plan(q_offsets, r_offsets, n_pairs, score_matrix, alphabet_size, gap_open,
                            gap_extend, SW_MODE_AUTO, S->sms, -1, 0.5, &req->hp, &msg);
    if (prev >= 0 && prev != S->device) cudaSetDevice(prev);
    if (rc != SW_OK) return set_error(rc, ("sw_server_submit: " + msg).c_str());
    if ((req->hp.q_bytes > 0 && !q_seqs) || (req->hp.r_bytes > 0 && !r_seqs))
        return set_error(SW_EINVAL, "sw_server_submit: NULL sequences");
    req->n_pairs = n_pairs;
    req->A = alphabet_size;
    req->go = gap_open;
    req->ge = gap_extend;
    std::memcpy(req->mat, score_matrix, (size_t)alphabet_size * alphabet_size);
    req->L = layout_of(req->hp, n_pairs);
    if (req->L.total > S->arena->size())
        return set_error(SW_EBUDGET, "sw_server_submit: request needs more device memory than the "
                                     "server's whole budget");
    if (req->L.total > S->pool->size())
        return set_error(SW_EBUDGET, "sw_server_submit: request larger than the staging pool");
    std::unique_lock<std::mutex> lk(S->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
    while (!S->pool->alloc(req->L.total, &req->stage_off)) {
        if (S->cv_space.wait_until(lk, deadline) == std::cv_status::timeout) {
            if (!S->pool->alloc(req->L.total, &req->stage_off))
                return set_error(SW_ETIMEOUT,
                                 "sw_server_submit: staging pool full until the timeout");
            break;
        }
    }
    lk.unlock();
    unsigned char *h = S->h_pool + req->stage_off;
    const Layout &L = req->L;
    if (req->hp.q_bytes) std::memcpy(h + L.q, q_seqs, (size_t)req->hp.q_bytes);
    if (req->hp.r_bytes) std::memcpy(h + L.r, r_seqs, (size_t)req->hp.r_bytes);
    if (!req->hp.pairs.empty())
        std::memcpy(h + L.pairs, req->hp.pairs.data(), req->hp.pairs.size() * sizeof(PairInfo));
    if (!req->hp.classes.empty())
        std::memcpy(h + L.classes, req->hp.classes.data(),
                    req->hp.classes.size() * sizeof(ClassInfo));
    if (!req->hp.plain.empty())
        std::memcpy(h + L.plain, req->hp.plain.data(), req->hp.plain.size() * sizeof(PairInfo));
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

int sw_server_wait(sw_server *S, int64_t request_id, int32_t timeout_ms, int32_t *out_host) {
    if (!S || !out_host) return set_error(SW_EINVAL, "sw_server_wait: bad argument");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(request_id);
    if (it == S->all.end()) return set_error(SW_EINVAL, "sw_server_wait: unknown request");
    auto req = it->second;
    const bool ok = S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                         [&] { return req->done; });
    if (!ok) return set_error(SW_ETIMEOUT, "sw_server_wait: request not done before the timeout");
    if (req->status != SW_OK)
        return set_error(req->status, ("sw_server_wait: " + S->worker_error).c_str());
    std::memcpy(out_host, S->h_pool + req->stage_off + req->L.out,
                (size_t)5 * req->n_pairs * sizeof(int32_t));
    S->pool->release(req->stage_off, req->L.total);
    S->all.erase(it);
    S->cv_space.notify_all();
    return SW_OK;
}

int sw_server_stats(sw_server *S, int64_t *completed, int64_t *in_flight, int64_t *queued,
                    int64_t *device_bytes_in_use, int64_t *device_bytes_peak) {
    if (!S) return set_error(SW_EINVAL, "sw_server_stats: bad argument");
    std::lock_guard<std::mutex> lk(S->mu);
    int64_t inflight = 0;
    for (auto &r : S->slots) inflight += r ? 1 : 0;
    if (completed) *completed = S->completed;
    if (in_flight) *in_flight = inflight;
    if (queued) *queued = (int64_t)S->queue.size();
    if (device_bytes_in_use) *device_bytes_in_use = (int64_t)S->arena->used();
    if (device_bytes_peak) *device_bytes_peak = (int64_t)S->arena->peak();
    return SW_OK;
}

int sw_server_destroy(sw_server *S) {
    if (!S) return SW_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    cudaSetDevice(S->device);
    for (size_t k = 0; k < S->streams.size(); ++k) {
        cudaStreamSynchronize(S->streams[k]);
        cudaStreamDestroy(S->streams[k]);
        cudaEventDestroy(S->events[k]);
    }
    cudaFree(S->d_arena);
    cudaFree(S->d_status);
    cudaFreeHost(S->h_pool);
    delete S;
    return SW_OK;
}

}  // extern "C"
