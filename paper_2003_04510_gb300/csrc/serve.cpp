// serve.cpp -- HE Mul serving with continuous batching.
//
// Requests (HE Mul + rescale of device-resident operands, any of the
// server's rings and levels) are queued by he_server_submit.  A scheduler
// thread admits them in arrival order as workspace in a fixed device arena
// (the HBM budget) and stream slots free up, groups the admitted requests of
// one ring into a batch (he_mul_batch: every stage is one launch over the
// whole batch) and launches it on a free stream, so batches formed while
// earlier ones are still running overlap on the GPU.  Completion is detected
// by polling each batch's CUDA event on the host; there are no device-side
// waits.  Results are bit-identical to he_mul_rescale on each request alone.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "he_internal.h"

namespace {

using clk = std::chrono::steady_clock;

// First-fit allocator over [0, size) in 256-byte units.
class Arena {
public:
    explicit Arena(size_t size) : size_(size) { free_[0] = size; }
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = (bytes + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                size_t rest = it->second - bytes, start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = (bytes + 255) & ~(size_t)255;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t size() const { return size_; }

private:
    size_t size_;
    std::map<size_t, size_t> free_;  // offset -> length
};

struct Req {
    uint64_t ticket;
    he_request r;
    clk::time_point t_submit;
};

// Finished tickets whose status is kept for he_server_poll / he_server_wait,
// and completion latencies kept for he_server_stats: the most recent ones
// (older entries are dropped, so a long-running server's memory stays bounded).
constexpr uint64_t kKeepTickets = 1u << 20;
constexpr size_t kKeepLatencies = 1u << 16;

struct Flight {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<uint64_t> tickets;
    std::vector<clk::time_point> t_submit;
    size_t ws_off = 0, ws_bytes = 0;
    int rc = HE_OK;
};

}  // namespace

struct he_server {
    std::vector<he_ctx *> ctxs;
    std::vector<const u64 *> evks;
    int max_batch = 64;
    void *arena_mem = nullptr;
    Arena *arena = nullptr;
    std::vector<Flight> flights;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req> pending;
    std::map<uint64_t, int> status;  // ticket -> 0 pending/in flight, 1 done, <0 -error
    std::vector<double> latencies_ms;  // ring of the last kKeepLatencies completions
    size_t lat_next = 0;
    uint64_t next_ticket = 1;
    uint64_t completed = 0, batches = 0, batched_requests = 0;
    clk::time_point t_first, t_last;
    bool have_first = false;
    std::atomic<bool> stop{false};
    std::thread worker;
    int device = 0;
};

namespace {

size_t request_bytes(he_server *s, const he_request &r)
{
    int lv = r.level;
    return he_batch_workspace_bytes(s->ctxs[r.ctx_index], 1, &lv);
}

// One scheduler step: retire finished batches, then launch new ones while a
// stream is free and the queue head fits.  Returns true if anything happened.
bool step(he_server *s)
{
    bool progress = false;
    // retire
    for (Flight &f : s->flights) {
        if (!f.busy) continue;
        cudaError_t q = cudaEventQuery(f.done);
        if (q == cudaErrorNotReady) continue;
        const auto now = clk::now();
        std::lock_guard<std::mutex> lk(s->mu);
        const int st = (q == cudaSuccess && f.rc == HE_OK) ? 1 : -(f.rc == HE_OK ? HE_ECUDA : f.rc);
        for (size_t i = 0; i < f.tickets.size(); i++) {
            s->status[f.tickets[i]] = st;
            const double ms = std::chrono::duration<double, std::milli>(now - f.t_submit[i]).count();
            if (s->latencies_ms.size() < kKeepLatencies) s->latencies_ms.push_back(ms);
            else s->latencies_ms[s->lat_next] = ms;
            s->lat_next = (s->lat_next + 1) % kKeepLatencies;
        }
        // forget finished tickets that are more than kKeepTickets old
        while (!s->status.empty() && s->status.begin()->first + kKeepTickets < s->next_ticket &&
               s->status.begin()->second != 0)
            s->status.erase(s->status.begin());
        s->completed += f.tickets.size();
        s->t_last = now;
        s->arena->release(f.ws_off, f.ws_bytes);
        f.busy = false;
        f.tickets.clear();
        f.t_submit.clear();
        progress = true;
        s->cv.notify_all();
    }
    // launch
    for (Flight &f : s->flights) {
        if (f.busy) continue;
        std::vector<Req> take;
        size_t off = 0, bytes = 0;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->pending.empty()) break;
            const int ci = s->pending.front().r.ctx_index;
            std::vector<int> levels;
            // arrival order within the head's ring, up to max_batch, while the batch's workspace fits
            for (auto it = s->pending.begin(); it != s->pending.end() && (int)take.size() < s->max_batch;) {
                if (it->r.ctx_index != ci) {
                    ++it;
                    continue;
                }
                levels.push_back(it->r.level);
                size_t need = he_batch_workspace_bytes(s->ctxs[ci], (int)levels.size(), levels.data());
                if (!s->arena->alloc(need, &off)) {
                    levels.pop_back();
                    break;
                }
                s->arena->release(off, need);  // probe only; the final block is taken below
                bytes = need;
                take.push_back(*it);
                it = s->pending.erase(it);
            }
            if (take.empty()) break;  // the head does not fit yet: wait for a batch to retire
            if (!s->arena->alloc(bytes, &off)) {  // cannot fail: probed under the same lock
                for (auto it = take.rbegin(); it != take.rend(); ++it) s->pending.push_front(*it);
                break;
            }
        }
        he_ctx *c = s->ctxs[take[0].r.ctx_index];
        // operands written on other streams: the batch waits for their events
        int rc_wait = HE_OK;
        for (const Req &q : take)
            if (q.r.ready && cudaStreamWaitEvent(f.stream, (cudaEvent_t)q.r.ready, 0) != cudaSuccess)
                rc_wait = HE_ECUDA;
        std::vector<he_job> jobs(take.size());
        for (size_t i = 0; i < take.size(); i++) {
            jobs[i].ct1 = take[i].r.ct1;
            jobs[i].ct2 = take[i].r.ct2;
            jobs[i].out = take[i].r.out;
            jobs[i].level = take[i].r.level;
        }
        f.rc = rc_wait != HE_OK ? rc_wait
                                : he_mul_batch(c, (int)jobs.size(), jobs.data(), s->evks[take[0].r.ctx_index],
                                               (char *)s->arena_mem + off, bytes, f.stream);
        cudaEventRecord(f.done, f.stream);
        f.busy = true;
        f.ws_off = off;
        f.ws_bytes = bytes;
        for (const Req &q : take) {
            f.tickets.push_back(q.ticket);
            f.t_submit.push_back(q.t_submit);
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->batches++;
            s->batched_requests += take.size();
        }
        progress = true;
    }
    return progress;
}

void worker_main(he_server *s)
{
    cudaSetDevice(s->device);
    while (!s->stop.load()) {
        if (!step(s)) {
            bool idle;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                idle = s->pending.empty();
            }
            bool inflight = false;
            for (const Flight &f : s->flights) inflight |= f.busy;
            if (idle && !inflight) {
                std::unique_lock<std::mutex> lk(s->mu);
                s->cv.wait_for(lk, std::chrono::milliseconds(1));
            } else {
                std::this_thread::yield();
            }
        }
    }
}

}  // namespace

extern "C" {

int he_server_create(he_server **out, he_ctx *const *ctxs, const uint64_t *const *evks, int nctx, size_t hbm_budget,
                     int max_batch, int streams)
{
    if (!out || !ctxs || !evks || nctx < 1 || nctx > 16 || max_batch < 1 || max_batch > 1024 || streams < 1 ||
        streams > 16 || hbm_budget < 256)
        return HE_EINVAL;
    for (int i = 0; i < nctx; i++)
        if (!ctxs[i] || !ctxs[i]->device || !evks[i]) return HE_EINVAL;
    he_server *s = new (std::nothrow) he_server();
    if (!s) return HE_ENOMEM;
    s->ctxs.assign(ctxs, ctxs + nctx);
    s->evks.assign(evks, evks + nctx);
    s->max_batch = max_batch;
    cudaGetDevice(&s->device);
    if (cudaMalloc(&s->arena_mem, hbm_budget) != cudaSuccess) {
        delete s;
        return HE_ENOMEM;
    }
    s->arena = new Arena(hbm_budget);
    s->flights.resize(streams);
    for (Flight &f : s->flights) {
        if (cudaStreamCreateWithFlags(&f.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&f.done, cudaEventDisableTiming) != cudaSuccess) {
            he_server_destroy(s);
            return HE_ECUDA;
        }
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return HE_OK;
}

int he_server_submit(he_server *s, const he_request *r, uint64_t *ticket)
{
    if (!s || !r || !ticket) return HE_EINVAL;
    if (r->ctx_index < 0 || r->ctx_index >= (int)s->ctxs.size()) return HE_EINVAL;
    if (!r->ct1 || !r->ct2 || !r->out) return HE_EINVAL;
    if (r->level < 2 || r->level > s->ctxs[r->ctx_index]->L) return HE_ELEVEL;
    if (request_bytes(s, *r) > s->arena->size()) return HE_ENOMEM;  // can never be admitted
    std::lock_guard<std::mutex> lk(s->mu);
    Req q;
    q.ticket = s->next_ticket++;
    q.r = *r;
    q.t_submit = clk::now();
    if (!s->have_first) {
        s->t_first = q.t_submit;
        s->have_first = true;
    }
    s->pending.push_back(q);
    s->status[q.ticket] = 0;
    *ticket = q.ticket;
    s->cv.notify_all();
    return HE_OK;
}

int he_server_poll(he_server *s, uint64_t ticket, int *done)
{
    if (!s || !done) return HE_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->status.find(ticket);
    if (it == s->status.end()) return HE_EINVAL;
    *done = it->second > 0 ? 1 : 0;
    return it->second < 0 ? -it->second : HE_OK;
}

int he_server_wait(he_server *s, uint64_t ticket, int timeout_ms)
{
    if (!s) return HE_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->status.find(ticket);
    if (it == s->status.end()) return HE_EINVAL;
    const bool ok = s->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                   [&] { return s->status[ticket] != 0; });
    if (!ok) return HE_ETIMEOUT;
    const int st = s->status[ticket];
    return st > 0 ? HE_OK : -st;
}

int he_server_stats(he_server *s, he_server_report *out)
{
    if (!s || !out) return HE_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    memset(out, 0, sizeof(*out));
    out->completed = s->completed;
    out->pending = s->pending.size();
    out->batches = s->batches;
    out->mean_batch = s->batches ? (double)s->batched_requests / (double)s->batches : 0.0;
    std::vector<double> l = s->latencies_ms;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto pct = [&](double p) { return l[std::min(l.size() - 1, (size_t)(p * (l.size() - 1) + 0.5))]; };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        out->max_ms = l.back();
        double span = std::chrono::duration<double>(s->t_last - s->t_first).count();
        out->throughput = span > 0 ? (double)s->completed / span : 0.0;
    }
    return HE_OK;
}

int he_server_destroy(he_server *s)
{
    if (!s) return HE_EINVAL;
    s->stop.store(true);
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (Flight &f : s->flights) {
        if (f.stream) cudaStreamSynchronize(f.stream);
        if (f.done) cudaEventDestroy(f.done);
        if (f.stream) cudaStreamDestroy(f.stream);
    }
    if (s->arena_mem) cudaFree(s->arena_mem);
    delete s->arena;
    delete s;
    return HE_OK;
}

}  // extern "C"
