// Request queue with continuous batching (serving).
//
// pac_submit appends a request and returns at once.  A scheduler thread
// admits waiting requests in arrival order as soon as a slot and device
// memory are free (at most max_inflight running, running bytes within the
// HBM budget), launches each on its own stream
// of a pool so that requests overlap on the GPU, and marks completion from a
// host callback enqueued behind the request's kernels.  Requests that arrive
// while others run are admitted as earlier ones finish: the batch on the
// device changes continuously instead of in waves.
//
// Quality of service: a request is "small" when its device bytes (2 N S) are
// at most 8 MiB.  Small requests run on high-priority streams (the GPU's
// block scheduler starts their CTAs before those of large requests as SMs
// free up) and a quarter of the slots is kept for them, so a burst of large
// requests cannot hold every slot while small ones wait; within each class
// admission stays in arrival order.  Large complex FP64 requests are bound by
// the FP64 pipe (on GB300 a fraction of the FP32 rate) and take milliseconds
// each: at most two of them run at once (PAC_QUEUE_FP64_LARGE overrides), so
// that a burst of them cannot fill the SMs for long stretches while smaller
// requests wait behind their CTAs.
//
// Fault injection (host side only, no device fault): the environment
// variable PAC_FAULT=launch:K makes the K-th admitted request (1-based) fail
// as if its launch had failed; the request is marked PAC_ERR_CUDA and the
// others proceed.
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <thread>
#include <unordered_map>

#include "pac_internal.h"

namespace pac {
int run_convolve(pac_plan p, const void* x, void* y, cudaStream_t s, bool allow_single);
}

using namespace pac;
using Clock = std::chrono::steady_clock;

constexpr size_t kSmallBytes = size_t(8) << 20;  // requests up to this many device bytes are "small"

namespace {

struct Request {
    uint64_t ticket = 0;
    pac_plan plan = nullptr;
    const void* x = nullptr;
    void* y = nullptr;
    size_t bytes = 0;
    Clock::time_point t_submit;
    Clock::time_point t_done;
    int status = PAC_PENDING;
    int slot = -1;
    bool small = false;
    bool fp64 = false;
    std::atomic<bool> gpu_done{false};
    pac_queue owner = nullptr;
};

}  // namespace

struct pac_queue_s {
    size_t budget = 0;
    int max_inflight = 1;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;       // wakes the scheduler
    std::condition_variable cv_done;  // wakes pac_queue_drain
    std::deque<Request*> waiting;        // large requests, arrival order
    std::deque<Request*> waiting_small;  // small requests, arrival order
    std::vector<Request*> running;
    int running_large = 0;
    int running_large_fp64 = 0;
    int max_large_fp64 = 2;              // large complex FP64 requests running at once
    int reserve_small = 1;               // slots large requests may not take
    std::vector<int> slot_small;         // slot's stream has high priority
    std::unordered_map<uint64_t, Request*> by_ticket;
    std::vector<cudaStream_t> streams;
    std::vector<int> slot_busy;
    size_t running_bytes = 0;
    uint64_t next_ticket = 1;
    uint64_t admitted = 0;
    int64_t fault_launch = -1;
    bool stop = false;
    std::thread worker;
};

static void CUDART_CB on_request_done(void* arg) {
    // runs on a CUDA driver thread once the request's kernels finished: no CUDA calls here
    Request* r = static_cast<Request*>(arg);
    r->t_done = Clock::now();
    r->gpu_done.store(true, std::memory_order_release);
    pac_queue q = r->owner;
    {
        std::lock_guard<std::mutex> lk(q->mu);
    }
    q->cv.notify_one();
}

// Admission: a free slot, and the running requests' device bytes plus this
// one within the HBM budget.  A request larger than the whole budget runs
// alone rather than never.
static bool fits(pac_queue q, const Request* r) {
    if ((int)q->running.size() >= q->max_inflight) return false;
    if (!r->small && q->running_large >= q->max_inflight - q->reserve_small) return false;
    if (!r->small && r->fp64 && q->running_large_fp64 >= q->max_large_fp64) return false;
    if (q->running.empty()) return true;
    return q->running_bytes + r->bytes <= q->budget;
}

// a free slot of the request's class (high-priority streams for small requests), else any free slot
static int pick_slot(pac_queue q, const Request* r) {
    int any = -1;
    for (int s = 0; s < (int)q->slot_busy.size(); ++s) {
        if (q->slot_busy[s]) continue;
        if ((q->slot_small[s] != 0) == r->small) return s;
        if (any < 0) any = s;
    }
    return any;
}

static void scheduler(pac_queue q) {
    cudaSetDevice(q->device);
    std::unique_lock<std::mutex> lk(q->mu);
    while (true) {
        bool progress = false;
        // retire finished requests
        for (size_t i = 0; i < q->running.size();) {
            Request* r = q->running[i];
            if (r->gpu_done.load(std::memory_order_acquire)) {
                r->status = PAC_OK;
                q->running_bytes -= r->bytes;
                if (!r->small) --q->running_large;
                if (!r->small && r->fp64) --q->running_large_fp64;
                q->slot_busy[r->slot] = 0;
                q->running[i] = q->running.back();
                q->running.pop_back();
                progress = true;
            } else {
                ++i;
            }
        }
        // admit in arrival order within each class (small first) while a slot and memory are free
        while (true) {
            std::deque<Request*>* from = nullptr;
            if (!q->waiting_small.empty() && fits(q, q->waiting_small.front()))
                from = &q->waiting_small;
            else if (!q->waiting.empty() && fits(q, q->waiting.front()))
                from = &q->waiting;
            if (!from) break;
            Request* r = from->front();
            from->pop_front();
            const int slot = pick_slot(q, r);
            r->slot = slot;
            q->admitted++;
            int rc;
            if (q->fault_launch > 0 && (int64_t)q->admitted == q->fault_launch) {
                rc = PAC_ERR_CUDA;  // injected host-side launch failure
            } else {
                // per-pass launches: requests on different streams interleave on the SMs
                rc = run_convolve(r->plan, r->x, r->y, q->streams[slot], false);
                if (rc == PAC_OK) {
                    cudaError_t e = cudaLaunchHostFunc(q->streams[slot], on_request_done, r);
                    if (e != cudaSuccess) rc = PAC_ERR_CUDA;
                }
            }
            if (rc != PAC_OK) {
                r->status = rc;
                r->t_done = Clock::now();
                progress = true;
                continue;
            }
            q->slot_busy[slot] = 1;
            q->running_bytes += r->bytes;
            if (!r->small) ++q->running_large;
            if (!r->small && r->fp64) ++q->running_large_fp64;
            q->running.push_back(r);
            progress = true;
        }
        if (progress) q->cv_done.notify_all();
        if (q->stop && q->waiting.empty() && q->waiting_small.empty() && q->running.empty()) break;
        if (!progress) q->cv.wait_for(lk, std::chrono::microseconds(200));
    }
}

extern "C" int pac_queue_create(size_t hbm_budget_bytes, int max_inflight, pac_queue* out) {
    if (!out) return fail(PAC_ERR_ARG, "null out");
    *out = nullptr;
    if (max_inflight < 1 || max_inflight > 64) return fail(PAC_ERR_ARG, "max_inflight must be in [1, 64]");
    if (hbm_budget_bytes == 0) return fail(PAC_ERR_ARG, "zero HBM budget");
    pac_queue q = new (std::nothrow) pac_queue_s();
    if (!q) return fail(PAC_ERR_NOMEM, "host allocation failed");
    q->budget = hbm_budget_bytes;
    q->max_inflight = max_inflight;
    cudaError_t e = cudaGetDevice(&q->device);
    if (e != cudaSuccess) {
        delete q;
        return cuda_fail(e, "cudaGetDevice");
    }
    size_t free_b = 0, total_b = 0;  // the admission budget is at most the device memory free now
    e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) {
        delete q;
        return cuda_fail(e, "cudaMemGetInfo");
    }
    if (free_b < q->budget) q->budget = free_b;
    q->streams.resize(max_inflight);
    q->slot_busy.assign(max_inflight, 0);
    q->reserve_small = max_inflight >= 4 ? max_inflight / 4 : (max_inflight > 1 ? 1 : 0);
    q->slot_small.assign(max_inflight, 0);
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);  // numerically lower = higher priority
    for (int i = 0; i < max_inflight; ++i) {
        q->slot_small[i] = i < q->reserve_small ? 1 : (i % 2);  // the reserved slots, then every other one
        e = cudaStreamCreateWithPriority(&q->streams[i], cudaStreamNonBlocking, q->slot_small[i] ? prio_hi : prio_lo);
        if (e != cudaSuccess) {
            for (int j = 0; j < i; ++j) cudaStreamDestroy(q->streams[j]);
            delete q;
            return cuda_fail(e, "cudaStreamCreate");
        }
    }
    if (const char* f = std::getenv("PAC_QUEUE_FP64_LARGE")) {
        const int v = std::atoi(f);
        if (v >= 1) q->max_large_fp64 = v;
    }
    if (const char* f = std::getenv("PAC_FAULT")) {
        if (std::strncmp(f, "launch:", 7) == 0) q->fault_launch = std::atoll(f + 7);
    }
    q->worker = std::thread(scheduler, q);
    *out = q;
    return PAC_OK;
}

extern "C" int pac_submit(pac_queue q, pac_plan p, const void* x_dev, void* y_dev, uint64_t* ticket) {
    if (!q || !p || !x_dev || !y_dev || !ticket) return fail(PAC_ERR_ARG, "null argument");
    if (!p->has_spec) return fail(PAC_ERR_NO_SPECTRUM, "plan has no filter spectrum");
    Request* r = new (std::nothrow) Request();
    if (!r) return fail(PAC_ERR_NOMEM, "host allocation failed");
    r->plan = p;
    r->x = x_dev;
    r->y = y_dev;
    r->bytes = 2 * (size_t)p->bytes();
    r->small = r->bytes <= kSmallBytes;
    r->fp64 = p->dtype != PAC_C64;  // complex FP64 arrays (either arithmetic)
    r->owner = q;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(q->mu);
        if (q->waiting.size() + q->waiting_small.size() >= 65536) {
            delete r;
            return fail(PAC_ERR_BUSY, "request queue full");
        }
        r->ticket = q->next_ticket++;
        (r->small ? q->waiting_small : q->waiting).push_back(r);
        q->by_ticket[r->ticket] = r;
        *ticket = r->ticket;
    }
    q->cv.notify_one();
    return PAC_OK;
}

extern "C" int pac_poll(pac_queue q, uint64_t ticket, double* latency_us) {
    if (!q) return fail(PAC_ERR_ARG, "null queue");
    std::lock_guard<std::mutex> lk(q->mu);
    auto it = q->by_ticket.find(ticket);
    if (it == q->by_ticket.end()) return fail(PAC_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
    Request* r = it->second;
    if (r->status == PAC_PENDING) return PAC_PENDING;
    const int st = r->status;
    if (latency_us) latency_us[0] = std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count();
    q->by_ticket.erase(it);
    delete r;
    if (st != PAC_OK) return fail(st, "request %llu failed", (unsigned long long)ticket);
    return PAC_OK;
}

extern "C" int pac_queue_drain(pac_queue q, int timeout_ms) {
    if (!q) return fail(PAC_ERR_ARG, "null queue");
    std::unique_lock<std::mutex> lk(q->mu);
    bool ok = q->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                  [&] { return q->waiting.empty() && q->waiting_small.empty() && q->running.empty(); });
    return ok ? PAC_OK : fail(PAC_ERR_TIMEOUT, "queue did not drain within %d ms", timeout_ms);
}

extern "C" int pac_queue_destroy(pac_queue q) {
    if (!q) return fail(PAC_ERR_ARG, "null queue");
    int rc = pac_queue_drain(q, 60000);
    {
        std::lock_guard<std::mutex> lk(q->mu);
        q->stop = true;
        if (rc != PAC_OK) {  // give up on waiting requests; running ones still finish
            for (Request* r : q->waiting) r->status = PAC_ERR_TIMEOUT;
            for (Request* r : q->waiting_small) r->status = PAC_ERR_TIMEOUT;
            q->waiting.clear();
            q->waiting_small.clear();
        }
    }
    q->cv.notify_all();
    q->worker.join();
    for (cudaStream_t s : q->streams) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    for (auto& kv : q->by_ticket) delete kv.second;
    delete q;
    return rc;
}
