// server.cu -- continuous-batching sort server (include/bitsort.h, serving
// section).
//
// A scheduler thread owns the device side:
//   * requests wait in arrival order; the head request is admitted while the
//     bytes its bitmap and output need, ceil(M/8) + 4n, fit in what is left of
//     the budget after the admitted requests and the device memory the
//     streams' contexts hold (for a large request, plus the growth of that
//     memory its plain sort asks for); strict FIFO, so a large request is
//     never starved;
//   * admitted work is launched at once as batches: a request of at least
//     kPlainMinKeys keys alone, as one plain sort (one kernel per phase,
//     every SM), or else the run of smaller requests at the head, up to
//     kBatchQuantum bytes of work, as one batch (one persistent launch);
//   * `max_inflight` streams, each with its own context, take the batches
//     (large requests on stream 0, one after another; small-request batches
//     on the others); a stream holds up to kDepth batches queued, so the
//     device always has the next batch in its queue while the scheduler
//     prepares more, and work on different streams overlaps on the device;
//     a stream that still has work queued takes only full batches, so that
//     small requests gather into few launches while the device is busy;
//   * a finished batch (its event has completed) releases its budget, and its
//     requests' outcomes (copied to pinned host memory behind the kernel) are
//     handed to the waiters together with their latency, measured from
//     submission to the moment the scheduler saw the batch complete.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "engine.h"
#include "internal.h"

namespace {

using clock_type = std::chrono::steady_clock;

struct Request {
    const uint32_t *keys = nullptr;
    uint32_t *out = nullptr;
    uint64_t n = 0;
    uint32_t max_value = 0;
    uint64_t bytes = 0;
    clock_type::time_point submitted;
    bool done = false;
    bitsort_status_t status = BITSORT_OK;
    uint64_t count = 0;
    double latency = 0;
};

struct Lane {                     // one stream and the context of its plain sorts
    cudaStream_t stream = nullptr;
    bitsort_ctx *ctx = nullptr;
    uint32_t queued = 0;             // batches launched on it and not yet finished
    std::deque<size_t> inflight;     // their batch records, in launch order (they finish in that order)
};

struct Batch {                    // one launched unit of work and its outcome buffers
    int lane = -1;
    cudaEvent_t done = nullptr;
    // kMaxBatch outcomes: written by the kernels straight into mapped pinned
    // host memory (dev_results is its device address); without mapping, a
    // device buffer copied to host_results behind the kernels
    bitsort_result_t *dev_results = nullptr;
    bitsort_result_t *host_results = nullptr;
    bool mapped = false;
    void *staging = nullptr;                   // pinned host copy of the batch plan's tables
    size_t staging_cap = 0;
    bool busy = false;
    uint64_t seq = 0;                          // launch order (finished in order per lane)
    std::vector<uint64_t> tickets;
};

constexpr size_t kMaxBatch = 1024;
// requests this large run as plain sorts (from 2^20 keys: on GB300, the
// serving benchmark's saturated mix measured 1.083x back-to-back plain calls
// at 2^20, 1.066x at 2^22 and 0.943x at 2^16: below 2^20 keys batching gains,
// above it the plain kernels' own efficiency)
constexpr uint64_t kPlainMinKeys = 1ull << 20;
constexpr uint64_t kBatchQuantum = 64ull << 20;  // work bytes (8n + M/4) of one batch of small requests
constexpr size_t kStagingBytes = 1u << 20;       // pinned table staging per batch (larger plans stage on their own)
constexpr uint32_t kDepth = 4;                   // batches queued per stream of small-request batches
constexpr uint32_t kDepthLarge = 16;             // plain sorts queued on stream 0

uint64_t work_bytes(uint64_t n, uint32_t max_value) { return 8 * n + ((uint64_t)max_value + 1) / 4; }
uint64_t request_bytes(uint64_t n, uint32_t max_value) {
    const uint64_t M = (uint64_t)max_value + 1;
    return (M + 7) / 8 + 4 * n;
}
// Device memory a lane's context keeps between calls (its partition buffer
// and global bitmap, at their high-water sizes).
uint64_t lane_scratch(const bitsort_ctx *c) { return c->part_cap * 4 + c->bitmap_words * 4; }
// The scratch a plain sort of (n, max_value) asks its context for.
uint64_t plain_scratch(bitsort_ctx *c, uint64_t n, uint32_t max_value) {
    const uint64_t M = (uint64_t)max_value + 1;
    bsx_single_plan pl;
    bsx_plan_single(c->sms, c->smem_optin, bsx_lookup_config(c, n, M), n, M, false, true, pl);
    if (pl.cfg.path == BITSORT_PATH_PARTITION && pl.a.layout == bsx::LAYOUT_CAPACITY)
        return (uint64_t)pl.a.nslices * pl.a.cap * 4;
    if (pl.cfg.path == BITSORT_PATH_GLOBAL) return ((M + 31) / 32 + 3) / 4 * 16;
    return 0;
}

}  // namespace

struct bitsort_server {
    int device = 0;
    uint64_t budget = 0;
    uint64_t in_use = 0;
    uint64_t held = 0;     // device memory the lanes' contexts keep (counted against the budget)
    bitsort_ctx *ctx = nullptr;
    std::vector<Lane> lanes;
    std::vector<Batch> pool;
    std::deque<uint64_t> waiting;
    std::unordered_map<uint64_t, Request> reqs;
    uint64_t next_ticket = 1, next_seq = 1;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::thread thread;
    bool stop = false;
    bitsort_status_t fatal = BITSORT_OK;
    uint64_t completed = 0, keys = 0, batches = 0, max_concurrent = 0;

    void run();
    bool launch_batch(Batch &b, const std::vector<bitsort_desc_t> &jobs);
    void finish_batch(Batch &b);
};

// Launches one batch on its stream.  Runs without the server lock: it reads
// only `jobs` (copied under the lock) and state that the scheduler thread
// alone touches (the batch record, the streams, the scheduler's context).
bool bitsort_server::launch_batch(Batch &b, const std::vector<bitsort_desc_t> &jobs) {
    if (!b.host_results) return false;
    if (!b.staging) {
        if (cudaMallocHost(&b.staging, kStagingBytes) != cudaSuccess) return false;
        b.staging_cap = kStagingBytes;
    }
    Lane &ln = lanes[b.lane];
    bitsort_status_t st = BITSORT_OK;
    const bitsort_desc_t &j0 = jobs[0];
    if (jobs.size() == 1 && j0.n >= kPlainMinKeys) {
        st = bitsort_ex(ln.ctx, j0.keys, j0.n, j0.max_value, j0.out, b.dev_results,
                        reinterpret_cast<bitsort_stream_t>(ln.stream));
    } else {
        bitsort_batch_plan *pl = nullptr;
        st = bsx_plan_build(ctx, jobs.data(), jobs.size(), b.dev_results, ln.stream, true, &pl, b.staging,
                            b.staging_cap);
        if (st != BITSORT_OK) return false;
        st = bsx_plan_launch_direct(pl, ln.stream);
        bsx_plan_release_async(pl, ln.stream);
    }
    if (!b.mapped)
        cudaMemcpyAsync(b.host_results, b.dev_results, jobs.size() * sizeof(bitsort_result_t),
                        cudaMemcpyDeviceToHost, ln.stream);
    cudaEventRecord(b.done, ln.stream);
    b.seq = next_seq++;
    ++ln.queued;
    return st == BITSORT_OK;
}

void bitsort_server::finish_batch(Batch &b) {
    const auto now = clock_type::now();
    for (size_t i = 0; i < b.tickets.size(); ++i) {
        auto it = reqs.find(b.tickets[i]);
        if (it == reqs.end()) continue;
        Request &r = it->second;
        r.status = (bitsort_status_t)b.host_results[i].status;
        r.count = b.host_results[i].count;
        r.latency = std::chrono::duration<double>(now - r.submitted).count();
        r.done = true;
        in_use -= r.bytes;
        ++completed;
        keys += r.n;
    }
    b.tickets.clear();
    b.busy = false;
    --lanes[b.lane].queued;
}

void bitsort_server::run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        bool progressed = false;
        uint64_t busy = 0;
        // a stream's batches finish in launch order: only its oldest one is
        // asked whether it is done
        for (Lane &ln : lanes) {
            while (!ln.inflight.empty() && cudaEventQuery(pool[ln.inflight.front()].done) == cudaSuccess) {
                finish_batch(pool[ln.inflight.front()]);
                ln.inflight.pop_front();
                progressed = true;
            }
            busy += ln.inflight.size();
        }
        if (progressed) cv_done.notify_all();
        while (!waiting.empty()) {
            // a free batch record and the stream with the fewest queued batches
            Batch *b = nullptr;
            for (Batch &x : pool)
                if (!x.busy) {
                    b = &x;
                    break;
                }
            // large requests run one after another on stream 0, as a plain
            // caller's would (concurrent large sorts only contend for the L2
            // that each one's partition pass fills for its bucket pass);
            // batches of small requests take the least loaded other stream
            const bool head_large = reqs[waiting.front()].n >= kPlainMinKeys;
            const int first = (!head_large && lanes.size() > 1) ? 1 : 0;
            const int last = head_large ? 1 : (int)lanes.size();
            int lane = -1;
            for (int i = first; i < last; ++i) {
                const uint32_t depth = (i == 0 && lanes.size() > 1) ? kDepthLarge : kDepth;
                if (lanes[i].queued < depth && (lane < 0 || lanes[i].queued < lanes[lane].queued)) lane = i;
            }
            if (!b || lane < 0) break;
            if (lanes[lane].queued > 0) {
                // the device has work: launch only a full batch (a large
                // request, or small ones worth a quantum), so that small
                // requests gather into few launches; an idle stream takes
                // whatever is waiting
                bool full = false;
                uint64_t w = 0;
                size_t k = 0;
                for (auto it = waiting.begin(); it != waiting.end() && !full; ++it) {
                    const Request &r = reqs[*it];
                    w += work_bytes(r.n, r.max_value);
                    full = r.n >= kPlainMinKeys || w >= kBatchQuantum || ++k >= kMaxBatch;
                }
                if (!full) break;
            }
            // the head request alone if it is large, else the run of small
            // requests at the head up to one quantum of work (FIFO admission)
            std::vector<uint64_t> batch;
            uint64_t work = 0;
            while (!waiting.empty() && batch.size() < kMaxBatch) {
                Request &r = reqs[waiting.front()];
                const bool large = r.n >= kPlainMinKeys;
                if (large && !batch.empty()) break;
                // a plain sort may grow its lane's buffers, which then stay
                // held: that growth is charged too
                uint64_t growth = 0;
                if (large) {
                    const uint64_t need = plain_scratch(lanes[lane].ctx, r.n, r.max_value);
                    const uint64_t have = lane_scratch(lanes[lane].ctx);
                    growth = need > have ? need - have : 0;
                }
                if (in_use + held + growth + r.bytes > budget) break;
                in_use += r.bytes;
                batch.push_back(waiting.front());
                waiting.pop_front();
                work += work_bytes(r.n, r.max_value);
                if (large || work >= kBatchQuantum) break;
            }
            if (batch.empty()) break;
            std::vector<bitsort_desc_t> jobs(batch.size());
            for (size_t i = 0; i < batch.size(); ++i) {
                const Request &r = reqs[batch[i]];
                jobs[i].keys = r.keys;
                jobs[i].out = r.out;
                jobs[i].n = r.n;
                jobs[i].max_value = r.max_value;
                jobs[i].reserved = 0;
            }
            b->lane = lane;
            b->tickets = batch;
            b->busy = true;   // reserved: only this thread finishes batches
            // launch without the lock, so that submissions are not held up
            lk.unlock();
            const uint32_t before = lanes[lane].queued;
            const bool ok = launch_batch(*b, jobs);
            lk.lock();
            held = 0;
            for (const Lane &ln : lanes) held += lane_scratch(ln.ctx);
            ++batches;
            if (!ok) {
                fatal = BITSORT_ERR_CUDA;
                for (uint64_t t : batch) {
                    Request &r = reqs[t];
                    r.status = BITSORT_ERR_CUDA;
                    r.done = true;
                    in_use -= r.bytes;
                }
                if (lanes[lane].queued > before) --lanes[lane].queued;
                b->busy = false;
                b->tickets.clear();
                cv_done.notify_all();
                continue;
            }
            lanes[lane].inflight.push_back((size_t)(b - pool.data()));
            ++busy;
            progressed = true;
        }
        if (busy > max_concurrent) max_concurrent = busy;
        if (stop && waiting.empty() && busy == 0) break;
        if (!progressed) {
            if (busy > 0) {
                // a timed sleep lasts tens of microseconds (timer slack): poll
                // the batches' events between yields while work is in flight
                lk.unlock();
                std::this_thread::yield();
                lk.lock();
            } else {
                cv_sched.wait_for(lk, std::chrono::milliseconds(2));
            }
        }
    }
}

extern "C" bitsort_status_t bitsort_server_create(int device, uint64_t budget_bytes, int max_inflight,
                                                  bitsort_server_t **out) {
    if (!out || budget_bytes == 0 || max_inflight < 1 || max_inflight > 64) return BITSORT_ERR_INVALID;
    *out = nullptr;
    bitsort_server *sv = new (std::nothrow) bitsort_server();
    if (!sv) return BITSORT_ERR_NOMEM;
    bitsort_status_t st = bitsort_ctx_create(device, &sv->ctx);
    if (st != BITSORT_OK) {
        delete sv;
        return st;
    }
    sv->device = device;
    sv->budget = budget_bytes;
    // batch plans allocate their tables and scratch stream-ordered: keep the
    // device's pool from handing that memory back to the system at every
    // synchronisation (its default), which would make each plan allocate anew
    cudaMemPool_t pool = nullptr;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    sv->lanes.resize(max_inflight);
    // stream 0 (large requests, one after another) at the lowest priority,
    // the batch streams at the highest: the block scheduler then starts a
    // batch's CTAs as soon as a large sort's CTAs free an SM, instead of
    // queueing them behind the large sort's remaining waves
    int prio_low = 0, prio_high = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high) != cudaSuccess) prio_low = prio_high = 0;
    for (size_t li = 0; li < sv->lanes.size(); ++li) {
        Lane &ln = sv->lanes[li];
        const int prio = (li == 0 && sv->lanes.size() > 1) ? prio_low : prio_high;
        if (cudaStreamCreateWithPriority(&ln.stream, cudaStreamNonBlocking, prio) != cudaSuccess ||
            bitsort_ctx_create(device, &ln.ctx) != BITSORT_OK) {
            bitsort_server_destroy(sv);
            return BITSORT_ERR_CUDA;
        }
        ln.ctx->stream_ordered = true;   // used on this stream only
    }
    sv->pool.resize((size_t)max_inflight * kDepth + kDepthLarge);
    int can_map = 0;
    cudaDeviceGetAttribute(&can_map, cudaDevAttrCanMapHostMemory, device);
    for (Batch &b : sv->pool) {
        if (cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming) != cudaSuccess) {
            bitsort_server_destroy(sv);
            return BITSORT_ERR_CUDA;
        }
        const size_t bytes = kMaxBatch * sizeof(bitsort_result_t);
        void *dev = nullptr;
        if (can_map && cudaHostAlloc(reinterpret_cast<void **>(&b.host_results), bytes, cudaHostAllocMapped) ==
                           cudaSuccess &&
            cudaHostGetDevicePointer(&dev, b.host_results, 0) == cudaSuccess) {
            b.dev_results = static_cast<bitsort_result_t *>(dev);
            b.mapped = true;
        } else {
            cudaGetLastError();
            if (b.host_results) cudaFreeHost(b.host_results);
            b.host_results = nullptr;
            if (cudaMallocHost(&b.host_results, bytes) != cudaSuccess ||
                cudaMalloc(&b.dev_results, bytes) != cudaSuccess) {
                bitsort_server_destroy(sv);
                return BITSORT_ERR_CUDA;
            }
        }
    }
    sv->thread = std::thread([sv] { sv->run(); });
    *out = sv;
    return BITSORT_OK;
}

extern "C" bitsort_status_t bitsort_server_submit(bitsort_server_t *sv, const uint32_t *keys, uint64_t n,
                                                  uint32_t max_value, uint32_t *out, uint64_t *ticket) {
    bsx_range nvtx_range_("bitsort_server_submit");
    if (!sv || !ticket) return BITSORT_ERR_INVALID;
    bitsort_status_t st = bsx_validate(keys, n, max_value, out);
    if (st != BITSORT_OK) return st;
    const uint64_t bytes = request_bytes(n, max_value);
    if (bytes > sv->budget) return BITSORT_ERR_BUDGET;
    if (n >= kPlainMinKeys && bytes + plain_scratch(sv->ctx, n, max_value) > sv->budget) return BITSORT_ERR_BUDGET;
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) return BITSORT_ERR_INVALID;
    const uint64_t t = sv->next_ticket++;
    Request &r = sv->reqs[t];
    r.keys = keys;
    r.out = out;
    r.n = n;
    r.max_value = max_value;
    r.bytes = bytes;
    r.submitted = clock_type::now();
    sv->waiting.push_back(t);
    *ticket = t;
    sv->cv_sched.notify_one();
    return BITSORT_OK;
}

extern "C" bitsort_status_t bitsort_server_wait(bitsort_server_t *sv, uint64_t ticket, bitsort_status_t *status,
                                                uint64_t *count, double *latency_s) {
    if (!sv) return BITSORT_ERR_INVALID;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return BITSORT_ERR_INVALID;
    sv->cv_done.wait(lk, [&] { return sv->reqs[ticket].done; });
    Request r = sv->reqs[ticket];
    sv->reqs.erase(ticket);
    if (status) *status = r.status;
    if (count) *count = r.count;
    if (latency_s) *latency_s = r.latency;
    if (r.status == BITSORT_ERR_TIMEOUT) return BITSORT_ERR_TIMEOUT;
    return r.status == BITSORT_ERR_CUDA ? BITSORT_ERR_CUDA : BITSORT_OK;
}

extern "C" bitsort_status_t bitsort_server_stats(bitsort_server_t *sv, uint64_t *completed, uint64_t *keys,
                                                 uint64_t *batches, uint64_t *max_concurrent) {
    if (!sv) return BITSORT_ERR_INVALID;
    std::lock_guard<std::mutex> lk(sv->mu);
    if (completed) *completed = sv->completed;
    if (keys) *keys = sv->keys;
    if (batches) *batches = sv->batches;
    if (max_concurrent) *max_concurrent = sv->max_concurrent;
    return BITSORT_OK;
}

extern "C" bitsort_status_t bitsort_server_destroy(bitsort_server_t *sv) {
    if (!sv) return BITSORT_ERR_INVALID;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->cv_sched.notify_all();
    }
    if (sv->thread.joinable()) sv->thread.join();
    cudaSetDevice(sv->device);
    for (Lane &ln : sv->lanes)
        if (ln.stream) cudaStreamSynchronize(ln.stream);
    for (Batch &b : sv->pool) {
        if (b.done) cudaEventDestroy(b.done);
        if (b.host_results) cudaFreeHost(b.host_results);
        if (b.staging) cudaFreeHost(b.staging);
        if (b.dev_results && !b.mapped) cudaFree(b.dev_results);
    }
    for (Lane &ln : sv->lanes) {
        if (ln.stream) cudaStreamDestroy(ln.stream);
        if (ln.ctx) bitsort_ctx_destroy(ln.ctx);
    }
    if (sv->ctx) bitsort_ctx_destroy(sv->ctx);
    delete sv;
    return BITSORT_OK;
}
