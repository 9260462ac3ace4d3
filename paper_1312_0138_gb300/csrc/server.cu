// server.cu -- continuous-batching sort server (include/bitsort.h, serving
// section).
//
// A scheduler thread owns the device side:
//   * requests wait in arrival order; the head request is admitted while the
//     bytes its bitmap and output need, ceil(M/8) + 4n, fit in what is left of
//     the budget (strict FIFO, so a large request is never starved);
//   * whenever one of `max_inflight` slots (a stream and a context each) is
//     free and admitted requests are waiting, they are launched on that
//     slot's stream: requests of at least kPlainMinKeys keys each as one
//     plain sort (one kernel per phase, every SM), the smaller ones together
//     as one batch (one persistent launch); work launched while other slots
//     run overlaps with it on the device;
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

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bitsort_ctx *ctx = nullptr;                // scratch of this slot's plain sorts
    bitsort_result_t *dev_results = nullptr;   // kMaxBatch outcomes on the device
    bitsort_result_t *host_results = nullptr;  // pinned
    size_t host_cap = 0;
    bool busy = false;
    std::vector<uint64_t> tickets;
    uint64_t bytes = 0;
};

constexpr size_t kMaxBatch = 1024;
constexpr uint64_t kPlainMinKeys = 1ull << 20;   // requests this large run as plain sorts

uint64_t request_bytes(uint64_t n, uint32_t max_value) {
    const uint64_t M = (uint64_t)max_value + 1;
    return (M + 7) / 8 + 4 * n;
}

}  // namespace

struct bitsort_server {
    int device = 0;
    uint64_t budget = 0;
    uint64_t in_use = 0;
    bitsort_ctx *ctx = nullptr;
    std::vector<Slot> slots;
    std::deque<uint64_t> waiting;
    std::unordered_map<uint64_t, Request> reqs;
    uint64_t next_ticket = 1;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::thread thread;
    bool stop = false;
    bitsort_status_t fatal = BITSORT_OK;
    uint64_t completed = 0, keys = 0, batches = 0, max_concurrent = 0;

    void run();
    bool launch_batch(Slot &s, std::vector<uint64_t> &batch);
    void finish_batch(Slot &s);
};

bool bitsort_server::launch_batch(Slot &s, std::vector<uint64_t> &batch) {
    if (!s.host_results) {
        if (cudaMallocHost(&s.host_results, kMaxBatch * sizeof(bitsort_result_t)) != cudaSuccess) return false;
        s.host_cap = kMaxBatch;
    }
    // large requests first (plain sorts), then the small ones (one batch);
    // outcome i of the slot belongs to ticket i of the reordered list
    std::stable_partition(batch.begin(), batch.end(), [&](uint64_t t) { return reqs[t].n >= kPlainMinKeys; });
    size_t nplain = 0;
    while (nplain < batch.size() && reqs[batch[nplain]].n >= kPlainMinKeys) ++nplain;
    bitsort_status_t st = BITSORT_OK;
    if (nplain < batch.size()) {
        std::vector<bitsort_desc_t> descs(batch.size() - nplain);
        for (size_t i = nplain; i < batch.size(); ++i) {
            const Request &r = reqs[batch[i]];
            bitsort_desc_t &d = descs[i - nplain];
            d.keys = r.keys;
            d.out = r.out;
            d.n = r.n;
            d.max_value = r.max_value;
            d.reserved = 0;
        }
        bitsort_batch_plan *pl = nullptr;
        st = bsx_plan_build(ctx, descs.data(), descs.size(), s.dev_results + nplain, s.stream, true, &pl);
        if (st != BITSORT_OK) return false;
        st = bsx_plan_launch_direct(pl, s.stream);
        bsx_plan_release_async(pl, s.stream);
    }
    for (size_t i = 0; i < nplain && st == BITSORT_OK; ++i) {
        const Request &r = reqs[batch[i]];
        st = bitsort_ex(s.ctx, r.keys, r.n, r.max_value, r.out, s.dev_results + i,
                        reinterpret_cast<bitsort_stream_t>(s.stream));
    }
    cudaMemcpyAsync(s.host_results, s.dev_results, batch.size() * sizeof(bitsort_result_t), cudaMemcpyDeviceToHost,
                    s.stream);
    cudaEventRecord(s.done, s.stream);
    s.tickets = batch;
    s.busy = true;
    ++batches;
    return st == BITSORT_OK;
}

void bitsort_server::finish_batch(Slot &s) {
    const auto now = clock_type::now();
    for (size_t i = 0; i < s.tickets.size(); ++i) {
        auto it = reqs.find(s.tickets[i]);
        if (it == reqs.end()) continue;
        Request &r = it->second;
        r.status = (bitsort_status_t)s.host_results[i].status;
        r.count = s.host_results[i].count;
        r.latency = std::chrono::duration<double>(now - r.submitted).count();
        r.done = true;
        in_use -= r.bytes;
        ++completed;
        keys += r.n;
    }
    s.tickets.clear();
    s.busy = false;
}

void bitsort_server::run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        bool progressed = false;
        uint64_t busy = 0;
        for (Slot &s : slots) {
            if (s.busy && cudaEventQuery(s.done) == cudaSuccess) {
                finish_batch(s);
                progressed = true;
            }
            busy += s.busy ? 1 : 0;
        }
        if (progressed) cv_done.notify_all();
        size_t free_slots = 0;
        for (Slot &s : slots) free_slots += s.busy ? 0 : 1;
        for (Slot &s : slots) {
            if (s.busy || waiting.empty()) continue;
            // an even share of the waiting requests per free slot, so that a
            // burst spreads over the slots and overlaps on the device
            const size_t share = std::min(kMaxBatch, (waiting.size() + free_slots - 1) / std::max<size_t>(1, free_slots));
            --free_slots;
            std::vector<uint64_t> batch;
            while (!waiting.empty() && batch.size() < share) {
                Request &r = reqs[waiting.front()];
                if (in_use + r.bytes > budget) break;
                in_use += r.bytes;
                batch.push_back(waiting.front());
                waiting.pop_front();
            }
            if (batch.empty()) break;
            if (!launch_batch(s, batch)) {
                fatal = BITSORT_ERR_CUDA;
                for (uint64_t t : batch) {
                    Request &r = reqs[t];
                    r.status = BITSORT_ERR_CUDA;
                    r.done = true;
                    in_use -= r.bytes;
                }
                s.busy = false;
                cv_done.notify_all();
                continue;
            }
            ++busy;
            progressed = true;
        }
        if (busy > max_concurrent) max_concurrent = busy;
        if (stop && waiting.empty() && busy == 0) break;
        if (!progressed) {
            if (busy > 0) {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(5));
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
    sv->slots.resize(max_inflight);
    for (Slot &s : sv->slots) {
        if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess ||
            bitsort_ctx_create(device, &s.ctx) != BITSORT_OK ||
            cudaMalloc(&s.dev_results, kMaxBatch * sizeof(bitsort_result_t)) != cudaSuccess) {
            bitsort_server_destroy(sv);
            return BITSORT_ERR_CUDA;
        }
    }
    sv->thread = std::thread([sv] { sv->run(); });
    *out = sv;
    return BITSORT_OK;
}

extern "C" bitsort_status_t bitsort_server_submit(bitsort_server_t *sv, const uint32_t *keys, uint64_t n,
                                                  uint32_t max_value, uint32_t *out, uint64_t *ticket) {
    if (!sv || !ticket) return BITSORT_ERR_INVALID;
    bitsort_status_t st = bsx_validate(keys, n, max_value, out);
    if (st != BITSORT_OK) return st;
    const uint64_t bytes = request_bytes(n, max_value);
    if (bytes > sv->budget) return BITSORT_ERR_BUDGET;
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
    for (Slot &s : sv->slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
        if (s.done) cudaEventDestroy(s.done);
        if (s.stream) cudaStreamDestroy(s.stream);
        if (s.host_results) cudaFreeHost(s.host_results);
        if (s.dev_results) cudaFree(s.dev_results);
        if (s.ctx) bitsort_ctx_destroy(s.ctx);
    }
    if (sv->ctx) bitsort_ctx_destroy(sv->ctx);
    delete sv;
    return BITSORT_OK;
}
