// batch.cu -- many independent arrays sorted by ONE persistent launch of the
// engine kernel (include/bitsort.h, batching section), replayed from a CUDA
// graph.
//
// Every array gets its own strategy (fused single slice, partition, or global
// bitmap), its own scratch and its own outcome.  The work items of all arrays
// form one ticket sequence:
//   1. single-slice (fused) arrays, largest first, so that the longest items
//      start first (longest-processing-time order);
//   2. the multi-slice arrays, largest first, in a skewed pipeline: at stage
//      k the first phase (HIST or GSCATTER) of array k, the PART phase of
//      array k-L and the slice phase (BUCKET or GSCAN) of array k-2L.  An item
//      only waits for earlier phases of its own array, which are at least one
//      stage earlier in the sequence, so waits are short and never circular.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include <stdio.h>

#include "engine.h"
#include "internal.h"

using namespace bsx;

namespace {

constexpr uint64_t kFusedMaxM = 1ull << 20;
constexpr int kLag = 2;
constexpr uint64_t kGroupSlicesWithKeys = 32;   // slices with keys a bucket item meets, at most about

inline size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }
inline uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

}  // namespace

struct bitsort_batch_plan {
    bitsort_ctx *ctx = nullptr;
    size_t count = 0;
    int threads = 512;
    uint32_t smem = 0;
    int grid = 1;
    void *tables = nullptr;    // arrays table, segments, results, ticket
    void *scratch = nullptr;   // per-array scratch (zero at rest)
    size_t scratch_bytes = 0;
    bool async_alloc = false;
    bitsort_result_t *d_results = nullptr;
    EngineParams params;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<bsx_config> cfg;
};

// Per-array configuration inside a batch, from the context's batch policy:
// an array whose values fit one slice (M <= policy.S) is sorted by one fused
// slice; a larger one takes the policy's path (shared-memory slices after a
// partition, or the global L2 bitmap) with slices of policy.S values.  One
// persistent launch: every item waits for its own array's earlier phases;
// exact bucket ranges, so the partition buffer is the output (or an n-entry
// plan buffer when sorting in place).
static bsx_config batch_config(bitsort_ctx *c, uint64_t n, uint64_t M, int threads) {
    bsx_config cfg = c->batch;
    cfg.threads = threads;
    cfg.persistent = true;
    cfg.layout = LAYOUT_EXACT;
    cfg.emit = EMIT_WORD;
    if (n == 0) {
        cfg.path = BITSORT_PATH_FUSED;
        cfg.S = 128;
        return cfg;
    }
    if (M <= std::min<uint64_t>(c->batch.S, kFusedMaxM)) cfg.path = BITSORT_PATH_FUSED;
    cfg = bsx_sanitize(cfg, n, M);
    cfg.persistent = true;
    cfg.layout = LAYOUT_EXACT;
    cfg.emit = EMIT_WORD;
    return cfg;
}

bitsort_status_t bsx_plan_build(bitsort_ctx *c, const bitsort_desc_t *descs, size_t count,
                                   bitsort_result_t *d_results_user, cudaStream_t stream, bool async_alloc,
                                   bitsort_batch_plan **out, void *staging, size_t staging_cap) {
    *out = nullptr;
    if (count == 0 || !descs || count > (1u << 24)) return BITSORT_ERR_INVALID;
    for (size_t i = 0; i < count; ++i) {
        bitsort_status_t st = bsx_validate(descs[i].keys, descs[i].n, descs[i].max_value, descs[i].out);
        if (st != BITSORT_OK) return st;
    }
    bitsort_batch_plan *pl = new (std::nothrow) bitsort_batch_plan();
    if (!pl) return BITSORT_ERR_NOMEM;
    pl->ctx = c;
    pl->count = count;
    pl->threads = c->batch.threads == 256 ? 256 : 512;
    pl->async_alloc = async_alloc;
    const int T = pl->threads;

    // configurations and descriptors (pointers filled in below)
    std::vector<ArrayDesc> arr(count);
    pl->cfg.resize(count);
    std::vector<size_t> scr_off(count);
    size_t scr = 0;
    uint32_t smem = 0;
    for (size_t i = 0; i < count; ++i) {
        const uint64_t n = descs[i].n;
        const uint64_t M = n == 0 ? 1 : (uint64_t)descs[i].max_value + 1;
        bsx_config cfg = batch_config(c, n, M, T);
        pl->cfg[i] = cfg;
        bsx_describe(cfg, descs[i].keys, descs[i].out, n, M, arr[i]);
        if (arr[i].phased || arr[i].layout != LAYOUT_EXACT) {  // the buffers below are sized for this
            delete pl;
            return BITSORT_ERR_INVALID;
        }
        // a sparse array over a wide range (fewer than 64 keys per slice on
        // average): bucket items of several slices, about
        // kGroupSlicesWithKeys of them with keys each (item_bucket)
        if (cfg.path == BITSORT_PATH_PARTITION && arr[i].nslices > 1 && n < 64ull * arr[i].nslices) {
            const uint64_t busy = std::min<uint64_t>(n, arr[i].nslices);   // slices that can have keys
            const uint64_t items = std::max<uint64_t>(1, (busy + kGroupSlicesWithKeys - 1) / kGroupSlicesWithKeys);
            const uint64_t g = (arr[i].nslices + items - 1) / items;
            arr[i].sgroup = g > 1 ? (uint32_t)g : 1u;
        }
        smem = std::max(smem, bsx_smem_for(cfg, arr[i].nslices, arr[i].tile_keys, arr[i].stage_cap));
        scr_off[i] = scr;
        size_t need = SY_COUNT * 4;
        if (arr[i].nslices > 1) need += (size_t)arr[i].nslices * 8;                  // look-back
        if (cfg.path == BITSORT_PATH_PARTITION) {
            need += (size_t)arr[i].nslices * 16;                                    // counts, cursor, offsets
            if (descs[i].keys == descs[i].out) need += align256(n * 4);             // partition buffer
        }
        if (cfg.path == BITSORT_PATH_GLOBAL) need += align256((ceil_div(M, 32) + 3) / 4 * 16);
        scr += align256(need + 512);  // + room for the alignment padding of the layout below
    }
    if (smem > c->smem_optin) {
        delete pl;
        return BITSORT_ERR_INVALID;
    }

    // ticket order
    std::vector<Segment> segs;
    uint32_t t = 0;
    auto add = [&](uint32_t a, uint32_t type, uint32_t cnt) {
        if (cnt == 0) return;
        Segment s;
        s.start = t;
        s.array = a;
        s.type = type;
        s.first = 0;
        segs.push_back(s);
        t += cnt;
    };
    std::vector<uint32_t> fused, multi;
    for (size_t i = 0; i < count; ++i) (arr[i].nslices == 1 ? fused : multi).push_back((uint32_t)i);
    auto work = [&](uint32_t i) { return arr[i].n * 4 + arr[i].M / 8; };
    std::stable_sort(fused.begin(), fused.end(), [&](uint32_t x, uint32_t y) { return work(x) > work(y); });
    std::stable_sort(multi.begin(), multi.end(), [&](uint32_t x, uint32_t y) { return work(x) > work(y); });
    for (uint32_t i : fused) add(i, IT_BUCKET, 1);
    const int A = (int)multi.size();
    for (int k = 0; k < A + 2 * kLag; ++k) {
        if (k < A) {
            const uint32_t i = multi[k];
            add(i, arr[i].path == BITSORT_PATH_PARTITION ? IT_HIST : IT_GSCATTER, arr[i].key_tiles);
        }
        const int k2 = k - kLag;
        if (k2 >= 0 && k2 < A) {
            const uint32_t i = multi[k2];
            if (arr[i].path == BITSORT_PATH_PARTITION) add(i, IT_PART, arr[i].key_tiles);
        }
        const int k3 = k - 2 * kLag;
        if (k3 >= 0 && k3 < A) {
            const uint32_t i = multi[k3];
            const uint32_t g = arr[i].sgroup > 1 ? arr[i].sgroup : 1u;
            add(i, arr[i].path == BITSORT_PATH_PARTITION ? IT_BUCKET : IT_GSCAN, (arr[i].nslices + g - 1) / g);
        }
    }

    // device memory: tables and scratch
    const size_t off_results = 256;
    const size_t off_arrays = off_results + align256(count * sizeof(bitsort_result_t));
    const size_t off_segs = off_arrays + align256(count * sizeof(ArrayDesc));
    const size_t tables_bytes = off_segs + align256(segs.size() * sizeof(Segment));
    cudaError_t e;
    if (async_alloc) {
        e = cudaMallocAsync(&pl->tables, tables_bytes, stream);
        if (e == cudaSuccess) e = cudaMallocAsync(&pl->scratch, std::max<size_t>(scr, 256), stream);
    } else {
        e = cudaMalloc(&pl->tables, tables_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&pl->scratch, std::max<size_t>(scr, 256));
    }
    if (e != cudaSuccess) {
        if (pl->tables) (async_alloc ? cudaFreeAsync(pl->tables, stream) : cudaFree(pl->tables));
        delete pl;
        return bsx_check(e);
    }
    pl->scratch_bytes = std::max<size_t>(scr, 256);
    char *tb = (char *)pl->tables;
    char *sb = (char *)pl->scratch;
    pl->d_results = (bitsort_result_t *)(tb + off_results);
    for (size_t i = 0; i < count; ++i) {
        ArrayDesc &a = arr[i];
        char *p = sb + scr_off[i];
        a.sync = (uint32_t *)p;
        p += 64;
        if (a.nslices > 1) {
            a.look = (uint64_t *)p;
            p += (size_t)a.nslices * 8;
        }
        if (pl->cfg[i].path == BITSORT_PATH_PARTITION) {
            a.offsets = (uint64_t *)p;
            p += (size_t)a.nslices * 8;
            a.counts = (uint32_t *)p;
            p += (size_t)a.nslices * 4;
            a.cursor = (uint32_t *)p;
            p += (size_t)a.nslices * 4;
            p = sb + align256((size_t)(p - sb));
            if (descs[i].keys == descs[i].out) {
                a.part = (uint32_t *)p;
                p += align256(a.n * 4);
            } else {
                a.part = descs[i].out;
            }
        }
        if (pl->cfg[i].path == BITSORT_PATH_GLOBAL) {
            p = sb + align256((size_t)(p - sb));
            a.bitmap = (uint32_t *)p;
        }
        a.result = d_results_user ? d_results_user + i : pl->d_results + i;
    }
    const bool use_staging = async_alloc && staging && staging_cap >= tables_bytes;
    std::vector<char> host(use_staging ? 0 : tables_bytes, 0);
    char *hb = use_staging ? (char *)staging : host.data();
    memset(hb, 0, tables_bytes);
    memcpy(hb + off_arrays, arr.data(), count * sizeof(ArrayDesc));
    memcpy(hb + off_segs, segs.data(), segs.size() * sizeof(Segment));
    if (use_staging) {
        // pinned staging that the caller keeps until the stream has passed this copy
        e = cudaMemcpyAsync(pl->tables, hb, tables_bytes, cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(pl->scratch, 0, pl->scratch_bytes, stream);
    } else if (async_alloc) {
        e = cudaMemcpyAsync(pl->tables, host.data(), tables_bytes, cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(pl->scratch, 0, pl->scratch_bytes, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);  // host staging buffer goes out of scope
    } else {
        // a copy from pageable memory may return before it reaches the
        // device, and cudaMemset returns before the memory is written; both
        // run on the legacy default stream, which the caller's (possibly
        // non-blocking) launch stream does not wait for
        e = cudaMemcpy(pl->tables, host.data(), tables_bytes, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(pl->scratch, 0, pl->scratch_bytes);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        bitsort_batch_plan_destroy(pl);
        return bsx_check(e);
    }
    EngineParams &P = pl->params;
    memset(&P, 0, sizeof(P));
    P.arrays = (const ArrayDesc *)(tb + off_arrays);
    P.segments = (const Segment *)(tb + off_segs);
    P.nseg = (uint32_t)segs.size();
    P.total_items = t;
    P.ticket = (uint32_t *)tb;
    P.wait_limit_ns = c->wait_limit_ns;
    pl->smem = smem;
    pl->grid = bsx_grid_for(c, T, smem, std::max<uint32_t>(t, 1));
    *out = pl;
    return BITSORT_OK;
}

extern "C" bitsort_status_t bitsort_batch_plan_create(bitsort_ctx_t *c, const bitsort_desc_t *descs, size_t count,
                                                      bitsort_batch_plan_t **plan) {
    bsx_range nvtx_range_("bitsort_batch_plan_create");
    if (!plan) return BITSORT_ERR_INVALID;
    if (!c) c = bsx_default_ctx();
    if (!c) return BITSORT_ERR_CUDA;
    if (cudaSetDevice(c->device) != cudaSuccess) return BITSORT_ERR_CUDA;
    return bsx_plan_build(c, descs, count, nullptr, nullptr, false, plan, nullptr, 0);
}

bitsort_status_t bsx_plan_launch_direct(bitsort_batch_plan *pl, cudaStream_t s) {
    if (pl->params.total_items == 0) return BITSORT_OK;
    int e = engine_launch(pl->params, pl->threads, pl->smem, pl->grid, s);
    if (e != 0) {
        bsx_note_error(e, "batched engine launch");
        return BITSORT_ERR_CUDA;
    }
    pl->ctx->launches.fetch_add(1);
    return BITSORT_OK;
}

extern "C" bitsort_status_t bitsort_batch_plan_launch(bitsort_batch_plan_t *pl, bitsort_stream_t stream) {
    bsx_range nvtx_range_("bitsort_batch_plan_launch");
    if (!pl) return BITSORT_ERR_INVALID;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaSetDevice(pl->ctx->device) != cudaSuccess) return BITSORT_ERR_CUDA;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return BITSORT_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) return bsx_plan_launch_direct(pl, s);  // caller is capturing
    if (!pl->exec) {
        cudaStream_t cs;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return BITSORT_ERR_CUDA;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            int le = pl->params.total_items ? engine_launch(pl->params, pl->threads, pl->smem, pl->grid, cs) : 0;
            e = cudaStreamEndCapture(cs, &pl->graph);
            if (le != 0) e = cudaErrorLaunchFailure;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&pl->exec, pl->graph, 0);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) {
            if (pl->graph) cudaGraphDestroy(pl->graph);
            pl->graph = nullptr;
            pl->exec = nullptr;
            return BITSORT_ERR_CUDA;
        }
    }
    if (cudaGraphLaunch(pl->exec, s) != cudaSuccess) return BITSORT_ERR_CUDA;
    if (pl->params.total_items) pl->ctx->launches.fetch_add(1);
    return BITSORT_OK;
}

extern "C" bitsort_status_t bitsort_batch_plan_results(bitsort_batch_plan_t *pl, bitsort_stream_t stream,
                                                       bitsort_result_t *results) {
    if (!pl || !results) return BITSORT_ERR_INVALID;
    if (cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) return BITSORT_ERR_CUDA;
    if (cudaMemcpy(results, pl->d_results, pl->count * sizeof(bitsort_result_t), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
        return BITSORT_ERR_CUDA;
    bitsort_status_t first = BITSORT_OK;
    bool timeout = false;
    for (size_t i = 0; i < pl->count; ++i) {
        if (results[i].status != BITSORT_OK && first == BITSORT_OK) first = (bitsort_status_t)results[i].status;
        if (results[i].status == BITSORT_ERR_TIMEOUT) timeout = true;
    }
    if (timeout) {
        cudaDeviceSynchronize();
        cudaMemset(pl->scratch, 0, pl->scratch_bytes);
        cudaMemset(pl->params.ticket, 0, 16);
        cudaDeviceSynchronize();   // cleared before the next launch, on whatever stream
    }
    return first;
}

extern "C" const bitsort_result_t *bitsort_batch_plan_device_results(const bitsort_batch_plan_t *pl) {
    return pl ? pl->d_results : nullptr;
}

extern "C" bitsort_status_t bitsort_batch_plan_destroy(bitsort_batch_plan_t *pl) {
    if (!pl) return BITSORT_ERR_INVALID;
    cudaSetDevice(pl->ctx->device);
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    if (!pl->async_alloc) cudaDeviceSynchronize();
    if (pl->tables) cudaFree(pl->tables);
    if (pl->scratch) cudaFree(pl->scratch);
    delete pl;
    return BITSORT_OK;
}

// Release a plan built with stream-ordered allocations after the work
// already enqueued on `s` (the memory is reused only after it completes).
void bsx_plan_release_async(bitsort_batch_plan *pl, cudaStream_t s) {
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    if (pl->tables) cudaFreeAsync(pl->tables, s);
    if (pl->scratch) cudaFreeAsync(pl->scratch, s);
    delete pl;
}

const bitsort_result_t *bsx_plan_results_ptr(const bitsort_batch_plan *pl) { return pl->d_results; }

extern "C" bitsort_status_t bitsort_batched(bitsort_ctx_t *c, const bitsort_desc_t *descs, size_t count,
                                            bitsort_result_t *d_results, bitsort_stream_t stream) {
    bsx_range nvtx_range_("bitsort_batched");
    if (!c) c = bsx_default_ctx();
    if (!c) return BITSORT_ERR_CUDA;
    if (cudaSetDevice(c->device) != cudaSuccess) return BITSORT_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    bitsort_batch_plan *pl = nullptr;
    bitsort_status_t st = bsx_plan_build(c, descs, count, d_results, s, true, &pl, nullptr, 0);
    if (st != BITSORT_OK) return st;
    st = bsx_plan_launch_direct(pl, s);
    bsx_plan_release_async(pl, s);
    return st;
}

// --------------------------------------------------------------- batch policy
extern "C" bitsort_status_t bitsort_set_batch_config(bitsort_ctx_t *c, const bitsort_config_t *in) {
    if (!c) c = bsx_default_ctx();
    if (!c || !in) return BITSORT_ERR_INVALID;
    if (in->path != BITSORT_PATH_PARTITION && in->path != BITSORT_PATH_GLOBAL) return BITSORT_ERR_INVALID;
    bsx_config b = bitsort_ctx::batch_default();
    b.path = (bitsort_path_t)in->path;
    if (in->slice_values) b.S = std::max<uint32_t>(128, std::min<uint32_t>(in->slice_values, 1u << 20)) / 128 * 128;
    if (in->block_threads) b.threads = in->block_threads == 256 ? 256 : 512;
    if (in->words_per_lane) b.wpl = in->words_per_lane;
    b.stage = in->stage != 0;
    if (b.stage && b.wpl == 2) b.wpl = 1;
    if (!b.stage && b.wpl == 8) b.wpl = 4;
    if (b.wpl != 1 && b.wpl != 2 && b.wpl != 4 && b.wpl != 8) b.wpl = 1;
    std::lock_guard<std::mutex> lk(c->mu);
    c->batch = b;
    return BITSORT_OK;
}

extern "C" bitsort_status_t bitsort_get_batch_config(bitsort_ctx_t *c, bitsort_config_t *out) {
    if (!c) c = bsx_default_ctx();
    if (!c || !out) return BITSORT_ERR_INVALID;
    std::lock_guard<std::mutex> lk(c->mu);
    memset(out, 0, sizeof(*out));
    out->path = (int32_t)c->batch.path;
    out->slice_values = c->batch.S;
    out->block_threads = (uint32_t)c->batch.threads;
    out->words_per_lane = c->batch.wpl;
    out->stage = c->batch.stage ? 1 : 0;
    out->persistent = 1;
    out->ms = c->batch.ms;
    return BITSORT_OK;
}

extern "C" bitsort_status_t bitsort_batch_autotune(bitsort_ctx_t *c, const bitsort_desc_t *descs, size_t count,
                                                   bitsort_config_t *best_out) {
    bsx_range nvtx_range_("bitsort_batch_autotune");
    if (!c) c = bsx_default_ctx();
    if (!c) return BITSORT_ERR_CUDA;
    if (cudaSetDevice(c->device) != cudaSuccess) return BITSORT_ERR_CUDA;
    const bsx_config saved = c->batch;
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return BITSORT_ERR_CUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // outcomes of the default policy: a candidate counts only if every array
    // comes out with the same status and count (a policy that loses keys
    // must never be picked because it ran fast)
    std::vector<bitsort_result_t> want(count);
    {
        c->batch = bitsort_ctx::batch_default();
        bitsort_batch_plan *pl = nullptr;
        bitsort_status_t st = bsx_plan_build(c, descs, count, nullptr, nullptr, false, &pl, nullptr, 0);
        if (st == BITSORT_OK) {
            st = bsx_plan_launch_direct(pl, s);
            bitsort_status_t rs = bitsort_batch_plan_results(pl, s, want.data());
            bitsort_batch_plan_destroy(pl);
            if (st == BITSORT_OK && (rs == BITSORT_ERR_TIMEOUT || rs == BITSORT_ERR_CUDA)) st = rs;
        }
        if (st != BITSORT_OK) {
            c->batch = saved;
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            cudaStreamDestroy(s);
            return st;
        }
    }
    double best = 1e30;
    bsx_config best_cfg = saved;
    uint64_t rejected = 0;
    for (int path : {(int)BITSORT_PATH_PARTITION, (int)BITSORT_PATH_GLOBAL}) {
        for (uint32_t S : {1u << 17, 1u << 18, 1u << 19, 1u << 20}) {
            for (int T : {256, 512}) {
                for (uint32_t wpl : {1u, 2u}) {
                    bsx_config b = bitsort_ctx::batch_default();
                    b.path = (bitsort_path_t)path;
                    b.S = S;
                    b.threads = T;
                    b.wpl = wpl;
                    c->batch = b;
                    bitsort_batch_plan *pl = nullptr;
                    if (bsx_plan_build(c, descs, count, nullptr, nullptr, false, &pl, nullptr, 0) != BITSORT_OK) continue;
                    bool ok = bsx_plan_launch_direct(pl, s) == BITSORT_OK;   // warm-up
                    float ms = 0, sum = 0;
                    for (int r = 0; r < 3 && ok; ++r) {
                        cudaEventRecord(e0, s);
                        ok = bsx_plan_launch_direct(pl, s) == BITSORT_OK;
                        cudaEventRecord(e1, s);
                        if (cudaEventSynchronize(e1) != cudaSuccess) ok = false;
                        cudaEventElapsedTime(&ms, e0, e1);
                        sum += ms;
                    }
                    std::vector<bitsort_result_t> res(count);
                    bitsort_status_t st = bitsort_batch_plan_results(pl, s, res.data());
                    bitsort_batch_plan_destroy(pl);
                    if (!ok || st == BITSORT_ERR_TIMEOUT || st == BITSORT_ERR_CUDA) continue;
                    bool same = true;
                    for (size_t i = 0; i < count && same; ++i)
                        same = res[i].status == want[i].status && res[i].count == want[i].count;
                    if (!same) {
                        ++rejected;
                        continue;
                    }
                    const double mean = sum / 3.0;
                    if (mean < best) {
                        best = mean;
                        best_cfg = b;
                    }
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    if (rejected) {
        char msg[160];
        snprintf(msg, sizeof(msg), "batch autotune: %llu policies left out, their outcomes differ from the default's",
                 (unsigned long long)rejected);
        bsx_note_msg(msg);
    }
    if (best >= 1e30) {
        c->batch = saved;
        return BITSORT_ERR_CUDA;
    }
    best_cfg.ms = best;
    c->batch = best_cfg;
    if (best_out) {
        bitsort_get_batch_config(c, best_out);
        best_out->ms = best;
    }
    return BITSORT_OK;
}
