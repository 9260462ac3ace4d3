// noalloc.cu -- bitsort_noalloc(): the partition path of the sort with its
// scratch in a fixed device array, for callers that must not allocate device
// memory (see include/bitsort.h for who they are).
//
// The scratch (bucket counters, bucket offsets, look-back words, the ticket
// and synchronisation words) lives in g_noalloc_scratch, a file-scope
// __device__ array of kScratchBytes (49,408 bytes) that every GPU loading the
// library holds until the process exits.  The keys' partition buffer is the
// caller's output buffer, so keys and out must not overlap.  Host code cannot
// use the array's name as a device address: the address is fetched with
// cudaGetSymbolAddress once per device (the first call on a device, with that
// device current) and passed to the kernels.  Each call clears the array
// before its kernels run; calls that overlap on the GPU share it and race.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "engine.h"
#include "internal.h"

using namespace bsx;

namespace {

constexpr uint32_t kSlices = 2048;                    // buckets the array has room for
constexpr uint32_t kSliceValues = 1u << 20;           // values per bucket at most
constexpr uint64_t kMaxValues = (uint64_t)kSlices * kSliceValues;   // M <= 2^31
constexpr size_t kHead = 256;                         // ticket[4] | sync[8] | spare
constexpr size_t kScratchBytes = kHead + (size_t)kSlices * (4 + 4 + 8 + 8);
constexpr int kThreads = 512;
constexpr int kMaxDevices = 64;

struct DeviceState {
    bool ready = false;
    unsigned char *scratch = nullptr;   // device address of g_noalloc_scratch on this device
    int sms = 0;
    uint32_t smem_limit = 0;
};

std::mutex g_mu;
DeviceState g_dev[kMaxDevices];

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Once per device, with that device current: the scratch array's device
// address, the SM count and the shared-memory limit of the kernels.
static bitsort_status_t device_setup(int dev, DeviceState **out) {
    if (dev < 0 || dev >= kMaxDevices) return BITSORT_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState &d = g_dev[dev];
    if (!d.ready) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            bsx_note_error((int)(e != cudaSuccess ? e : cudaErrorInvalidSymbol), "cudaGetSymbolAddress");
            return BITSORT_ERR_CUDA;
        }
        int sms = 0, optin = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            return BITSORT_ERR_CUDA;
        const uint32_t limit = (uint32_t)optin - 1024;
        if (engine_set_smem_limit(kThreads, limit) != 0) return BITSORT_ERR_CUDA;
        d.scratch = (unsigned char *)p;
        d.sms = sms;
        d.smem_limit = limit;
        d.ready = true;
    }
    *out = &d;
    return BITSORT_OK;
}

extern "C" bitsort_status_t bitsort_noalloc(const uint32_t *keys, uint64_t n, uint32_t max_value, uint32_t *out,
                                            bitsort_result_t *d_result, bitsort_stream_t stream) {
    bsx_range nvtx_range_("bitsort_noalloc");
    if (!d_result) return BITSORT_ERR_INVALID;
    bitsort_status_t st = bsx_validate(keys, n, max_value, out);
    if (st != BITSORT_OK) return st;
    const uint64_t M = (uint64_t)max_value + 1;
    if (M > kMaxValues) return BITSORT_ERR_INVALID;             // beyond what the fixed scratch covers
    if (n > 0 && keys == out) return BITSORT_ERR_INVALID;       // out is the partition buffer
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BITSORT_ERR_CUDA;
    DeviceState *d = nullptr;
    if ((st = device_setup(dev, &d)) != BITSORT_OK) return st;
    if (n == 0) return bsx_check(cudaMemsetAsync(d_result, 0, sizeof(bitsort_result_t), s));

    // partition path, exact bucket ranges in `out`, one kernel per phase
    bsx_config cfg;
    cfg.path = BITSORT_PATH_PARTITION;
    cfg.layout = LAYOUT_EXACT;
    cfg.threads = kThreads;
    cfg.wpl = 1;
    cfg.stage = false;
    cfg.emit = EMIT_WORD;
    cfg.persistent = false;
    uint64_t S = (M + 2ull * d->sms - 1) / (2ull * d->sms);
    S = std::max<uint64_t>(S, std::max<uint64_t>(128, (M + kSlices - 1) / kSlices));
    S = std::min<uint64_t>(S, kSliceValues);
    S = std::min<uint64_t>(S, (M + 127) / 128 * 128);
    cfg.S = (uint32_t)((S + 127) / 128 * 128);

    EngineParams p;
    memset(&p, 0, sizeof(p));
    ArrayDesc &a = p.one;
    bsx_describe(cfg, keys, out, n, M, a);
    if (a.nslices > kSlices) return BITSORT_ERR_INVALID;
    unsigned char *sc = d->scratch;
    p.ticket = (uint32_t *)sc;
    a.sync = (uint32_t *)(sc + 16);
    a.counts = (uint32_t *)(sc + kHead);
    a.cursor = a.counts + kSlices;
    a.offsets = (uint64_t *)(a.cursor + kSlices);
    a.look = a.offsets + kSlices;
    a.part = out;
    a.result = d_result;
    p.wait_limit_ns = 4000ull * 1000ull * 1000ull;

    // the array keeps the last call's contents: start from zero
    cudaError_t e = cudaMemsetAsync(sc, 0, kScratchBytes, s);
    if (e != cudaSuccess) return bsx_check(e);

    struct Phase { int kind; uint32_t items; uint32_t smem; };
    const Phase phases[3] = {
        {IT_HIST, a.key_tiles, hist_smem_bytes(a.nslices)},
        {IT_PART, a.key_tiles, part_phase_smem_bytes(a.nslices, a.tile_keys)},
        {IT_BUCKET, a.nslices, slice_smem_bytes(cfg.S, kThreads, false)},
    };
    for (int i = 0; i < 3; ++i) {
        const Phase &ph = phases[i];
        if (ph.smem > d->smem_limit) return BITSORT_ERR_INVALID;
        int per_sm = 1;
        if (kernel_max_blocks_per_sm(ph.kind, kThreads, ph.smem, &per_sm) != 0 || per_sm < 1) per_sm = 1;
        uint64_t grid = (uint64_t)d->sms * (uint64_t)per_sm * (ph.kind == IT_PART ? 8u : 1u);
        if (grid > ph.items) grid = ph.items;
        if (grid < 1) grid = 1;
        EngineParams q = p;
        q.total_items = ph.items;
        int le = kernel_launch(ph.kind, q, kThreads, ph.smem, (int)grid, s, i > 0);
        if (le != 0) {
            bsx_note_error(le, "bitsort_noalloc launch");
            return BITSORT_ERR_CUDA;
        }
    }
    return BITSORT_OK;
}
