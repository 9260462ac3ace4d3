// internal.h -- host-side state shared by api.cu, batch.cu, server.cu, noalloc.cu, msort.cu and widths.cu.
#pragma once
#include <stdint.h>

#include <atomic>
#include <map>
#include <mutex>
#include <utility>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/bitsort.h"
#include "engine.h"

// One tuned or default configuration of the sort of one array.
struct bsx_config {
    bitsort_path_t path = BITSORT_PATH_PARTITION;
    uint32_t S = 1u << 18;   // values per shared-memory slice (multiple of 128)
    int threads = 512;       // block size of the engine kernel
    bool persistent = false; // all phases in one persistent launch (else one kernel per phase)
    uint32_t layout = 1;     // PARTITION: bsx::LAYOUT_EXACT (0) or bsx::LAYOUT_CAPACITY (1)
    uint32_t wpl = 2;        // bitmap words per lane in the scan (1, 2, 4)
    bool stage = false;      // stage set-bit positions per warp in shared memory
    uint32_t emit = 0;       // bsx::EMIT_WORD (0) or bsx::EMIT_RANK (1)
    bool summary = true;     // sparse slices keep a summary bitmap (word emission)
    bool stream_part = false; // phased PARTITION: stream tiles through bulk copies when keys are 16-byte aligned
    int part_threads = 0;     // phased PARTITION: block size of the HIST/PART phases (0 = the plan's rule)
    uint32_t part_tile_keys = 0; // phased PARTITION at 1024 threads: 16384 or 32768 keys a tile (0 = the plan's rule)
    double ms = 0;           // measured time when tuned (0 = not measured)
};

struct bitsort_ctx {
    int device = 0;
    int sms = 0;
    int force_path = 0;   // BITSORT_FORCE_PATH at creation: a bitsort_path_t for every single sort, 0 = none
    size_t l2_bytes = 0;
    uint32_t smem_optin = 0;
    uint64_t wait_limit_ns = 0;

    // fixed scratch: ticket/sync/result block and per-slice arrays (zero at rest)
    void *fixed = nullptr;
    size_t fixed_bytes = 0;
    uint32_t *ticket = nullptr;
    uint32_t *sync = nullptr;
    bitsort_result_t *result = nullptr;
    uint32_t *counts = nullptr;
    uint32_t *cursor = nullptr;
    uint64_t *offsets = nullptr;
    uint64_t *look = nullptr;

    // grown on demand
    uint32_t *part = nullptr;     // partition buffer for in-place sorts
    uint64_t part_cap = 0;
    uint32_t *bitmap = nullptr;   // global bitmap (zero at rest)
    uint64_t bitmap_words = 0;
    void *flush = nullptr;        // L2 flush buffer for tuning
    size_t flush_bytes = 0;
    bool stream_ordered = false;  // used from one stream only: buffers regrow in its order
    uint32_t *host_io = nullptr;  // bitsort_host(): device copies of the keys and the output (2 x cap)
    uint64_t host_io_cap = 0;

    // multiset path (msort.cu): look-back words tagged with a pass epoch
    // (never cleared between passes) and a small block cleared per call
    uint64_t *ms_look = nullptr;
    uint64_t ms_look_words = 0;
    uint32_t ms_epoch = 0;        // epoch of the last pass launched
    uint32_t *ms_misc = nullptr;

    // 64-bit keys (widths.cu): the narrowed 32-bit copy and a flag block
    uint32_t *wide = nullptr;
    uint64_t wide_cap = 0;
    void *wide_misc = nullptr;

    // optional per-phase timing of single sorts
    bool timing = false;
    cudaEvent_t tev[9] = {};
    int tkind[8] = {};
    int tcount = 0;

    std::mutex mu;
    std::map<std::pair<int, int>, bsx_config> table;  // (ceil log2 n, ceil log2 M) -> config
    // policy of batched launches: arrays with M <= batch.S are one fused
    // slice, the others take batch.path with slices of batch.S values
    bsx_config batch = batch_default();

    static bsx_config batch_default() {
        bsx_config b;
        b.path = BITSORT_PATH_PARTITION;
        b.S = 1u << 19;
        b.threads = 512;
        b.wpl = 1;
        b.stage = false;
        b.persistent = true;
        b.layout = 0;
        return b;
    }
    std::atomic<uint64_t> launches{0};
};

// NVTX range over a library call (host side: the call's enqueue), for
// profilers that filter or group by range; a no-op when no tool is attached.
struct bsx_range {
    explicit bsx_range(const char *name) { nvtxRangePushA(name); }
    ~bsx_range() { nvtxRangePop(); }
    bsx_range(const bsx_range &) = delete;
    bsx_range &operator=(const bsx_range &) = delete;
};

bitsort_status_t bsx_check(cudaError_t e);
void bsx_note_error(int e, const char *where);
void bsx_note_msg(const char *msg);   // the text bitsort_last_error() returns next
bitsort_ctx *bsx_default_ctx();
uint64_t bsx_div_magic(uint32_t S);
bsx_config bsx_default_config(int sms, uint64_t n, uint64_t M);
bsx_config bsx_lookup_config(bitsort_ctx *c, uint64_t n, uint64_t M);
bsx_config bsx_sanitize(bsx_config cfg, uint64_t n, uint64_t M);
uint32_t bsx_smem_for(const bsx_config &cfg, uint32_t nslices, uint32_t tile_keys, uint32_t stage_cap);
uint32_t bsx_stage_cap(const bsx_config &cfg, uint64_t n, uint64_t M);
void bsx_describe(const bsx_config &cfg, const uint32_t *keys, uint32_t *out, uint64_t n, uint64_t M,
                  bsx::ArrayDesc &a);
// plan of one array (api.cu, bsx_plan_single): host logic only
struct bsx_single_plan {
    bsx_config cfg;
    bsx::ArrayDesc a;                 // descriptor shape; pointers null
    int Tp = 0, Tb = 0;               // block size of the HIST/PART phases and of the BUCKET phase
    bool stream_part = false;         // the partition streams its tiles through bulk copies
    bool wide_part = false;           // the partition takes wide tiles (IT_PARTW, 1024 threads)
    uint32_t slice_smem = 0, part_smem = 0, hist_smem = 0;   // dynamic shared memory per phase (bytes)
    uint32_t engine_smem = 0;         // persistent plan: of the one launch
};
void bsx_plan_single(int sms, uint32_t smem_optin, const bsx_config &cfg0, uint64_t n, uint64_t M, bool in_place,
                     bool keys_aligned, bsx_single_plan &pl);
bool bsx_ranges_overlap(const void *a, const void *b, uint64_t bytes);
int bsx_grid_for(bitsort_ctx *c, int threads, uint32_t smem, uint32_t items);
bitsort_status_t bsx_validate(const uint32_t *keys, uint64_t n, uint32_t max_value, const uint32_t *out);
bitsort_status_t bsx_reset_scratch(bitsort_ctx *c);
bitsort_status_t bsx_ensure_part(bitsort_ctx *c, uint64_t n, cudaStream_t s);
void bsx_multiset_free(bitsort_ctx *c);
void bsx_widths_free(bitsort_ctx *c);

// batch plans (batch.cu)
bitsort_status_t bsx_plan_build(bitsort_ctx *c, const bitsort_desc_t *descs, size_t count,
                                bitsort_result_t *d_results_user, cudaStream_t stream, bool async_alloc,
                                bitsort_batch_plan **out, void *staging = nullptr, size_t staging_cap = 0);
bitsort_status_t bsx_plan_launch_direct(bitsort_batch_plan *pl, cudaStream_t s);
void bsx_plan_release_async(bitsort_batch_plan *pl, cudaStream_t s);
const bitsort_result_t *bsx_plan_results_ptr(const bitsort_batch_plan *pl);
