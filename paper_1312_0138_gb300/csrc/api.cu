// api.cu -- host side of the C ABI in include/bitsort.h: contexts, planning,
// launching, batching with CUDA graphs, autotuning.
//
// Planning an array (n keys, M = max_value + 1 possible values) means picking
//   FUSED      one BUCKET item reads the whole array into one shared-memory
//              bitmap (needs M <= the largest slice);
//   PARTITION  HIST + PART tiles move the keys to contiguous bucket ranges
//              (bucket = value range of S values, S a multiple of 32), then
//              one BUCKET item per bucket;
//   GLOBAL     GSCATTER tiles OR the keys into a global bitmap in L2, then
//              one GSCAN item per slice of S values;
// together with the slice size S and the block size.  The choice comes from
// the context's tuned table (bitsort_autotune / bitsort_tune_load) or, for a
// size class never tuned, from a fixed rule.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "engine.h"
#include "internal.h"

using namespace bsx;

namespace {

constexpr uint32_t kMaxSliceValues = 1u << 20;   // 128 KiB of bitmap per CTA
// largest CAPACITY partition buffer (bytes): 4 GiB, or twice the keys' own
// bytes for a larger array (a dense array of 2^31 keys over 2^32 values
// then skips the histogram pass for 16 GiB of scratch)
constexpr uint64_t kCapacityScratchMax = 4ull << 30;
inline uint64_t capacity_scratch_max(uint64_t n) { return n * 8 > kCapacityScratchMax ? n * 8 : kCapacityScratchMax; }

constexpr uint64_t kDefaultWaitNs = 4000ull * 1000ull * 1000ull;

inline uint32_t round_up_u32(uint32_t v, uint32_t m) { return (v + m - 1) / m * m; }
inline uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

inline int ilog2_ceil(uint64_t v) {
    int k = 0;
    while (k < 64 && (1ull << k) < v) ++k;
    return k;
}

}  // namespace

// ---------------------------------------------------------------- context
static thread_local char g_last_error[256] = "";

void bsx_note_error(int e, const char *where) {
    if (e == 0) return;
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%d)", where, cudaGetErrorString((cudaError_t)e), e);
    if (getenv("BITSORT_VERBOSE")) fprintf(stderr, "bitsort: %s\n", g_last_error);
}

void bsx_note_msg(const char *msg) {
    snprintf(g_last_error, sizeof(g_last_error), "%s", msg);
    if (getenv("BITSORT_VERBOSE")) fprintf(stderr, "bitsort: %s\n", g_last_error);
}

extern "C" const char *bitsort_last_error(void) { return g_last_error; }

bitsort_status_t bsx_check(cudaError_t e) {
    if (e != cudaSuccess) bsx_note_error((int)e, "CUDA runtime");
    if (e == cudaSuccess) return BITSORT_OK;
    if (e == cudaErrorMemoryAllocation) return BITSORT_ERR_NOMEM;
    return BITSORT_ERR_CUDA;
}

static bitsort_status_t ctx_alloc_fixed(bitsort_ctx *c) {
    // small block: ticket[4] | sync[8] | result(16 B), then per-slice arrays
    size_t small = 256;
    size_t per = (size_t)kMaxSlices;
    size_t bytes = small + per * (4 + 4 + 8 + 8);
    cudaError_t e = cudaMalloc(&c->fixed, bytes);
    if (e != cudaSuccess) return bsx_check(e);
    // cudaMemset returns before the memory is written (it runs on the legacy
    // default stream, which a caller's non-blocking stream does not wait
    // for): the device is synchronised before any sort can use the block
    e = cudaMemset(c->fixed, 0, bytes);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return bsx_check(e);
    char *p = (char *)c->fixed;
    c->ticket = (uint32_t *)p;
    c->sync = (uint32_t *)(p + 16);
    c->result = (bitsort_result_t *)(p + 64);
    c->counts = (uint32_t *)(p + small);
    c->cursor = c->counts + per;
    c->offsets = (uint64_t *)(c->cursor + per);
    c->look = c->offsets + per;
    c->fixed_bytes = bytes;
    return BITSORT_OK;
}

// "fused", "partition" or "global" (BITSORT_FORCE_PATH) -> a path; else 0
static int parse_path(const char *s) {
    if (!s) return 0;
    if (!strcmp(s, "fused")) return BITSORT_PATH_FUSED;
    if (!strcmp(s, "partition")) return BITSORT_PATH_PARTITION;
    if (!strcmp(s, "global")) return BITSORT_PATH_GLOBAL;
    return 0;
}

extern "C" bitsort_status_t bitsort_ctx_create(int device, bitsort_ctx_t **out) {
    if (!out) return BITSORT_ERR_INVALID;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return BITSORT_ERR_INVALID;
    if (cudaSetDevice(device) != cudaSuccess) return BITSORT_ERR_CUDA;
    bitsort_ctx *c = new (std::nothrow) bitsort_ctx();
    if (!c) return BITSORT_ERR_NOMEM;
    c->device = device;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete c;
        return BITSORT_ERR_CUDA;
    }
    c->sms = prop.multiProcessorCount;
    c->l2_bytes = (size_t)prop.l2CacheSize;
    // dynamic shared memory available next to the kernel's static block
    c->smem_optin = (uint32_t)prop.sharedMemPerBlockOptin - 1024;
    c->wait_limit_ns = kDefaultWaitNs;
    if (engine_set_smem_limit(256, c->smem_optin) != 0 || engine_set_smem_limit(512, c->smem_optin) != 0 ||
        engine_set_smem_limit(1024, c->smem_optin) != 0) {
        delete c;
        return BITSORT_ERR_CUDA;
    }
    bitsort_status_t st = ctx_alloc_fixed(c);
    if (st != BITSORT_OK) {
        if (c->fixed) cudaFree(c->fixed);
        delete c;
        return st;
    }
    // environment: a tuned table saved by bitsort_tune_save, and a path
    // forced for every single sort (debugging, comparisons)
    const char *cache = getenv("BITSORT_TUNE_CACHE");
    if (cache && cache[0] && bitsort_tune_load(c, cache) != BITSORT_OK) {
        snprintf(g_last_error, sizeof(g_last_error), "BITSORT_TUNE_CACHE: %s not loaded", cache);
        if (getenv("BITSORT_VERBOSE")) fprintf(stderr, "bitsort: %s\n", g_last_error);
    }
    c->force_path = parse_path(getenv("BITSORT_FORCE_PATH"));
    *out = c;
    return BITSORT_OK;
}

extern "C" bitsort_status_t bitsort_ctx_destroy(bitsort_ctx_t *c) {
    if (!c) return BITSORT_ERR_INVALID;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    if (c->fixed) cudaFree(c->fixed);
    if (c->part) cudaFree(c->part);
    if (c->bitmap) cudaFree(c->bitmap);
    if (c->flush) cudaFree(c->flush);
    if (c->host_io) cudaFree(c->host_io);
    bsx_multiset_free(c);
    bsx_widths_free(c);
    for (int i = 0; i < 9; ++i)
        if (c->tev[i]) cudaEventDestroy(c->tev[i]);
    delete c;
    return BITSORT_OK;
}

extern "C" const char *bitsort_status_string(bitsort_status_t s) {
    switch (s) {
        case BITSORT_OK: return "ok";
        case BITSORT_ERR_INVALID: return "invalid argument";
        case BITSORT_ERR_KEY_RANGE: return "key above max_value";
        case BITSORT_ERR_DUPLICATE: return "duplicate keys";
        case BITSORT_ERR_NOMEM: return "out of memory";
        case BITSORT_ERR_TIMEOUT: return "device wait timed out";
        case BITSORT_ERR_CUDA: return "CUDA error";
        case BITSORT_ERR_BUDGET: return "request exceeds the memory budget";
    }
    return "unknown status";
}

static std::mutex g_default_mu;
static std::map<int, bitsort_ctx *> g_default;

bitsort_ctx *bsx_default_ctx() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_default_mu);
    auto it = g_default.find(dev);
    if (it != g_default.end()) return it->second;
    bitsort_ctx *c = nullptr;
    if (bitsort_ctx_create(dev, &c) != BITSORT_OK) return nullptr;
    g_default[dev] = c;
    return c;
}

// ------------------------------------------------------------- planning
uint64_t bsx_div_magic(uint32_t S) {
    // ceil(2^64 / S); exact floor(x / S) = mulhi(x, magic) for all x < 2^32
    // when S < 2^32 (the error x * (magic - 2^64/S) / 2^64 < 1/S).
    return UINT64_MAX / S + 1;
}

bsx_config bsx_default_config(int sms, uint64_t n, uint64_t M) {
    bsx_config cfg;
    cfg.threads = 256;
    cfg.wpl = 2;
    cfg.stage = false;
    if (M <= (1ull << 17) || (M <= kMaxSliceValues && n <= (1ull << 16))) {
        cfg.path = BITSORT_PATH_FUSED;
        cfg.threads = 512;
        cfg.S = round_up_u32((uint32_t)M, 128);
        return cfg;
    }
    if (M <= (1ull << 22) && n <= (1ull << 20)) {
        // a bitmap of at most 512 KiB stays in L2: OR the keys straight into
        // it and scan it in 16 Ki-value slices (measured 22.7 us against
        // 26.1 us for the partition path at n = 10^5, M = 2^20, where every
        // kernel is latency-bound)
        cfg.path = BITSORT_PATH_GLOBAL;
        cfg.threads = 512;
        cfg.wpl = 1;
        cfg.S = 1u << 14;
        return bsx_sanitize(cfg, n, M);
    }
    cfg.path = BITSORT_PATH_PARTITION;
    cfg.layout = LAYOUT_CAPACITY;
    // two slices per SM, word emission, one lane per word, 512 threads: the
    // best measured rule on GB300 for sparse and medium densities.  From
    // about one key per ten values the words hold several set bits each and
    // the lanes' own stores scatter: staging them per warp in shared memory
    // and writing them out in 16-byte stores measured 1.09x faster at
    // density 1/8, 1.9x at 1/4 and 2.6x at 1/2 (slower at 1/16)
    cfg.threads = 512;
    cfg.wpl = 1;
    cfg.emit = EMIT_WORD;
    cfg.stage = n * 10 >= M;
    uint64_t target = 2ull * (uint64_t)sms;
    uint64_t S = ceil_div(M, target);
    uint64_t lo = std::max<uint64_t>(4096, ceil_div(M, kMaxSlices));
    S = std::max(S, lo);
    S = std::min<uint64_t>(S, kMaxSliceValues);
    cfg.S = round_up_u32((uint32_t)S, 128);
    return bsx_sanitize(cfg, n, M);
}

bsx_config bsx_lookup_config(bitsort_ctx *c, uint64_t n, uint64_t M) {
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->table.find(std::make_pair(ilog2_ceil(n), ilog2_ceil(M)));
    bsx_config cfg = it != c->table.end() ? it->second : bsx_default_config(c->sms, n, M);
    if (c->force_path) cfg.path = (bitsort_path_t)c->force_path;   // the size rules still apply (bsx_sanitize)
    return cfg;
}

// Make a configuration valid for (n, M): the slice count within bounds, the
// slice a multiple of 128 values, FUSED only where one slice covers M.
bsx_config bsx_sanitize(bsx_config cfg, uint64_t n, uint64_t M) {
    if (cfg.threads != 256 && cfg.threads != 512 && cfg.threads != 1024) cfg.threads = 512;
    if (cfg.threads == 1024 && cfg.persistent) cfg.threads = 512;   // the persistent engine has 256 / 512
    if (cfg.part_threads != 0 && cfg.part_threads != 256 && cfg.part_threads != 512 && cfg.part_threads != 1024)
        cfg.part_threads = 0;
    if (cfg.part_tile_keys != 8192u && cfg.part_tile_keys != 16384u && cfg.part_tile_keys != 32768u)
        cfg.part_tile_keys = 0;
    if (cfg.wpl != 1 && cfg.wpl != 2 && cfg.wpl != 4 && cfg.wpl != 8) cfg.wpl = 2;
    if (cfg.stage && cfg.wpl == 2) cfg.wpl = 1;    // staged emission: 1, 4 or 8 words per lane
    if (!cfg.stage && cfg.wpl == 8) cfg.wpl = 4;   // direct emission: 1, 2 or 4
    if (cfg.layout != LAYOUT_EXACT && cfg.layout != LAYOUT_CAPACITY) cfg.layout = LAYOUT_EXACT;
    if (cfg.path == BITSORT_PATH_FUSED && M > kMaxSliceValues) cfg.path = BITSORT_PATH_PARTITION;
    if (cfg.path == BITSORT_PATH_FUSED) {
        cfg.S = round_up_u32((uint32_t)M, 128);
        return cfg;
    }
    if (cfg.path != BITSORT_PATH_PARTITION && cfg.path != BITSORT_PATH_GLOBAL) cfg.path = BITSORT_PATH_PARTITION;
    uint64_t S = cfg.S ? cfg.S : (1u << 18);
    S = std::max<uint64_t>(S, ceil_div(M, kMaxSlices));
    S = std::min<uint64_t>(S, kMaxSliceValues);
    S = std::min<uint64_t>(S, (M + 127) / 128 * 128);   // a slice never needs more than M values
    S = std::max<uint64_t>(S, 128);
    cfg.S = round_up_u32((uint32_t)S, 128);
    if (cfg.path == BITSORT_PATH_PARTITION && cfg.layout == LAYOUT_CAPACITY) {
        const uint64_t nb = ceil_div(M, cfg.S);
        const uint64_t cap = std::min<uint64_t>(cfg.S, n);
        if (nb * cap * 4 > capacity_scratch_max(n)) cfg.layout = LAYOUT_EXACT;
    }
    if (cfg.path == BITSORT_PATH_GLOBAL) cfg.emit = EMIT_WORD;   // a global slice has no keys to rank
    if (cfg.emit != EMIT_WORD && cfg.emit != EMIT_RANK) cfg.emit = EMIT_WORD;
    return cfg;
}

// Outputs a slice may stage under EMIT_RANK: 5/4 of the expected count plus
// a margin (every key lands in one slice: expected = n S / M), at most n.
uint32_t bsx_stage_cap(const bsx_config &cfg, uint64_t n, uint64_t M) {
    if (cfg.emit != EMIT_RANK) return 0;
    if (cfg.path == BITSORT_PATH_FUSED) return (uint32_t)((n + 3) & ~3ull);
    const double expected = (double)n * (double)cfg.S / (double)M;
    uint64_t cap = (uint64_t)(expected * 1.25) + 512;
    cap = std::min<uint64_t>(cap, n);
    return (uint32_t)((cap + 3) & ~3ull);
}

uint32_t bsx_smem_for(const bsx_config &cfg, uint32_t nslices, uint32_t tile_keys, uint32_t stage_cap) {
    uint32_t s = cfg.emit == EMIT_RANK ? rank_smem_bytes(cfg.S, stage_cap)
                                       : slice_smem_bytes(cfg.S, cfg.threads, cfg.stage);
    if (cfg.path == BITSORT_PATH_PARTITION) {
        s = std::max(s, part_smem_bytes(nslices, tile_keys));
        s = std::max(s, hist_smem_bytes(nslices));
    }
    return s;
}

// Fill the descriptor of one array and append its item segments.
void bsx_describe(const bsx_config &cfg, const uint32_t *keys, uint32_t *out, uint64_t n, uint64_t M,
                  ArrayDesc &a) {
    memset(&a, 0, sizeof(a));
    a.keys = keys;
    a.out = out;
    a.n = n;
    a.M = M;
    a.path = (uint32_t)cfg.path;
    a.S = cfg.S;
    a.div_magic = bsx_div_magic(cfg.S);
    a.nslices = (uint32_t)ceil_div(M, cfg.S);
    a.tile_keys = (uint32_t)(kKeysPerThread * cfg.threads);
    a.key_tiles = (uint32_t)ceil_div(n, a.tile_keys);
    a.wpl = cfg.wpl;
    a.stage = cfg.stage ? 1 : 0;
    a.phased = cfg.persistent ? 0 : 1;
    a.layout = cfg.path == BITSORT_PATH_PARTITION ? cfg.layout : LAYOUT_EXACT;
    a.cap = a.layout == LAYOUT_CAPACITY ? std::min<uint64_t>(cfg.S, n) : 0;
    a.emit = cfg.emit;
    a.stage_cap = bsx_stage_cap(cfg, n, M);
    a.summary = (cfg.summary && cfg.path != BITSORT_PATH_GLOBAL) ? 1u : 0u;
    a.s_shift = (cfg.S & (cfg.S - 1)) == 0 ? (uint32_t)__builtin_ctz(cfg.S) : 0u;
    if (cfg.path == BITSORT_PATH_FUSED) {
        a.nslices = 1;
        a.key_tiles = 0;
    }
}

bool bsx_ranges_overlap(const void *a, const void *b, uint64_t bytes) {
    uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + bytes && y < x + bytes;
}

// Grown on demand.  A context may be used from several streams, so growth
// normally waits for the whole device before freeing the old buffer; a
// context bound to one stream (c->stream_ordered, the server's) frees and
// allocates in that stream's order instead, without stalling other streams.
static cudaError_t regrow(bitsort_ctx *c, void **buf, size_t bytes, cudaStream_t s) {
    if (c->stream_ordered) {
        if (*buf) cudaFreeAsync(*buf, s);
        *buf = nullptr;
        return cudaMallocAsync(buf, bytes, s);
    }
    if (*buf) {
        cudaDeviceSynchronize();
        cudaFree(*buf);
        *buf = nullptr;
    }
    return cudaMalloc(buf, bytes);
}

bitsort_status_t bsx_ensure_part(bitsort_ctx *c, uint64_t n, cudaStream_t s) {
    if (c->part_cap >= n) return BITSORT_OK;
    c->part_cap = 0;
    cudaError_t e = regrow(c, reinterpret_cast<void **>(&c->part), n * sizeof(uint32_t), s);
    if (e != cudaSuccess) {
        c->part = nullptr;
        return bsx_check(e);
    }
    c->part_cap = n;
    return BITSORT_OK;
}

static bitsort_status_t ensure_bitmap(bitsort_ctx *c, uint64_t M, cudaStream_t s) {
    const uint64_t words = (ceil_div(M, 32) + 3) / 4 * 4;
    if (c->bitmap_words >= words) return BITSORT_OK;
    c->bitmap_words = 0;
    cudaError_t e = regrow(c, reinterpret_cast<void **>(&c->bitmap), words * 4, s);
    if (e != cudaSuccess) {
        c->bitmap = nullptr;
        return bsx_check(e);
    }
    // zeroed in the order of the stream whose kernels use it next
    e = cudaMemsetAsync(c->bitmap, 0, words * 4, s);
    if (e != cudaSuccess) return bsx_check(e);
    c->bitmap_words = words;
    return BITSORT_OK;
}

int bsx_grid_for(bitsort_ctx *c, int threads, uint32_t smem, uint32_t items) {
    int per_sm = 1;
    if (engine_max_blocks_per_sm(threads, smem, &per_sm) != 0 || per_sm < 1) per_sm = 1;
    uint64_t g = (uint64_t)per_sm * (uint64_t)c->sms;
    if (g > items) g = items;
    if (g < 1) g = 1;
    return (int)g;
}

// Segments of a single array, ticket order: HIST, PART, BUCKET or
// GSCATTER, GSCAN or one BUCKET (fused).
uint32_t bsx_single_segments(const ArrayDesc &a, Segment *seg, uint32_t *nseg) {
    uint32_t t = 0, k = 0;
    auto add = [&](uint32_t type, uint32_t count) {
        if (count == 0) return;
        seg[k].start = t;
        seg[k].array = 0;
        seg[k].type = type;
        seg[k].first = 0;
        ++k;
        t += count;
    };
    if (a.path == BITSORT_PATH_FUSED) {
        add(IT_BUCKET, 1);
    } else if (a.path == BITSORT_PATH_PARTITION) {
        if (a.layout == LAYOUT_EXACT) add(IT_HIST, a.key_tiles);
        add(IT_PART, a.key_tiles);
        add(IT_BUCKET, a.nslices);
    } else {
        add(IT_GSCATTER, a.key_tiles);
        add(IT_GSCAN, a.nslices);
    }
    *nseg = k;
    return t;
}

// Shrink a configuration until its shared memory fits one CTA: rank
// emission falls back to word emission, staging to direct stores.
static bsx_config fit_smem(uint32_t smem_optin, bsx_config cfg, uint64_t n, uint64_t M) {
    for (int tries = 0; tries < 3; ++tries) {
        ArrayDesc probe;
        bsx_describe(cfg, nullptr, nullptr, n, M, probe);
        if (bsx_smem_for(cfg, probe.nslices, probe.tile_keys, probe.stage_cap) <= smem_optin) break;
        if (cfg.emit == EMIT_RANK) cfg.emit = EMIT_WORD;
        else if (cfg.stage) cfg.stage = false;
        else break;
    }
    return cfg;
}

// The plan of one array on a device with `sms` SMs and `smem_optin` bytes of
// shared memory per block (host logic only): the configuration after the
// size rules and the shared-memory fit, the array's descriptor (pointers
// left null), the block size of each phase and each phase's shared memory.
// In place, a capacity bucket that overflowed (repeated keys) would read the
// whole input while other slices write their outputs over it: exact bucket
// ranges never overflow, so an in-place sort takes the exact layout.
// A phased 512-thread plan runs two phases at 1024 threads (one CTA per SM)
// where that measured faster on GB300: the partition with a wide fan-out
// (its tile doubles to 16 Ki keys, so the per-bucket work of a tile is
// spread over twice the keys: 16.0 -> 12.6 ms at 4096 buckets, n = 2^31),
// and the bucket phase when every SM works through many slices without
// staging (255.9 -> 212.0 us for 4096 sparse slices, n = 2^24); with
// staging, or one or two slices per SM, 512 threads stay faster.
void bsx_plan_single(int sms, uint32_t smem_optin, const bsx_config &cfg0, uint64_t n, uint64_t M, bool in_place,
                     bool keys_aligned, bsx_single_plan &pl) {
    bsx_config cfg = fit_smem(smem_optin, bsx_sanitize(cfg0, n, M), n, M);
    if (in_place && cfg.path == BITSORT_PATH_PARTITION && cfg.layout == LAYOUT_CAPACITY) cfg.layout = LAYOUT_EXACT;
    ArrayDesc &a = pl.a;
    bsx_describe(cfg, nullptr, nullptr, n, M, a);
    const int T = cfg.threads;
    const bool partitioned = a.path == BITSORT_PATH_PARTITION;
    pl.stream_part = !cfg.persistent && partitioned && keys_aligned && cfg.stream_part;
    int Tp = T, Tb = T;
    if (!cfg.persistent && partitioned && cfg.part_threads) {
        const uint32_t tk = (uint32_t)(kKeysPerThread * cfg.part_threads);
        const uint32_t ps = pl.stream_part ? part_stream_smem_bytes(a.nslices, tk) : part_phase_smem_bytes(a.nslices, tk);
        if (ps <= smem_optin) Tp = cfg.part_threads;
    } else if (!cfg.persistent && T == 512 && partitioned) {
        const uint32_t wide = (uint32_t)(kKeysPerThread * 1024);
        const uint32_t part_smem =
            pl.stream_part ? part_stream_smem_bytes(a.nslices, wide) : part_phase_smem_bytes(a.nslices, wide);
        if (a.nslices >= 1024 && part_smem <= smem_optin) Tp = 1024;
    }
    // the bucket phase's block size, whatever the partition's
    if (!cfg.persistent && T == 512 && partitioned && !cfg.stage && cfg.emit == EMIT_WORD &&
        a.nslices >= 4u * (uint32_t)sms && slice_smem_bytes(cfg.S, 1024, false) <= smem_optin)
        Tb = 1024;
    if (Tp != T) {
        a.tile_keys = (uint32_t)(kKeysPerThread * Tp);
        a.key_tiles = (uint32_t)ceil_div(n, (uint64_t)a.tile_keys);
    }
    // wide partition tiles (32 keys a thread) at 512 or 1024 threads: where
    // the shared memory holds one and the array gives every SM at least
    // three of them at 1024 threads (one CTA per SM), four at 512 (two CTAs
    // per SM); fewer tiles leave SMs idle at the end.  Or where the
    // configuration asks for 32 * Tp keys a tile (16 * Tp keeps them narrow).
    // Measured on GB300: c2a's partition (1024 threads, 4,096 buckets)
    // 11.82 -> 8.59 ms; c2b's (1024 threads, 3.4 tiles per SM) 98.6 ->
    // 84.6 us; c1's (512 threads, 304 buckets) 64.1 -> 62.1 us.
    pl.wide_part = false;
    if (!cfg.persistent && partitioned && !pl.stream_part && (Tp == 1024 || Tp == 512)) {
        const uint32_t wk = (uint32_t)(kWideKeysPerThread * Tp);
        const bool fits = part_phase_smem_bytes(a.nslices, wk) <= smem_optin;
        const bool many = ceil_div(n, (uint64_t)wk) >= (Tp == 1024 ? 3ull : 4ull) * (uint64_t)sms;
        if (fits && (cfg.part_tile_keys == wk || (cfg.part_tile_keys == 0 && many))) {
            pl.wide_part = true;
            a.tile_keys = wk;
            a.key_tiles = (uint32_t)ceil_div(n, (uint64_t)wk);
        }
    }
    pl.cfg = cfg;
    pl.Tp = Tp;
    pl.Tb = Tb;
    pl.slice_smem = cfg.emit == EMIT_RANK ? rank_smem_bytes(cfg.S, a.stage_cap) : slice_smem_bytes(cfg.S, Tb, cfg.stage);
    pl.part_smem = !partitioned ? 0u
                   : pl.stream_part ? part_stream_smem_bytes(a.nslices, a.tile_keys)
                                    : part_phase_smem_bytes(a.nslices, a.tile_keys);
    pl.hist_smem = partitioned && a.layout == LAYOUT_EXACT ? hist_smem_bytes(a.nslices) : 0u;
    pl.engine_smem = cfg.persistent ? bsx_smem_for(cfg, a.nslices, a.tile_keys, a.stage_cap) : 0u;
}

static bitsort_status_t launch_single(bitsort_ctx *c, const bsx_config &cfg0, const uint32_t *keys, uint64_t n,
                                      uint64_t M, uint32_t *out, bitsort_result_t *d_result, cudaStream_t stream,
                                      uint32_t stall, uint32_t bias = 0) {
    const bool alias = keys == out;
    const bool aligned = ((uintptr_t)keys & 15u) == 0;
    bsx_single_plan pl;
    bsx_plan_single(c->sms, c->smem_optin, cfg0, n, M, alias, aligned, pl);
    if (pl.cfg.path == BITSORT_PATH_PARTITION && pl.a.layout == LAYOUT_CAPACITY) {
        const uint64_t entries = (uint64_t)pl.a.nslices * pl.a.cap;
        bitsort_status_t st = bsx_ensure_part(c, entries, stream);
        if (st == BITSORT_ERR_NOMEM && entries * 4 > kCapacityScratchMax) {
            // no room for a large capacity buffer: the exact layout needs
            // none outside the output (the failed allocation is not sticky)
            cudaGetLastError();
            bsx_config exact = pl.cfg;
            exact.layout = LAYOUT_EXACT;
            bsx_plan_single(c->sms, c->smem_optin, exact, n, M, alias, aligned, pl);
            st = BITSORT_OK;
        }
        if (st != BITSORT_OK) return st;
    }
    const bsx_config &cfg = pl.cfg;
    EngineParams p;
    memset(&p, 0, sizeof(p));
    p.one = pl.a;
    ArrayDesc &a = p.one;
    a.keys = keys;
    a.out = out;
    a.stall = stall;
    a.bias = bias;
    if (cfg.path == BITSORT_PATH_PARTITION && a.layout == LAYOUT_CAPACITY) {
        a.part = c->part;
    } else if (cfg.path == BITSORT_PATH_PARTITION) {
        if (alias) {
            bitsort_status_t st = bsx_ensure_part(c, n, stream);
            if (st != BITSORT_OK) return st;
            a.part = c->part;
        } else {
            a.part = out;  // partition in the output buffer, sort in place per bucket
        }
    }
    if (cfg.path == BITSORT_PATH_GLOBAL) {
        bitsort_status_t st = ensure_bitmap(c, M, stream);
        if (st != BITSORT_OK) return st;
        a.bitmap = c->bitmap;
    }
    a.counts = c->counts;
    a.cursor = c->cursor;
    a.offsets = c->offsets;
    a.look = c->look;
    a.sync = c->sync;
    a.result = d_result ? d_result : c->result;
    p.arrays = nullptr;
    p.segments = nullptr;
    p.total_items = bsx_single_segments(a, p.seg, &p.nseg);
    p.ticket = c->ticket;
    p.wait_limit_ns = c->wait_limit_ns;
    const int T = cfg.threads;
    if (cfg.persistent) {
        // every phase in one persistent launch (items in ticket order)
        const uint32_t smem = pl.engine_smem;
        if (smem > c->smem_optin) return BITSORT_ERR_INVALID;
        int grid = bsx_grid_for(c, T, smem, p.total_items);
        if (c->timing) {
            cudaEventRecord(c->tev[0], stream);
            c->tkind[0] = -1;
        }
        int e = engine_launch(p, T, smem, grid, stream);
        if (e != 0) {
            bsx_note_error(e, "engine launch");
            return BITSORT_ERR_CUDA;
        }
        if (c->timing) {
            cudaEventRecord(c->tev[1], stream);
            c->tcount = 1;
        }
        c->launches.fetch_add(1);
        return BITSORT_OK;
    }
    // one kernel per phase, each at the occupancy its shared memory allows
    // and with the plan's block size; later phases use programmatic
    // dependent launch to hide the launch gap
    const int Tp = pl.Tp, Tb = pl.Tb;
    int launched = 0;
    auto phase = [&](int kind, uint32_t items, uint32_t smem) -> bool {
        const int Tk = (kind == IT_HIST || kind == IT_PART || kind == IT_PARTS || kind == IT_PARTW) ? Tp
                       : kind == IT_BUCKET ? Tb : T;
        if (items == 0) return true;
        if (smem > c->smem_optin) {
            bsx_note_error((int)cudaErrorInvalidValue, "shared memory above the per-block limit");
            return false;
        }
        EngineParams q = p;
        q.total_items = items;
        if (c->timing && launched < 8) {
            if (launched == 0) cudaEventRecord(c->tev[0], stream);
            c->tkind[launched] = kind;
        }
        int per_sm = 1;
        if (kernel_max_blocks_per_sm(kind, Tk, smem, &per_sm) != 0 || per_sm < 1) per_sm = 1;
        // slice phases and the streaming HIST / GSCATTER / PARTS
        // phases: one wave of resident CTAs; PART: a few tiles per CTA
        const bool one_wave = kind != IT_PART && kind != IT_PARTW;
        uint64_t grid = (uint64_t)c->sms * (uint64_t)per_sm * (one_wave ? 1u : 8u);
        if (grid > items) grid = items;
        int e = kernel_launch(kind, q, Tk, smem, (int)grid, stream, launched > 0);
        if (e != 0) {
            bsx_note_error(e, "phase kernel launch");
            return false;
        }
        ++launched;
        if (c->timing && launched <= 8) {
            cudaEventRecord(c->tev[launched], stream);
            c->tcount = launched;
        }
        return true;
    };
    const uint32_t sl = pl.slice_smem;
    bool ok = true;
    if (a.path == BITSORT_PATH_FUSED) {
        ok = phase(IT_BUCKET, 1, sl);
    } else if (a.path == BITSORT_PATH_PARTITION) {
        // tiles of 16-byte aligned keys may stream through bulk copies
        const int pk = pl.stream_part ? (int)IT_PARTS : pl.wide_part ? (int)IT_PARTW : (int)IT_PART;
        if (a.layout == LAYOUT_EXACT) ok = phase(IT_HIST, a.key_tiles, pl.hist_smem);
        ok = ok && phase(pk, a.key_tiles, pl.part_smem) && phase(IT_BUCKET, a.nslices, sl);
    } else {
        ok = phase(IT_GSCATTER, a.key_tiles, 0) && phase(IT_GSCAN, a.nslices, sl);
    }
    c->launches.fetch_add((uint64_t)launched);
    return ok ? BITSORT_OK : BITSORT_ERR_CUDA;
}

static bitsort_status_t write_trivial_result(bitsort_ctx *c, bitsort_result_t *d_result, cudaStream_t s) {
    bitsort_result_t *r = d_result ? d_result : c->result;
    return bsx_check(cudaMemsetAsync(r, 0, sizeof(bitsort_result_t), s));
}

bitsort_status_t bsx_validate(const uint32_t *keys, uint64_t n, uint32_t max_value, const uint32_t *out) {
    if (n == 0) return BITSORT_OK;
    if (!keys || !out) return BITSORT_ERR_INVALID;
    uint64_t M = (uint64_t)max_value + 1;
    if (n > M) return BITSORT_ERR_INVALID;  // pigeonhole: keys cannot be distinct
    if (((uintptr_t)keys & 3u) || ((uintptr_t)out & 3u)) return BITSORT_ERR_INVALID;
    if (keys != out && bsx_ranges_overlap(keys, out, n * sizeof(uint32_t))) return BITSORT_ERR_INVALID;
    return BITSORT_OK;
}

extern "C" bitsort_status_t bitsort_ex(bitsort_ctx_t *c, const uint32_t *keys, uint64_t n, uint32_t max_value,
                                       uint32_t *out, bitsort_result_t *d_result, bitsort_stream_t stream) {
    bsx_range nvtx_range_("bitsort_ex");
    if (!c) c = bsx_default_ctx();
    if (!c) return BITSORT_ERR_CUDA;
    bitsort_status_t st = bsx_validate(keys, n, max_value, out);
    if (st != BITSORT_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaSetDevice(c->device) != cudaSuccess) return BITSORT_ERR_CUDA;
    if (n == 0) return write_trivial_result(c, d_result, s);
    uint64_t M = (uint64_t)max_value + 1;
    bsx_config cfg = bsx_lookup_config(c, n, M);
    return launch_single(c, cfg, keys, n, M, out, d_result, s, 0);
}

extern "C" bitsort_status_t bitsort_i32(bitsort_ctx_t *c, const int32_t *keys, uint64_t n, int32_t min_value,
                                        int32_t max_value, int32_t *out, bitsort_result_t *d_result,
                                        bitsort_stream_t stream) {
    bsx_range nvtx_range_("bitsort_i32");
    if (!c) c = bsx_default_ctx();
    if (!c) return BITSORT_ERR_CUDA;
    if (min_value > max_value) return BITSORT_ERR_INVALID;
    // x -> x - min_value (mod 2^32) maps [min_value, max_value] onto
    // [0, max_value - min_value] in the same order: the unsigned sort of the
    // shifted keys, with the shift undone on output
    const uint32_t bias = (uint32_t)min_value;
    const uint32_t span_max = (uint32_t)max_value - bias;
    const uint32_t *k = reinterpret_cast<const uint32_t *>(keys);
    uint32_t *o = reinterpret_cast<uint32_t *>(out);
    bitsort_status_t st = bsx_validate(k, n, span_max, o);
    if (st != BITSORT_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaSetDevice(c->device) != cudaSuccess) return BITSORT_ERR_CUDA;
    if (n == 0) return write_trivial_result(c, d_result, s);
    const uint64_t M = (uint64_t)span_max + 1;
    bsx_config cfg = bsx_lookup_config(c, n, M);
    return launch_single(c, cfg, k, n, M, o, d_result, s, 0, bias);
}

extern "C" bitsort_status_t bitsort_span(bitsort_ctx_t *c, const uint32_t *keys, uint64_t n, uint32_t min_value,
                                         uint32_t max_value, uint32_t *out, bitsort_result_t *d_result,
                                         bitsort_stream_t stream) {
    bsx_range nvtx_range_("bitsort_span");
    if (!c) c = bsx_default_ctx();
    if (!c) return BITSORT_ERR_CUDA;
    if (min_value > max_value) return BITSORT_ERR_INVALID;
    // keys in [min_value, max_value] are classified as x - min_value, the
    // offsets 0 .. max_value - min_value, and written back unshifted
    const uint32_t span_max = max_value - min_value;
    bitsort_status_t st = bsx_validate(keys, n, span_max, out);
    if (st != BITSORT_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaSetDevice(c->device) != cudaSuccess) return BITSORT_ERR_CUDA;
    if (n == 0) return write_trivial_result(c, d_result, s);
    const uint64_t M = (uint64_t)span_max + 1;
    bsx_config cfg = bsx_lookup_config(c, n, M);
    return launch_single(c, cfg, keys, n, M, out, d_result, s, 0, min_value);
}

extern "C" bitsort_status_t bitsort_host(bitsort_ctx_t *c, const uint32_t *h_keys, uint64_t n, uint32_t max_value,
                                         uint32_t *h_out, bitsort_result_t *h_result, bitsort_stream_t stream) {
    bsx_range nvtx_range_("bitsort_host");
    if (!c) c = bsx_default_ctx();
    if (!c) return BITSORT_ERR_CUDA;
    if (n > 0 && (!h_keys || !h_out)) return BITSORT_ERR_INVALID;
    if (n > (uint64_t)max_value + 1) return BITSORT_ERR_INVALID;   // the keys cannot be distinct
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaSetDevice(c->device) != cudaSuccess) return BITSORT_ERR_CUDA;
    cudaError_t e = cudaSuccess;
    if (n == 0) {
        e = cudaMemsetAsync(c->result, 0, sizeof(bitsort_result_t), s);
    } else {
        if (c->host_io_cap < n) {
            c->host_io_cap = 0;
            e = regrow(c, reinterpret_cast<void **>(&c->host_io), 2 * n * sizeof(uint32_t), s);
            if (e != cudaSuccess) {
                c->host_io = nullptr;
                return BITSORT_ERR_NOMEM;
            }
            c->host_io_cap = n;
        }
        uint32_t *dk = c->host_io, *dout = c->host_io + c->host_io_cap;
        e = cudaMemcpyAsync(dk, h_keys, n * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return bsx_check(e);
        const uint64_t M = (uint64_t)max_value + 1;
        bitsort_status_t st = launch_single(c, bsx_lookup_config(c, n, M), dk, n, M, dout, nullptr, s, 0);
        if (st != BITSORT_OK) return st;
        e = cudaMemcpyAsync(h_out, dout, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess && h_result)
        e = cudaMemcpyAsync(h_result, c->result, sizeof(bitsort_result_t), cudaMemcpyDeviceToHost, s);
    return bsx_check(e);
}

extern "C" bitsort_status_t bitsort(const uint32_t *keys, size_t n, uint32_t max_value, uint32_t *out,
                                    bitsort_stream_t stream) {
    return bitsort_ex(nullptr, keys, (uint64_t)n, max_value, out, nullptr, stream);
}

bitsort_status_t bsx_reset_scratch(bitsort_ctx *c) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return BITSORT_ERR_CUDA;
    e = cudaMemset(c->fixed, 0, c->fixed_bytes);
    if (e == cudaSuccess && c->bitmap) e = cudaMemset(c->bitmap, 0, c->bitmap_words * 4);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();   // the memsets are done before any stream uses the scratch
    return bsx_check(e);
}

extern "C" bitsort_status_t bitsort_sync_status(bitsort_ctx_t *c, bitsort_stream_t stream, uint64_t *count) {
    if (!c) c = bsx_default_ctx();
    if (!c) return BITSORT_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) return BITSORT_ERR_CUDA;
    bitsort_result_t r;
    if (cudaMemcpy(&r, c->result, sizeof(r), cudaMemcpyDeviceToHost) != cudaSuccess) return BITSORT_ERR_CUDA;
    if (count) *count = r.count;
    if (r.status == BITSORT_ERR_TIMEOUT) bsx_reset_scratch(c);
    return (bitsort_status_t)r.status;
}

extern "C" bitsort_status_t bitsort_set_wait_limit_ms(bitsort_ctx_t *c, uint32_t ms) {
    if (!c) c = bsx_default_ctx();
    if (!c || ms == 0) return BITSORT_ERR_INVALID;
    c->wait_limit_ns = (uint64_t)ms * 1000000ull;
    return BITSORT_OK;
}

extern "C" bitsort_status_t bitsort_debug_stalled_launch(bitsort_ctx_t *c, const uint32_t *keys, uint64_t n,
                                                         uint32_t max_value, uint32_t *out,
                                                         bitsort_stream_t stream) {
    if (!c) c = bsx_default_ctx();
    if (!c) return BITSORT_ERR_CUDA;
    bitsort_status_t st = bsx_validate(keys, n, max_value, out);
    if (st != BITSORT_OK || n == 0) return st == BITSORT_OK ? BITSORT_ERR_INVALID : st;
    uint64_t M = (uint64_t)max_value + 1;
    bsx_config cfg;
    cfg.path = BITSORT_PATH_PARTITION;
    cfg.layout = LAYOUT_EXACT;
    cfg.persistent = true;  // the bucket items wait on the partition tiles inside one launch
    cfg.threads = 256;
    cfg.S = (uint32_t)std::max<uint64_t>(128, ceil_div(M, 4));  // four buckets
    return launch_single(c, cfg, keys, n, M, out, nullptr, reinterpret_cast<cudaStream_t>(stream), 1);
}

extern "C" bitsort_status_t bitsort_set_phase_timing(bitsort_ctx_t *c, int enable) {
    if (!c) c = bsx_default_ctx();
    if (!c) return BITSORT_ERR_CUDA;
    if (enable && !c->tev[0]) {
        for (int i = 0; i < 9; ++i)
            if (cudaEventCreate(&c->tev[i]) != cudaSuccess) return BITSORT_ERR_CUDA;
    }
    c->timing = enable != 0;
    c->tcount = 0;
    return BITSORT_OK;
}

extern "C" bitsort_status_t bitsort_phase_times(bitsort_ctx_t *c, float *ms, int *kinds, int *count) {
    if (!c) c = bsx_default_ctx();
    if (!c || !ms || !kinds || !count) return BITSORT_ERR_INVALID;
    *count = 0;
    if (!c->timing || c->tcount == 0) return BITSORT_OK;
    if (cudaEventSynchronize(c->tev[c->tcount]) != cudaSuccess) return BITSORT_ERR_CUDA;
    for (int i = 0; i < c->tcount; ++i) {
        float t = 0;
        cudaEventElapsedTime(&t, c->tev[i], c->tev[i + 1]);
        ms[i] = t;
        kinds[i] = c->tkind[i];
    }
    *count = c->tcount;
    return BITSORT_OK;
}

extern "C" uint64_t bitsort_kernel_launches(const bitsort_ctx_t *c) {
    if (!c) return 0;
    return c->launches.load();
}

// --------------------------------------------------------------- tuning
static void to_public(const bsx_config &c, bitsort_config_t *o) {
    o->path = (int32_t)c.path;
    o->slice_values = c.S;
    o->block_threads = (uint32_t)c.threads;
    o->words_per_lane = c.wpl;
    o->stage = c.stage ? 1 : 0;
    o->layout = c.layout;
    o->persistent = c.persistent ? 1 : 0;
    o->emit = c.emit;
    o->part_stream = c.stream_part ? 1 : 0;
    o->summary = c.summary ? 1 : 0;
    o->part_threads = (uint32_t)c.part_threads;
    o->part_tile_keys = c.part_tile_keys;
    o->ms = c.ms;
}

extern "C" bitsort_status_t bitsort_set_config(bitsort_ctx_t *c, uint64_t n, uint32_t max_value,
                                               const bitsort_config_t *in) {
    if (!c) c = bsx_default_ctx();
    if (!c || !in) return BITSORT_ERR_INVALID;
    uint64_t M = (uint64_t)max_value + 1;
    std::lock_guard<std::mutex> lk(c->mu);
    auto key = std::make_pair(ilog2_ceil(n), ilog2_ceil(M));
    if (in->path == BITSORT_PATH_AUTO) {
        c->table.erase(key);
        return BITSORT_OK;
    }
    if (in->path < BITSORT_PATH_FUSED || in->path > BITSORT_PATH_GLOBAL) return BITSORT_ERR_INVALID;
    bsx_config cfg = bsx_default_config(c->sms, n, M);
    cfg.path = (bitsort_path_t)in->path;
    if (in->slice_values) cfg.S = in->slice_values;
    if (in->block_threads) cfg.threads = (int)in->block_threads;
    if (in->words_per_lane) cfg.wpl = in->words_per_lane;
    cfg.stage = in->stage != 0;
    cfg.layout = in->layout;
    cfg.persistent = in->persistent != 0;
    cfg.emit = in->emit;
    cfg.stream_part = in->part_stream != 0;
    cfg.summary = in->summary != 0;
    cfg.part_threads = (int)in->part_threads;
    cfg.part_tile_keys = in->part_tile_keys;
    c->table[key] = bsx_sanitize(cfg, n, M);
    return BITSORT_OK;
}

extern "C" bitsort_status_t bitsort_get_config(bitsort_ctx_t *c, uint64_t n, uint32_t max_value,
                                               bitsort_config_t *out) {
    if (!c) c = bsx_default_ctx();
    if (!c || !out) return BITSORT_ERR_INVALID;
    uint64_t M = (uint64_t)max_value + 1;
    to_public(bsx_sanitize(bsx_lookup_config(c, n, M), n, M), out);
    return BITSORT_OK;
}

extern "C" bitsort_status_t bitsort_plan_rule(int sms, uint32_t smem_per_block, uint64_t n, uint32_t max_value,
                                              bitsort_config_t *config, bitsort_plan_shape_t *shape) {
    if (sms < 1 || smem_per_block == 0 || !config) return BITSORT_ERR_INVALID;
    const uint64_t M = (uint64_t)max_value + 1;
    if (n > M) return BITSORT_ERR_INVALID;
    bsx_single_plan pl;
    bsx_plan_single(sms, smem_per_block, bsx_default_config(sms, n, M), n, M, false, true, pl);
    to_public(pl.cfg, config);
    if (shape) {
        memset(shape, 0, sizeof(*shape));
        shape->slices = pl.a.nslices;
        shape->tile_keys = pl.a.tile_keys;
        shape->part_threads = (uint32_t)pl.Tp;
        shape->bucket_threads = (uint32_t)pl.Tb;
        shape->smem_bytes = pl.cfg.persistent ? pl.engine_smem
                                              : std::max(pl.slice_smem, std::max(pl.part_smem, pl.hist_smem));
        shape->scratch_bytes = pl.a.layout == LAYOUT_CAPACITY ? (uint64_t)pl.a.nslices * pl.a.cap * 4u : 0u;
    }
    return BITSORT_OK;
}

// Candidate configurations for (n, M), deduplicated after sanitizing.
std::vector<bsx_config> bsx_candidates(const bitsort_ctx *c, uint64_t n, uint64_t M) {
    std::vector<bsx_config> out;
    auto push = [&](bitsort_path_t path, uint64_t S, int threads, uint32_t wpl, bool stage, uint32_t layout,
                    uint32_t emit = EMIT_WORD) {
        bsx_config cfg;
        cfg.path = path;
        cfg.S = (uint32_t)std::min<uint64_t>(S, 0xFFFFFF80u);
        cfg.threads = threads;
        cfg.wpl = wpl;
        cfg.stage = stage;
        cfg.layout = layout;
        cfg.emit = emit;
        cfg = bsx_sanitize(cfg, n, M);
        for (auto &o : out)
            if (o.path == cfg.path && o.S == cfg.S && o.threads == cfg.threads && o.wpl == cfg.wpl &&
                o.stage == cfg.stage && o.layout == cfg.layout && o.emit == cfg.emit)
                return;
        out.push_back(cfg);
    };
    // rank emission: slices sized for 1 or 2 CTAs per SM
    for (int threads : {256, 512}) {
        for (int per_sm : {1, 2, 3}) {
            const double per_value = 0.25 + 5.0 * (double)n / (double)M;
            const double budget = (double)(c->smem_optin / per_sm) - 2048.0;
            if (budget <= 0) continue;
            const uint64_t S = (uint64_t)(budget / per_value);
            for (uint32_t layout : {(uint32_t)LAYOUT_EXACT, (uint32_t)LAYOUT_CAPACITY}) {
                push(BITSORT_PATH_PARTITION, S, threads, 1, false, layout, EMIT_RANK);
                push(BITSORT_PATH_PARTITION, S / 2, threads, 1, false, layout, EMIT_RANK);
            }
        }
        if (M <= kMaxSliceValues) push(BITSORT_PATH_FUSED, M, threads, 1, false, LAYOUT_EXACT, EMIT_RANK);
    }
    for (int threads : {256, 512}) {
        for (uint32_t wpl : {1u, 2u, 4u}) {
            if (M <= kMaxSliceValues) push(BITSORT_PATH_FUSED, M, threads, wpl, false, LAYOUT_EXACT);
            for (uint32_t layout : {(uint32_t)LAYOUT_EXACT, (uint32_t)LAYOUT_CAPACITY}) {
                for (int k : {1, 2, 3, 4, 6, 8})
                    push(BITSORT_PATH_PARTITION, ceil_div(M, (uint64_t)k * c->sms), threads, wpl, false, layout);
                for (int lg : {16, 18, 20}) push(BITSORT_PATH_PARTITION, 1ull << lg, threads, wpl, false, layout);
            }
            for (int lg : {14, 16, 18, 20}) push(BITSORT_PATH_GLOBAL, 1ull << lg, threads, wpl, false, 0);
        }
        if (M <= kMaxSliceValues) push(BITSORT_PATH_FUSED, M, threads, 1, true, LAYOUT_EXACT);
        for (int k : {1, 2, 3}) {   // partition tiles streamed through bulk copies
            bsx_config sc = bsx_sanitize(bsx_default_config(c->sms, n, M), n, M);
            sc.threads = threads;
            sc.S = (uint32_t)ceil_div(M, (uint64_t)k * c->sms);
            sc.stream_part = true;
            sc = bsx_sanitize(sc, n, M);
            if (sc.path == BITSORT_PATH_PARTITION) out.push_back(sc);
        }
        for (int k : {2, 4}) {
            bsx_config pc = bsx_sanitize(bsx_default_config(c->sms, n, M), n, M);
            pc.threads = threads;
            pc.S = (uint32_t)ceil_div(M, (uint64_t)k * c->sms);
            pc.persistent = true;
            pc = bsx_sanitize(pc, n, M);
            if (pc.path != BITSORT_PATH_FUSED) out.push_back(pc);
        }
        push(BITSORT_PATH_PARTITION, ceil_div(M, 2ull * c->sms), threads, 1, true, LAYOUT_CAPACITY);
        push(BITSORT_PATH_PARTITION, ceil_div(M, 2ull * c->sms), threads, 1, true, LAYOUT_EXACT);
    }
    // the partition phase at each block size (the rule takes 1024 threads
    // from 1024 buckets, else the plan's)
    const size_t base_count = out.size();
    for (size_t k = 0; k < base_count; ++k) {
        const bsx_config b = out[k];
        if (b.path != BITSORT_PATH_PARTITION || b.persistent || b.part_threads) continue;
        for (int pt : {512, 1024}) {   // both tile sizes of each block size
            bsx_config v = b;
            v.part_threads = pt;
            v.part_tile_keys = (uint32_t)(kKeysPerThread * pt);
            out.push_back(v);
            v.part_tile_keys = (uint32_t)(kWideKeysPerThread * pt);
            out.push_back(v);
        }
    }
    // shared memory must fit
    std::vector<bsx_config> fit;
    for (auto &cfg : out) {
        ArrayDesc a;
        bsx_describe(cfg, nullptr, nullptr, n, M, a);
        if (bsx_smem_for(cfg, a.nslices, a.tile_keys, a.stage_cap) <= c->smem_optin) fit.push_back(cfg);
    }
    return fit;
}

static bitsort_status_t ensure_flush(bitsort_ctx *c) {
    if (c->flush) return BITSORT_OK;
    size_t bytes = std::max<size_t>(2 * c->l2_bytes, 256u << 20);
    cudaError_t e = cudaMalloc(&c->flush, bytes);
    if (e != cudaSuccess) return bsx_check(e);
    c->flush_bytes = bytes;
    return BITSORT_OK;
}

extern "C" bitsort_status_t bitsort_autotune(bitsort_ctx_t *c, const uint32_t *keys, uint32_t *out, uint64_t n,
                                             uint32_t max_value, bitsort_config_t *best_out) {
    bsx_range nvtx_range_("bitsort_autotune");
    if (!c) c = bsx_default_ctx();
    if (!c) return BITSORT_ERR_CUDA;
    bitsort_status_t st = bsx_validate(keys, n, max_value, out);
    if (st != BITSORT_OK) return st;
    if (n == 0 || keys == out) return BITSORT_ERR_INVALID;
    if (cudaSetDevice(c->device) != cudaSuccess) return BITSORT_ERR_CUDA;
    uint64_t M = (uint64_t)max_value + 1;
    if ((st = ensure_flush(c)) != BITSORT_OK) return st;
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return BITSORT_ERR_CUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e30;
    bsx_config best_cfg = bsx_default_config(c->sms, n, M);
    for (const bsx_config &cfg : bsx_candidates(c, n, M)) {
        // one warm-up, then the median of five cold-L2 runs
        ArrayDesc probe;
        bsx_describe(cfg, nullptr, nullptr, n, M, probe);
        if (bsx_smem_for(cfg, probe.nslices, probe.tile_keys, probe.stage_cap) > c->smem_optin) continue;
        if (launch_single(c, cfg, keys, n, M, out, nullptr, s, 0) != BITSORT_OK) continue;
        std::vector<float> ts;
        bool ok = true;
        for (int r = 0; r < 5 && ok; ++r) {
            cudaMemsetAsync(c->flush, r, c->flush_bytes, s);
            cudaEventRecord(e0, s);
            ok = launch_single(c, cfg, keys, n, M, out, nullptr, s, 0) == BITSORT_OK;
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) ok = false;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            ts.push_back(ms);
        }
        bitsort_result_t r;
        cudaMemcpy(&r, c->result, sizeof(r), cudaMemcpyDeviceToHost);
        // only a configuration that sorted the whole array counts
        if (!ok || r.status != BITSORT_OK || r.count != n) {
            if (r.status == BITSORT_ERR_TIMEOUT) bsx_reset_scratch(c);
            continue;
        }
        std::sort(ts.begin(), ts.end());
        double med = ts[ts.size() / 2];
        if (med < best) {
            best = med;
            best_cfg = cfg;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    if (best >= 1e30) return BITSORT_ERR_CUDA;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        best_cfg.ms = best;
        c->table[std::make_pair(ilog2_ceil(n), ilog2_ceil(M))] = best_cfg;
    }
    if (best_out) to_public(best_cfg, best_out);
    return BITSORT_OK;
}

extern "C" bitsort_status_t bitsort_tune_save(bitsort_ctx_t *c, const char *path) {
    if (!c) c = bsx_default_ctx();
    if (!c || !path) return BITSORT_ERR_INVALID;
    FILE *f = fopen(path, "w");
    if (!f) return BITSORT_ERR_INVALID;
    std::lock_guard<std::mutex> lk(c->mu);
    fprintf(f, "{\"version\": 3, \"entries\": [");
    bool first = true;
    for (auto &kv : c->table) {
        const bsx_config &g = kv.second;
        fprintf(f,
                "%s\n  {\"log2n\": %d, \"log2m\": %d, \"path\": %d, \"slice_values\": %u, \"threads\": %d, "
                "\"wpl\": %u, \"stage\": %d, \"layout\": %u, \"persistent\": %d, \"emit\": %u, \"part_stream\": %d, "
                "\"summary\": %d, \"part_threads\": %d, \"part_tile_keys\": %u, \"ms\": %.6f}",
                first ? "" : ",", kv.first.first, kv.first.second, (int)g.path, g.S, g.threads, g.wpl,
                g.stage ? 1 : 0, g.layout, g.persistent ? 1 : 0, g.emit, g.stream_part ? 1 : 0, g.summary ? 1 : 0,
                g.part_threads, g.part_tile_keys, g.ms);
        first = false;
    }
    fprintf(f, "\n]}\n");
    fclose(f);
    return BITSORT_OK;
}

extern "C" bitsort_status_t bitsort_tune_load(bitsort_ctx_t *c, const char *path) {
    if (!c) c = bsx_default_ctx();
    if (!c || !path) return BITSORT_ERR_INVALID;
    FILE *f = fopen(path, "r");
    if (!f) return BITSORT_ERR_INVALID;
    std::string text;
    char buf[4096];
    size_t k;
    while ((k = fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, k);
    fclose(f);
    std::map<std::pair<int, int>, bsx_config> table;
    size_t pos = 0;
    while ((pos = text.find("{\"log2n\"", pos)) != std::string::npos) {
        int ln = 0, lm = 0, p = 0, th = 0, stage = 0, pers = 0, pstream = 0, summary = 1, pth = 0;
        unsigned S = 0, wpl = 0, layout = 0, emit = 0, ptk = 0;
        double ms = 0;
        // version 3 entries carry part_threads and part_tile_keys, version 2
        // entries part_threads, version 1 entries neither
        const char *entry = text.c_str() + pos;
        const int got3 = sscanf(entry,
                   "{\"log2n\": %d, \"log2m\": %d, \"path\": %d, \"slice_values\": %u, \"threads\": %d, "
                   "\"wpl\": %u, \"stage\": %d, \"layout\": %u, \"persistent\": %d, \"emit\": %u, \"part_stream\": %d, "
                   "\"summary\": %d, \"part_threads\": %d, \"part_tile_keys\": %u, \"ms\": %lf",
                   &ln, &lm, &p, &S, &th, &wpl, &stage, &layout, &pers, &emit, &pstream, &summary, &pth, &ptk, &ms);
        const int got2 = got3 == 15 ? 14 : sscanf(entry,
                   "{\"log2n\": %d, \"log2m\": %d, \"path\": %d, \"slice_values\": %u, \"threads\": %d, "
                   "\"wpl\": %u, \"stage\": %d, \"layout\": %u, \"persistent\": %d, \"emit\": %u, \"part_stream\": %d, "
                   "\"summary\": %d, \"part_threads\": %d, \"ms\": %lf",
                   &ln, &lm, &p, &S, &th, &wpl, &stage, &layout, &pers, &emit, &pstream, &summary, &pth, &ms);
        if (got3 != 15) ptk = 0;
        if (got2 != 14) {
            pth = 0;
            if (sscanf(entry,
                       "{\"log2n\": %d, \"log2m\": %d, \"path\": %d, \"slice_values\": %u, \"threads\": %d, "
                       "\"wpl\": %u, \"stage\": %d, \"layout\": %u, \"persistent\": %d, \"emit\": %u, "
                       "\"part_stream\": %d, \"summary\": %d, \"ms\": %lf",
                       &ln, &lm, &p, &S, &th, &wpl, &stage, &layout, &pers, &emit, &pstream, &summary, &ms) != 13)
                return BITSORT_ERR_INVALID;
        }
        if (p < 1 || p > 3 || (th != 256 && th != 512 && th != 1024) || ln < 0 || ln > 64 || lm < 0 || lm > 33)
            return BITSORT_ERR_INVALID;
        bsx_config cfg;
        cfg.path = (bitsort_path_t)p;
        cfg.S = S;
        cfg.threads = th;
        cfg.wpl = wpl;
        cfg.stage = stage != 0;
        cfg.layout = layout;
        cfg.persistent = pers != 0;
        cfg.emit = emit;
        cfg.stream_part = pstream != 0;
        cfg.summary = summary != 0;
        cfg.part_threads = pth;
        cfg.part_tile_keys = ptk;
        cfg.ms = ms;
        table[std::make_pair(ln, lm)] = cfg;
        ++pos;
    }
    std::lock_guard<std::mutex> lk(c->mu);
    for (auto &kv : table) c->table[kv.first] = kv.second;
    return BITSORT_OK;
}
