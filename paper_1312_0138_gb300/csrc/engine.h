// engine.h -- device-side data layout shared by the sort kernels (engine.cu)
// and the host code that plans and launches them (api.cu, batch.cu,
// server.cu, noalloc.cu).
//
// The sort of one array (the paper's bitwise sort, Section V, in its bit-set
// form) is split into work items, executed either by one persistent kernel
// that takes items from a ticket counter in ascending order, or phase by phase
// by one kernel per item type:
//
//   HIST      count the keys of one tile per bucket (bucket = the value range
//             [b*S, (b+1)*S) of the array's bitmap); the last HIST tile of an
//             array turns the counts into bucket offsets.
//   PART      move the keys of one tile to their bucket's range of the
//             partition buffer.
//   BUCKET    build bucket b's bitmap slice in shared memory (OR of shifted
//             ones, Table I / Example 2), count its set bits (Example 6),
//             and write the set-bit positions to the output from its
//             bucket's offset (with distinct keys the set bits of the earlier
//             buckets are their key counts; repeated keys are closed up by
//             the array's last CTA).  An array of one bucket is sorted by
//             one BUCKET item straight from its input (the fused path).
//   GSCATTER  OR the keys of one tile into a global bitmap (atomics in L2).
//   GSCAN     load a slice of the global bitmap into shared memory, zero it
//             behind (so the bitmap is clean for the next call), then count,
//             look back and write out like BUCKET.
//
// An item only ever waits for items with smaller tickets, and every wait is
// bounded in time, so the kernel always terminates.
#pragma once
#include <stdint.h>
#include "../../include/bitsort.h"

namespace bsx {

enum ItemType : uint32_t { IT_HIST = 0, IT_PART = 1, IT_BUCKET = 2, IT_GSCATTER = 3, IT_GSCAN = 4,
                           IT_PARTS = 5 /* PART tiles streamed through bulk copies (phase kernel only) */,
                           IT_PARTW = 6 /* PART with wide tiles, 32 keys a thread (phase kernel, 512 or 1024 threads) */ };

enum SyncSlot : uint32_t {
    SY_HIST_DONE = 0,     // HIST tiles finished
    SY_OFFSETS_READY = 1, // bucket offsets published
    SY_PART_DONE = 2,     // PART (or GSCATTER) tiles finished
    SY_RANGE = 3,         // a key above max_value was seen
    SY_TIMEOUT = 4,       // a bounded wait ran out
    SY_SLICES_DONE = 5,   // BUCKET / GSCAN items finished
    SY_OVERFLOW = 6,      // CAPACITY layout: a bucket got more keys than it can hold
    SY_MISMATCH = 7,      // PARTITION: a slice holds fewer set bits than its bucket had keys
    SY_COUNT = 8
};

// Look-back status word: flag in bits 62..63, value in bits 0..61.
constexpr uint64_t LB_AGG = 1ull << 62;
constexpr uint64_t LB_PREFIX = 2ull << 62;
constexpr uint64_t LB_VALUE = (1ull << 62) - 1;

// Per-array descriptor, 16-byte aligned (kernel parameter or device table).
struct __align__(16) ArrayDesc {
    const uint32_t *keys;
    uint32_t *out;
    uint32_t *part;             // partition buffer (n entries; may alias out)
    uint32_t *bitmap;           // global bitmap (GLOBAL path), ceil(M/32) words, zero on entry
    uint32_t *counts;           // [nslices] keys per bucket (zero on entry)
    uint32_t *cursor;           // [nslices] reservation cursor (zero on entry)
    uint64_t *offsets;          // [nslices] first partition-buffer index of each bucket
    uint64_t *look;             // [nslices] look-back status (zero on entry)
    uint32_t *sync;             // [SY_COUNT] counters (zero on entry)
    bitsort_result_t *result;   // outcome
    uint64_t n;
    uint64_t M;                 // max_value + 1
    uint64_t div_magic;         // ceil(2^64 / S): bucket of x = mulhi(x, div_magic)
    uint32_t S;                 // values per slice, a multiple of 32
    uint32_t nslices;           // buckets (PARTITION/FUSED) or scan tiles (GLOBAL)
    uint32_t tile_keys;         // keys per HIST/PART/GSCATTER tile
    uint32_t key_tiles;         // number of such tiles
    uint32_t path;              // bitsort_path_t
    uint32_t stall;             // extra never-scheduled PART tiles (failure-path test)
    uint64_t cap;               // CAPACITY layout: partition-buffer entries per bucket
    uint32_t layout;            // LAYOUT_EXACT or LAYOUT_CAPACITY (PARTITION path)
    uint32_t wpl;               // bitmap words per lane in the scan (1, 2 or 4)
    uint32_t stage;             // 1: stage set-bit positions in shared memory per warp
    uint32_t phased;            // 1: phases are separate kernels (ordered by the stream)
    uint32_t emit;              // EMIT_WORD or EMIT_RANK (BUCKET items)
    uint32_t stage_cap;         // EMIT_RANK: outputs a slice may stage in shared memory
    uint32_t summary;           // 1: sparse slices keep a summary bitmap (one bit per word)
    uint32_t bias;              // keys are classified as x - bias (mod 2^32); outputs get it back
    uint32_t sgroup;            // slices per BUCKET item (0 or 1: one; see item_bucket)
    uint32_t s_shift;           // log2(S) when S is a power of 2 (bucket = shift), else 0 (division)
};

// How a BUCKET item turns its bitmap slice into output positions.
//   EMIT_WORD  every lane walks the set bits of its words (ascending) and
//              writes their positions; the lanes' counts are prefix-summed.
//   EMIT_RANK  the exclusive popcount prefix of every word is stored next to
//              the bitmap; each key x then finds its own index,
//              prefix[x/32] + popcount of the bits of word x/32 below x, and
//              is written there in a shared-memory copy of the slice's output,
//              which leaves in coalesced stores.  Same result: the set bits
//              in index order.  Needs the slice's keys twice and room for the
//              slice's outputs; a slice with more outputs than stage_cap falls
//              back to EMIT_WORD.
enum Emit : uint32_t { EMIT_WORD = 0, EMIT_RANK = 1 };

// PARTITION-path layouts of the partition buffer.
//   EXACT     a histogram pass gives every bucket its exact range (prefix of
//             the counts); n entries in all, the output buffer can hold them.
//   CAPACITY  bucket b owns entries [b*cap, (b+1)*cap) with cap = min(S, n):
//             distinct keys never overflow it, so no histogram pass is needed.
//             Every tile reserves its run in each bucket with a global atomic.
enum Layout : uint32_t { LAYOUT_EXACT = 0, LAYOUT_CAPACITY = 1 };

// A run of `count` consecutive tickets that all belong to one (array, type).
struct Segment {
    uint32_t start;  // first ticket
    uint32_t array;
    uint32_t type;
    uint32_t first;  // index of the first item within the array's items of this type
};

constexpr int kInlineSegments = 4;

struct EngineParams {
    const ArrayDesc *arrays;       // device table, or nullptr: use `one`
    const Segment *segments;       // device table, or nullptr: use `seg`
    uint32_t nseg;
    uint32_t total_items;
    uint32_t *ticket;              // [0] next ticket, [1] finished CTAs (zero on entry)
    uint64_t wait_limit_ns;
    ArrayDesc one;
    Segment seg[kInlineSegments];
};

// Shared-memory sizes (bytes) an item type needs for a given configuration.
// Slice items start with a summary bitmap of kSummaryWords words (one bit per
// bitmap word of a slice of up to 2^20 values), used by sparse slices.
constexpr uint32_t kSummaryWords = 1024;
constexpr uint32_t kStageWords = 1024 + 4;  // per warp: staged positions (+ room for the 16-byte alignment shift)
// Staging words per warp for a block of `threads`: the block's staging area
// stays at 16 x kStageWords words, so a 1024-thread block gives each warp
// half (a step that does not fit is stored directly).
__host__ __device__ constexpr uint32_t stage_words(int threads) {
    return threads > 512 ? 512u + 4u : kStageWords;
}
inline uint32_t slice_smem_bytes(uint32_t S, int threads, bool stage) {
    uint32_t words = (S + 31) / 32;
    uint32_t w4 = (words + 3) & ~3u;
    return kSummaryWords * 4 + w4 * 4 + (stage ? (uint32_t)(threads / 32) * stage_words(threads) * 4 : 0u);
}
// EMIT_RANK: bitmap + per-word prefix + staged outputs
inline uint32_t rank_smem_bytes(uint32_t S, uint32_t stage_cap) {
    uint32_t words = (S + 31) / 32;
    uint32_t w4 = (words + 3) & ~3u;
    return kSummaryWords * 4 + w4 * 8 + ((stage_cap + 3) & ~3u) * 4;
}
// PART: per bucket (plus one discard bin) count, delta, limit; the tile and its bucket tags
inline uint32_t part_smem_bytes(uint32_t nslices, uint32_t tile_keys) {
    return (nslices + 1) * 12u + tile_keys * 6u + 16u;
}
inline uint32_t hist_smem_bytes(uint32_t nslices) { return nslices * 4u; }
// PART phase kernel: per bin (plus the discard bin) count / prefix, bucket
// base and run words; the tile
inline uint32_t part_phase_smem_bytes(uint32_t nslices, uint32_t tile_keys) {
    const uint32_t nq = (nslices + 1 + 3) & ~3u;   // each per-bin array rounded to 16 bytes
    return nq * 16u + tile_keys * 4u + 16u;
}
// streaming PART: bins, bucket tags, two landing buffers, two mbarriers (128-byte aligned parts)
inline uint32_t part_stream_smem_bytes(uint32_t nslices, uint32_t tile_keys) {
    const uint32_t a = ((nslices + 1) * 12u + 127u) & ~127u;
    const uint32_t t = (tile_keys * 2u + 127u) & ~127u;
    return a + t + 2u * tile_keys * 4u + 16u;
}

constexpr int kKeysPerThread = 16;   // keys per thread in one HIST/PART/GSCATTER tile
constexpr int kWideKeysPerThread = 32;   // keys per thread in one wide PART tile (IT_PARTW)
constexpr uint32_t kMaxSlices = 8192;   // bucket ids fit 16 bits in the partition tile

// Host-side launch entry points (engine.cu).
int engine_launch(const EngineParams &p, int threads, uint32_t smem_bytes, int grid, void *stream);
int engine_max_blocks_per_sm(int threads, uint32_t smem_bytes, int *blocks);
int engine_set_smem_limit(int threads, uint32_t smem_bytes);
// One phase (kind = an ItemType) of a single array, or the persistent engine
// (kind = -1); pdl = may start while the previous kernel of the stream drains.
int kernel_launch(int kind, const EngineParams &p, int threads, uint32_t smem_bytes, int grid, void *stream,
                  bool pdl);
int kernel_max_blocks_per_sm(int kind, int threads, uint32_t smem_bytes, int *blocks);

}  // namespace bsx
