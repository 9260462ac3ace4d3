// shard.cu -- bitsort_range_split(): the exchange step of one sort spread
// over several GPUs by value range (include/bitsort.h, multi-GPU section).
//
// Rank g of G owns the values [g*W, (g+1)*W) with W = ceil(M / G) rounded up
// to a multiple of 128.  Before the exchange, every rank groups its keys by
// the rank that owns them: the histogram and partition phases of the sort
// (phase_kernel, engine.cu) with one "bucket" per rank, in the exact layout,
// so that group g occupies [offset_g, offset_g + count_g) of the output and
// the groups follow one another in rank order.  A last one-CTA kernel hands
// the G counts to the caller and returns the context's scratch to zero (the
// bucket phase, which does that in a full sort, does not run here).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "engine.h"
#include "internal.h"

using namespace bsx;

namespace {

constexpr int kSplitThreads = 512;

// counts[0..parts) -> d_counts, outcome, and the scratch back to zero
__global__ void split_finish_kernel(uint32_t *counts, uint32_t *cursor, uint32_t *sync, uint32_t parts,
                                    uint64_t *d_counts, bitsort_result_t *result) {
    __shared__ unsigned long long total;
    if (threadIdx.x == 0) total = 0;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < parts; i += blockDim.x) {
        const uint32_t c = counts[i];
        if (d_counts) d_counts[i] = c;
        atomicAdd(&total, (unsigned long long)c);
        counts[i] = 0;
        cursor[i] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool range = sync[SY_RANGE] != 0;
        result->status = range ? BITSORT_ERR_KEY_RANGE : BITSORT_OK;
        result->reserved = 0;
        result->count = total;
        for (int k = 0; k < SY_COUNT; ++k) sync[k] = 0;
    }
}

}  // namespace

extern "C" uint64_t bitsort_range_width(uint32_t max_value, uint32_t parts) {
    if (parts == 0) return 0;
    const uint64_t M = (uint64_t)max_value + 1;
    const uint64_t W = (M + parts - 1) / parts;
    return (W + 127) / 128 * 128;
}

extern "C" bitsort_status_t bitsort_range_split(bitsort_ctx_t *c, const uint32_t *keys, uint64_t n,
                                                uint32_t max_value, uint32_t parts, uint32_t *out,
                                                uint64_t *d_counts, bitsort_result_t *d_result,
                                                bitsort_stream_t stream) {
    bsx_range nvtx_range_("bitsort_range_split");
    if (!c) c = bsx_default_ctx();
    if (!c) return BITSORT_ERR_CUDA;
    if (parts < 1 || parts > kMaxSlices || !d_counts) return BITSORT_ERR_INVALID;
    if (n > 0 && (!keys || !out || keys == out)) return BITSORT_ERR_INVALID;
    if (((uintptr_t)keys & 3u) || ((uintptr_t)out & 3u)) return BITSORT_ERR_INVALID;
    if (n > 0 && bsx_ranges_overlap(keys, out, n * sizeof(uint32_t))) return BITSORT_ERR_INVALID;
    if (n >= (1ull << 32)) return BITSORT_ERR_INVALID;   // positions are 32-bit
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaSetDevice(c->device) != cudaSuccess) return BITSORT_ERR_CUDA;
    bitsort_result_t *res = d_result ? d_result : c->result;
    const uint64_t M = (uint64_t)max_value + 1;
    const uint64_t W = bitsort_range_width(max_value, parts);
    if (n == 0 || W >= (1ull << 32)) {
        // nothing to group, or one rank owns every value: a copy
        cudaError_t e = cudaMemsetAsync(d_counts, 0, parts * sizeof(uint64_t), s);
        if (e == cudaSuccess && n > 0)
            e = cudaMemcpyAsync(out, keys, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess && n > 0)
            e = cudaMemcpyAsync(d_counts, &n, sizeof(uint64_t), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) {
            bitsort_result_t r = {BITSORT_OK, 0, n};
            // (keys above max_value are not checked on this path)
            e = cudaMemcpyAsync(res, &r, sizeof(r), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host values above go out of scope
        }
        return bsx_check(e);
    }

    // the histogram and partition phases with `parts` buckets of W values
    bsx_config cfg;
    cfg.path = BITSORT_PATH_PARTITION;
    cfg.layout = LAYOUT_EXACT;
    cfg.threads = kSplitThreads;
    cfg.persistent = false;
    cfg.S = (uint32_t)W;
    EngineParams p;
    memset(&p, 0, sizeof(p));
    ArrayDesc &a = p.one;
    bsx_describe(cfg, keys, out, n, M, a);   // (no slice-size rules: no bitmap slices are built)
    a.nslices = parts;
    a.part = out;
    a.counts = c->counts;
    a.cursor = c->cursor;
    a.offsets = c->offsets;
    a.look = c->look;
    a.sync = c->sync;
    a.result = res;
    p.ticket = c->ticket;
    p.wait_limit_ns = c->wait_limit_ns;
    const uint32_t hist_smem = hist_smem_bytes(parts);
    const uint32_t part_smem = part_phase_smem_bytes(parts, a.tile_keys);
    if (part_smem > c->smem_optin) return BITSORT_ERR_INVALID;
    int launched = 0;
    for (int kind : {(int)IT_HIST, (int)IT_PART}) {
        const uint32_t smem = kind == IT_HIST ? hist_smem : part_smem;
        int per_sm = 1;
        if (kernel_max_blocks_per_sm(kind, kSplitThreads, smem, &per_sm) != 0 || per_sm < 1) per_sm = 1;
        uint64_t grid = (uint64_t)c->sms * (uint64_t)per_sm * (kind == IT_PART ? 8u : 1u);
        grid = std::min<uint64_t>(grid, a.key_tiles);
        EngineParams q = p;
        q.total_items = a.key_tiles;
        const int e = kernel_launch(kind, q, kSplitThreads, smem, (int)std::max<uint64_t>(grid, 1), s, launched > 0);
        if (e != 0) {
            bsx_note_error(e, "range split launch");
            return BITSORT_ERR_CUDA;
        }
        ++launched;
    }
    split_finish_kernel<<<1, 256, 0, s>>>(c->counts, c->cursor, c->sync, parts, d_counts, res);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        bsx_note_error((int)e, "range split finish launch");
        return BITSORT_ERR_CUDA;
    }
    c->launches.fetch_add((uint64_t)launched + 1);
    return BITSORT_OK;
}
