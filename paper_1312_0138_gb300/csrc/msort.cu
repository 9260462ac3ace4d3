// msort.cu -- the paper's Algorithm 1 itself on the GPU: the keys are split
// stably by their bits, least significant first (Section V, Algorithm 1's
// first function: for each bit, the keys whose bit is 0 go first and the keys
// whose bit is 1 follow, both in their current order).  Unlike the bitmap
// form this sorts any multiset (Theorem 1 covers an arbitrary array).
//
// A pass splits by D consecutive bits at once into 2^D groups kept in group
// order; D = 1 is the paper's own pass.  ceil(bits / D) passes cover the bits
// of the range's largest offset, where the paper's loop runs over the whole
// type.  Per pass one kernel reads every key once and writes it once:
//   * one histogram kernel reads the keys before the first pass and counts
//     the keys of every group of every pass, so the first tile of a pass knows
//     where each group starts in the output;
//   * a tile ranks its keys inside each group in index order (warp ballots on
//     the group's bits), publishes its per-group counts, and learns how many
//     keys of each group the tiles before it hold from a decoupled look-back
//     (Merrill & Garland, "Single-pass Parallel Prefix Scan with Decoupled
//     Look-back", NVIDIA NVR-2016-002), one thread per group;
//   * the tile is reordered by group in shared memory, then written so that
//     consecutive threads write consecutive positions of a group's run.
// A tile takes its index from a ticket counter when it starts, so it only
// waits on tiles that are already running; every wait is bounded in time.
//
// Look-back words carry the epoch of their pass, so the array is never
// cleared between passes: a word of an older pass reads as "not ready".
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "engine.h"
#include "internal.h"
#include "ptx.cuh"

namespace {

using namespace bsx;

constexpr unsigned kFull = 0xffffffffu;
constexpr int kT = 512;                  // threads of a tile
constexpr int kK = 16;                   // keys per thread
constexpr uint32_t kTile = kT * kK;      // keys per tile
constexpr int kNW = kT / 32;
constexpr uint32_t kMaxSplitBits = 8;    // at most 256 groups per pass
constexpr uint32_t kMaxPasses = 32;
constexpr uint32_t kHistWords = 1024;    // passes x groups: at most 4 x 256 (8 bits), 32 x 2 (1 bit)

// small per-call block (cleared before the histogram kernel)
constexpr uint32_t kMiscTicket = 0;      // [0, 32): tile ticket of each pass
constexpr uint32_t kMiscRange = 32;      // a key lies outside the range
constexpr uint32_t kMiscTimeout = 33;    // a bounded wait expired
constexpr uint32_t kMiscDone = 34;       // tiles of the last pass that have finished
constexpr uint32_t kMiscHist = 64;       // [64, 64 + passes x groups): group counts
constexpr uint32_t kMiscWords = kMiscHist + kHistWords;

// look-back word: epoch (30 bits) | flag (2 bits) | count (32 bits)
constexpr uint64_t kFlagAgg = 1ull << 32;      // the tile's own count
constexpr uint64_t kFlagPrefix = 2ull << 32;   // count of the group up to and including the tile
constexpr int kEpochShift = 34;
constexpr uint32_t kEpochMax = (1u << 30) - 1;

constexpr int kKindHist = 16, kKindSplit = 17;   // phase-timing kinds

struct PassArgs {
    const uint32_t *src;
    uint32_t *dst;
    uint64_t *look;              // ntiles x groups look-back words
    uint32_t *misc;
    bitsort_result_t *result;    // last pass only: written by the last tile to finish
    uint64_t wait_limit_ns;
    uint32_t n;
    uint32_t bias;               // keys are split by x - bias
    uint32_t shift;              // lowest bit of this pass's group
    uint32_t pass;
    uint32_t ntiles;
    uint32_t epoch;
};

// Exclusive prefix of v over the threads of the block (all threads call).
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *s_scan) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) s_scan[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < kNW ? s_scan[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, wi, d);
            if (lane >= d) wi += y;
        }
        if (lane < kNW) s_scan[lane] = wi - w;
    }
    __syncthreads();
    const uint32_t r = s_scan[warp] + incl - v;
    __syncthreads();
    return r;
}

__device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Keys of group g in the tiles before `tile` (the caller thread owns g).
// The statuses of kWindow predecessors are read at once, then consumed from
// the nearest down to the first inclusive count; an entry that is not yet
// published is read again after a short sleep.  Only the words' own values
// are used, so relaxed loads suffice.  Bounded: on expiry the call's timeout
// flag is raised and the partial sum is returned.
constexpr int kWindow = 8;
__device__ uint32_t tile_lookback(const uint64_t *look, uint32_t tile, uint32_t g, uint32_t R, uint32_t epoch,
                                  uint32_t *timeout, uint64_t limit_ns) {
    uint32_t excl = 0;
    int64_t top = (int64_t)tile - 1;   // nearest predecessor not yet consumed
    uint64_t spins = 0;
    WaitClock clk;
    const uint64_t cap = limit_ns / 16 + 4096;
    while (top >= 0) {
        uint64_t v[kWindow];
#pragma unroll
        for (int w = 0; w < kWindow; ++w)
            v[w] = top - w >= 0 ? ld_relaxed_u64(look + (uint64_t)(top - w) * R + g)
                                : ((uint64_t)epoch << kEpochShift) | kFlagPrefix;   // before tile 0: nothing
        int w = 0;
#pragma unroll
        for (; w < kWindow; ++w) {
            const uint32_t flag = (uint32_t)(v[w] >> 32) & 3u;
            if ((uint32_t)(v[w] >> kEpochShift) != epoch || flag == 0) break;
            excl += (uint32_t)v[w];
            if (flag == 2) return excl;
        }
        top -= w;
        if (w < kWindow && top >= 0) {   // wait for that one alone before reading a window again
            const uint64_t *p = look + (uint64_t)top * R + g;
            while (true) {
                const uint64_t u = ld_relaxed_u64(p);
                if ((uint32_t)(u >> kEpochShift) == epoch && ((uint32_t)(u >> 32) & 3u) != 0) break;
                if (spins == 0) clk.start();
                ++spins;
                if (spins > cap ||
                    ((spins & 15) == 0 && (clk.expired(limit_ns) || ld_acquire_u32(timeout) != 0))) {
                    atomicOr(timeout, 1u);
                    return excl;
                }
                __nanosleep(32);
            }
        }
    }
    return excl;
}

// Counts of every group of every pass (one read of the keys) and the range
// check: x - bias must not exceed maxv.
__global__ void __launch_bounds__(kT) ms_hist_kernel(const uint32_t *keys, uint64_t n, uint32_t bias, uint32_t maxv,
                                                     uint32_t D, uint32_t P, uint32_t *misc) {
    __shared__ uint32_t h[kHistWords];
    const uint32_t R = 1u << D, H = P * R, mask = R - 1;
    for (uint32_t i = threadIdx.x; i < H; i += kT) h[i] = 0;
    __syncthreads();
    bool bad = false;
    auto count = [&](uint32_t x) {
        const uint32_t y = x - bias;
        bad |= y > maxv;
        uint32_t sh = 0;
        for (uint32_t p = 0; p < P; ++p, sh += D) atomicAdd(&h[p * R + ((y >> sh) & mask)], 1u);
    };
    const uint64_t gt = (uint64_t)blockIdx.x * kT + threadIdx.x, stride = (uint64_t)gridDim.x * kT;
    const uint32_t mis = (uint32_t)((reinterpret_cast<uintptr_t>(keys) & 15u) >> 2);
    const uint64_t head = std::min<uint64_t>(mis ? 4u - mis : 0u, n);
    if (gt < head) count(__ldcg(keys + gt));
    const uint64_t nv = (n - head) >> 2;
    const uint4 *v = reinterpret_cast<const uint4 *>(keys + head);
    uint64_t i = gt;
    for (; i + 3 * stride < nv; i += 4 * stride) {
        uint4 q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) q[u] = __ldcg(v + i + u * stride);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            count(q[u].x);
            count(q[u].y);
            count(q[u].z);
            count(q[u].w);
        }
    }
    for (; i < nv; i += stride) {
        const uint4 q = __ldcg(v + i);
        count(q.x);
        count(q.y);
        count(q.z);
        count(q.w);
    }
    const uint64_t tail = head + (nv << 2);
    if (tail + gt < n) count(__ldcg(keys + tail + gt));
    bad = __syncthreads_or(bad);
    for (uint32_t k = threadIdx.x; k < H; k += kT)
        if (h[k]) atomicAdd(&misc[kMiscHist + k], h[k]);
    if (bad && threadIdx.x == 0) atomicOr(&misc[kMiscRange], 1u);
}

// One stable split by the D bits at `shift`: tile `ticket` of the pass.
template <int D>
__global__ void __launch_bounds__(kT, 1024 / kT) ms_pass_kernel(PassArgs a) {
    constexpr uint32_t R = 1u << D;
    __shared__ uint32_t s_keys[kTile];
    __shared__ uint16_t s_warp[kNW][R];   // keys of each group per warp, then the warp's offset in the group (< tile)
    __shared__ uint32_t s_start[R];       // the group's count, then its start in the reordered tile
    __shared__ uint32_t s_base[R];        // output position of the group's first key in the tile, minus its start
    __shared__ uint32_t s_scan[kNW];
    __shared__ uint32_t s_tile;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tile = atomicAdd(&a.misc[kMiscTicket + a.pass], 1u);
    for (uint32_t i = threadIdx.x; i < (uint32_t)kNW * R; i += kT) (&s_warp[0][0])[i] = 0;
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint64_t t0 = (uint64_t)tile * kTile;
    const uint32_t tn = (uint32_t)std::min<uint64_t>(kTile, a.n - t0);
    const uint64_t tag = (uint64_t)a.epoch << kEpochShift;

    // warp w holds tile positions [w * 32 * kK, (w + 1) * 32 * kK); in step j
    // lane l holds position w * 32 * kK + 32 * j + l, so (j, l) is index order
    const uint32_t wb = (uint32_t)warp * 32u * kK;
    uint32_t x[kK], rk[kK];
#pragma unroll
    for (int j = 0; j < kK; ++j) {
        const uint32_t i = wb + 32u * j + lane;
        x[j] = i < tn ? __ldcg(a.src + t0 + i) : 0u;
    }
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < kK; ++j) {
        const bool valid = wb + 32u * j + lane < tn;
        const uint32_t g = ((x[j] - a.bias) >> a.shift) & (R - 1);
        unsigned peers = __ballot_sync(kFull, valid);
#pragma unroll
        for (int b = 0; b < D; ++b) {
            const bool bit = (g >> b) & 1u;
            const unsigned bb = __ballot_sync(kFull, bit);
            peers &= bit ? bb : ~bb;
        }
        // valid lanes: `peers` = the valid lanes of this step in the same group
        // (one ballot per group bit: cheaper here than a warp match)
        const uint32_t below = __popc(peers & lt);
        uint32_t old = 0;
        if (valid && below == 0) {   // the group's first lane adds the step's keys of the group
            old = s_warp[warp][g];
            s_warp[warp][g] = (uint16_t)(old + __popc(peers));
        }
        old = __shfl_sync(kFull, old, valid ? __ffs(peers) - 1 : lane);
        rk[j] = old + below;
        __syncwarp();
    }
    __syncthreads();

    // per group: the tile's count and each warp's offset inside the group;
    // the count is published at once so that later tiles can go on
    for (uint32_t g = threadIdx.x; g < R; g += kT) {
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kNW; ++w) {
            const uint32_t c = s_warp[w][g];
            s_warp[w][g] = (uint16_t)run;
            run += c;
        }
        s_start[g] = run;
        if (tile != 0) st_relaxed_u64(a.look + (uint64_t)tile * R + g, tag | kFlagAgg | run);
    }
    __syncthreads();
    const uint32_t cnt = threadIdx.x < R ? s_start[threadIdx.x] : 0u;
    const uint32_t start = block_excl_scan(cnt, s_scan);
    uint32_t gstart = 0;   // tile 0: where each group starts in the output
    if (tile == 0) {
        const uint32_t h = threadIdx.x < R ? __ldcg(&a.misc[kMiscHist + a.pass * R + threadIdx.x]) : 0u;
        gstart = block_excl_scan(h, s_scan);
    }
    if (threadIdx.x < R) s_start[threadIdx.x] = start;
    __syncthreads();

    // reorder by group in shared memory: warps, steps and lanes in index order
#pragma unroll
    for (int j = 0; j < kK; ++j) {
        if (wb + 32u * j + lane < tn) {
            const uint32_t g = ((x[j] - a.bias) >> a.shift) & (R - 1);
            s_keys[s_start[g] + s_warp[warp][g] + rk[j]] = x[j];
        }
    }
    if (threadIdx.x < R) {
        const uint32_t g = threadIdx.x;
        uint32_t excl;
        if (tile == 0) {
            excl = gstart;
        } else {
            excl = tile_lookback(a.look, tile, g, R, a.epoch, &a.misc[kMiscTimeout], a.wait_limit_ns);
        }
        st_relaxed_u64(a.look + (uint64_t)tile * R + g, tag | kFlagPrefix | (uint32_t)(excl + cnt));
        s_base[g] = excl - start;
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < tn; i += kT) {
        const uint32_t v = s_keys[i];
        const uint32_t g = ((v - a.bias) >> a.shift) & (R - 1);
        a.dst[(uint32_t)(s_base[g] + i)] = v;
    }
    if (a.result) {
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicAdd(&a.misc[kMiscDone], 1u) == a.ntiles - 1) {
                __threadfence();
                uint32_t st = BITSORT_OK;
                if (ld_acquire_u32(&a.misc[kMiscTimeout]) != 0) st = BITSORT_ERR_TIMEOUT;
                else if (ld_acquire_u32(&a.misc[kMiscRange]) != 0) st = BITSORT_ERR_KEY_RANGE;
                a.result->count = a.n;
                a.result->reserved = 0;
                a.result->status = st;
            }
        }
    }
}

typedef void (*PassKernel)(PassArgs);
PassKernel pass_kernel(uint32_t D) {
    switch (D) {
        case 1: return ms_pass_kernel<1>;
        case 2: return ms_pass_kernel<2>;
        case 3: return ms_pass_kernel<3>;
        case 4: return ms_pass_kernel<4>;
        case 5: return ms_pass_kernel<5>;
        case 6: return ms_pass_kernel<6>;
        case 7: return ms_pass_kernel<7>;
        default: return ms_pass_kernel<8>;
    }
}

bitsort_status_t ensure_multiset_scratch(bitsort_ctx *c, uint64_t look_words, cudaStream_t s) {
    if (!c->ms_misc) {
        cudaError_t e = cudaMalloc(&c->ms_misc, kMiscWords * sizeof(uint32_t));
        if (e != cudaSuccess) {
            c->ms_misc = nullptr;
            return bsx_check(e);
        }
    }
    if (c->ms_look_words < look_words) {
        if (c->ms_look) {
            cudaDeviceSynchronize();
            cudaFree(c->ms_look);
            c->ms_look = nullptr;
            c->ms_look_words = 0;
        }
        cudaError_t e = cudaMalloc(&c->ms_look, look_words * sizeof(uint64_t));
        if (e != cudaSuccess) {
            c->ms_look = nullptr;
            return bsx_check(e);
        }
        // epoch 0 is never used; zeroed in the order of the stream that uses it
        e = cudaMemsetAsync(c->ms_look, 0, look_words * sizeof(uint64_t), s);
        if (e != cudaSuccess) return bsx_check(e);
        c->ms_look_words = look_words;
    }
    return BITSORT_OK;
}

// Split width and number of passes for keys whose offsets need `bits` bits.
void plan_passes(uint32_t bits, uint32_t split_bits, uint32_t *D, uint32_t *P) {
    if (split_bits) {
        *D = split_bits;
        *P = (bits + split_bits - 1) / split_bits;
    } else {   // fewest passes of at most 8 bits, the bits spread evenly over them
        *P = (bits + kMaxSplitBits - 1) / kMaxSplitBits;
        *D = (bits + *P - 1) / *P;
    }
}

bitsort_status_t multiset_run(bitsort_ctx *c, const uint32_t *keys, uint64_t n, uint32_t bias, uint32_t maxv,
                              uint32_t split_bits, uint32_t *out, bitsort_result_t *d_result, cudaStream_t s) {
    if (split_bits > kMaxSplitBits) return BITSORT_ERR_INVALID;
    if (n >= (1ull << 32)) return BITSORT_ERR_INVALID;   // positions are 32-bit
    if (n > 0 && (!keys || !out)) return BITSORT_ERR_INVALID;
    if (((uintptr_t)keys & 3u) || ((uintptr_t)out & 3u)) return BITSORT_ERR_INVALID;
    if (n > 0 && keys != out && bsx_ranges_overlap(keys, out, n * sizeof(uint32_t))) return BITSORT_ERR_INVALID;
    if (cudaSetDevice(c->device) != cudaSuccess) return BITSORT_ERR_CUDA;
    bitsort_result_t *res = d_result ? d_result : c->result;
    if (n == 0) return bsx_check(cudaMemsetAsync(res, 0, sizeof(bitsort_result_t), s));

    const uint32_t bits = maxv ? 32u - (uint32_t)__builtin_clz(maxv) : 1u;
    uint32_t D = 0, P = 0;
    plan_passes(bits, split_bits, &D, &P);
    if (P > kMaxPasses || P * (1u << D) > kHistWords) return BITSORT_ERR_INVALID;   // (never: D >= 1, bits <= 32)
    const uint32_t R = 1u << D;
    const uint32_t ntiles = (uint32_t)((n + kTile - 1) / kTile);
    bitsort_status_t st = ensure_multiset_scratch(c, (uint64_t)ntiles * R, s);
    if (st != BITSORT_OK) return st;
    const bool inplace = keys == out;
    // pass p writes `out` when P - 1 - p is even (the last pass ends in out);
    // in place with an odd P the first pass would write the keys it reads,
    // so the parity shifts and a copy ends the sort
    const bool copy_back = inplace && (P & 1u);
    if (P > 1 || inplace) {
        if ((st = bsx_ensure_part(c, n, s)) != BITSORT_OK) return st;
    }
    uint32_t *tmp = c->part;
    if (c->ms_epoch + P > kEpochMax) {   // epochs wrap: start the look-back array afresh
        if (cudaDeviceSynchronize() != cudaSuccess) return BITSORT_ERR_CUDA;
        if (cudaMemsetAsync(c->ms_look, 0, c->ms_look_words * sizeof(uint64_t), s) != cudaSuccess)
            return BITSORT_ERR_CUDA;
        c->ms_epoch = 0;
    }

    cudaError_t e = cudaMemsetAsync(c->ms_misc, 0, kMiscWords * sizeof(uint32_t), s);
    if (e != cudaSuccess) return bsx_check(e);
    if (c->timing) {
        cudaEventRecord(c->tev[0], s);
        c->tkind[0] = kKindHist;
        c->tkind[1] = kKindSplit;
    }
    {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ms_hist_kernel, kT, 0);
        uint64_t grid = (uint64_t)c->sms * (uint64_t)std::max(per_sm, 1);
        grid = std::min<uint64_t>(grid, (n + 4ull * kT - 1) / (4ull * kT));
        ms_hist_kernel<<<(unsigned)std::max<uint64_t>(grid, 1), kT, 0, s>>>(keys, n, bias, maxv, D, P, c->ms_misc);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            bsx_note_error((int)e, "multiset histogram launch");
            return BITSORT_ERR_CUDA;
        }
    }
    if (c->timing) cudaEventRecord(c->tev[1], s);
    PassKernel kern = pass_kernel(D);
    const uint32_t *src = keys;
    for (uint32_t p = 0; p < P; ++p) {
        const bool to_out = ((P - 1 - p + (copy_back ? 1u : 0u)) & 1u) == 0;
        PassArgs a;
        memset(&a, 0, sizeof(a));
        a.src = src;
        a.dst = to_out ? out : tmp;
        a.look = c->ms_look;
        a.misc = c->ms_misc;
        a.result = p + 1 == P ? res : nullptr;
        a.wait_limit_ns = c->wait_limit_ns;
        a.n = (uint32_t)n;
        a.bias = bias;
        a.shift = p * D;
        a.pass = p;
        a.ntiles = ntiles;
        a.epoch = ++c->ms_epoch;
        kern<<<ntiles, kT, 0, s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            bsx_note_error((int)e, "multiset split launch");
            return BITSORT_ERR_CUDA;
        }
        src = a.dst;
    }
    if (c->timing) {
        cudaEventRecord(c->tev[2], s);
        c->tcount = 2;
    }
    if (copy_back) {
        e = cudaMemcpyAsync(out, tmp, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return bsx_check(e);
    }
    c->launches.fetch_add(1 + P);
    return BITSORT_OK;
}

}  // namespace

void bsx_multiset_free(bitsort_ctx *c) {
    if (c->ms_look) cudaFree(c->ms_look);
    if (c->ms_misc) cudaFree(c->ms_misc);
    c->ms_look = nullptr;
    c->ms_misc = nullptr;
    c->ms_look_words = 0;
}

extern "C" bitsort_status_t bitsort_multiset(bitsort_ctx_t *c, const uint32_t *keys, uint64_t n, uint32_t max_value,
                                             uint32_t split_bits, uint32_t *out, bitsort_result_t *d_result,
                                             bitsort_stream_t stream) {
    bsx_range nvtx_range_("bitsort_multiset");
    if (!c) c = bsx_default_ctx();
    if (!c) return BITSORT_ERR_CUDA;
    return multiset_run(c, keys, n, 0u, max_value, split_bits, out, d_result,
                        reinterpret_cast<cudaStream_t>(stream));
}

extern "C" bitsort_status_t bitsort_multiset_i32(bitsort_ctx_t *c, const int32_t *keys, uint64_t n,
                                                 int32_t min_value, int32_t max_value, uint32_t split_bits,
                                                 int32_t *out, bitsort_result_t *d_result, bitsort_stream_t stream) {
    bsx_range nvtx_range_("bitsort_multiset_i32");
    if (!c) c = bsx_default_ctx();
    if (!c) return BITSORT_ERR_CUDA;
    if (min_value > max_value) return BITSORT_ERR_INVALID;
    // offsets x - min_value (mod 2^32) keep the signed order
    const uint32_t bias = (uint32_t)min_value;
    return multiset_run(c, reinterpret_cast<const uint32_t *>(keys), n, bias, (uint32_t)max_value - bias, split_bits,
                        reinterpret_cast<uint32_t *>(out), d_result, reinterpret_cast<cudaStream_t>(stream));
}
