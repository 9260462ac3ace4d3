// widths.cu -- the bitmap sort for keys stored in 8, 16 and 64 bits
// (Algorithm 1 is written for any integer type T; the bit-set form only
// needs the keys' values).
//   * 8- and 16-bit keys: at most 65,536 values, so the whole bitmap (8 KiB)
//     sits in one CTA's shared memory.  One kernel ORs every key into it
//     (Table I, Example 2), counts the set bits of each thread's words
//     (Example 6), prefix-sums the counts across the block and writes the set
//     positions, bit 0 first (Section II numbering), in the key type.
//   * 64-bit keys bounded by max_value < 2^32: one kernel narrows the keys
//     to 32 bits (a key above max_value, including one that differs only
//     above bit 31, is flagged and replaced by 2^32 - 1), the 32-bit sort
//     runs on the narrowed copy, and a last kernel widens the sorted values
//     into the caller's buffer and writes the outcome.  With
//     max_value = 2^32 - 1 a replaced key would land on the top value: the
//     narrowing kernel also records whether a genuine key holds that value,
//     and the widening kernel drops the top value when only replacements
//     produced it.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "engine.h"
#include "internal.h"

namespace {

constexpr int kSmallThreads = 1024;
constexpr uint32_t kSmallWords = 2048;   // 65,536 bits

// wide-key scratch block (device, per context): flags and the 32-bit sort's outcome
struct WideMisc {
    uint32_t bad;       // a key above max_value
    uint32_t top;       // a key equal to 2^32 - 1 (in range)
    uint32_t pad[2];
    bitsort_result_t inner;
};

template <typename K>
__global__ void __launch_bounds__(kSmallThreads) small_sort_kernel(const K *keys, uint32_t n, uint32_t maxv, K *out,
                                                                   bitsort_result_t *res) {
    __shared__ uint32_t bm[kSmallWords];
    __shared__ uint32_t wsum[kSmallThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t words = (maxv >> 5) + 1;
    for (uint32_t i = threadIdx.x; i < words; i += kSmallThreads) bm[i] = 0u;
    __syncthreads();
    bool bad = false;
    for (uint32_t i = threadIdx.x; i < n; i += kSmallThreads) {
        const uint32_t x = keys[i];
        if (x > maxv) bad = true;
        else atomicOr(&bm[x >> 5], 1u << (x & 31));
    }
    bad = __syncthreads_or(bad);   // every key is read before any output is written (in place allowed)
    const uint32_t per = (words + kSmallThreads - 1) / kSmallThreads;
    const uint32_t lo = min(words, threadIdx.x * per), hi = min(words, lo + per);
    uint32_t c = 0;
    for (uint32_t w = lo; w < hi; ++w) c += __popc(bm[w]);
    uint32_t incl = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t v = wsum[lane];
        uint32_t s = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, s, d);
            if (lane >= d) s += y;
        }
        wsum[lane] = s - v;   // exclusive prefix of the warps
        if (lane == 31) {
            res->count = s;
            res->reserved = 0;
            res->status = bad ? BITSORT_ERR_KEY_RANGE : (s < n ? BITSORT_ERR_DUPLICATE : BITSORT_OK);
        }
    }
    __syncthreads();
    uint32_t o = wsum[warp] + incl - c;
    for (uint32_t w = lo; w < hi; ++w) {
        uint32_t bits = bm[w];
        while (bits) {
            const uint32_t b = __ffs(bits) - 1;
            out[o++] = (K)(w * 32u + b);
            bits &= bits - 1;
        }
    }
}

__global__ void narrow_kernel(const uint64_t *keys, uint64_t n, uint64_t maxv, uint32_t *dst, WideMisc *m) {
    bool bad = false, top = false;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t x = __ldcs(keys + i);
        const bool in = x <= maxv;
        bad |= !in;
        top |= x == 0xFFFFFFFFull;
        dst[i] = in ? (uint32_t)x : 0xFFFFFFFFu;
    }
    bad = __syncthreads_or(bad);
    top = __syncthreads_or(top);
    if (threadIdx.x == 0) {
        if (bad) atomicOr(&m->bad, 1u);
        if (top) atomicOr(&m->top, 1u);
    }
}

__global__ void widen_kernel(const uint32_t *src, uint64_t *out, uint64_t maxv, const WideMisc *m,
                             bitsort_result_t *res) {
    uint64_t count = m->inner.count;
    const bool bad = m->bad != 0;
    // a replaced key landed on the top value that no genuine key holds
    if (bad && maxv == 0xFFFFFFFFull && !m->top && count > 0 && src[count - 1] == 0xFFFFFFFFu) --count;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
        __stcs(out + i, (uint64_t)src[i]);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        uint32_t st = m->inner.status;
        if (bad && st != BITSORT_ERR_TIMEOUT) st = BITSORT_ERR_KEY_RANGE;
        res->count = count;
        res->reserved = 0;
        res->status = st;
    }
}

template <typename K>
bitsort_status_t small_sort(bitsort_ctx *c, const K *keys, uint64_t n, uint32_t max_value, K *out,
                            bitsort_result_t *d_result, cudaStream_t s) {
    if (!c) c = bsx_default_ctx();
    if (!c) return BITSORT_ERR_CUDA;
    if (n > (uint64_t)max_value + 1) return BITSORT_ERR_INVALID;   // keys cannot be distinct
    if (n > 0 && (!keys || !out)) return BITSORT_ERR_INVALID;
    if (((uintptr_t)keys % sizeof(K)) || ((uintptr_t)out % sizeof(K))) return BITSORT_ERR_INVALID;
    if (n > 0 && keys != out && bsx_ranges_overlap(keys, out, n * sizeof(K))) return BITSORT_ERR_INVALID;
    if (cudaSetDevice(c->device) != cudaSuccess) return BITSORT_ERR_CUDA;
    bitsort_result_t *res = d_result ? d_result : c->result;
    if (n == 0) return bsx_check(cudaMemsetAsync(res, 0, sizeof(bitsort_result_t), s));
    small_sort_kernel<K><<<1, kSmallThreads, 0, s>>>(keys, (uint32_t)n, max_value, out, res);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        bsx_note_error((int)e, "small-width sort launch");
        return BITSORT_ERR_CUDA;
    }
    c->launches.fetch_add(1);
    return BITSORT_OK;
}

}  // namespace

void bsx_widths_free(bitsort_ctx *c) {
    if (c->wide) cudaFree(c->wide);
    if (c->wide_misc) cudaFree(c->wide_misc);
    c->wide = nullptr;
    c->wide_misc = nullptr;
    c->wide_cap = 0;
}

extern "C" bitsort_status_t bitsort_u16(bitsort_ctx_t *c, const uint16_t *keys, uint64_t n, uint16_t max_value,
                                        uint16_t *out, bitsort_result_t *d_result, bitsort_stream_t stream) {
    bsx_range nvtx_range_("bitsort_u16");
    return small_sort<uint16_t>(c, keys, n, max_value, out, d_result, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" bitsort_status_t bitsort_u8(bitsort_ctx_t *c, const uint8_t *keys, uint64_t n, uint8_t max_value,
                                       uint8_t *out, bitsort_result_t *d_result, bitsort_stream_t stream) {
    bsx_range nvtx_range_("bitsort_u8");
    return small_sort<uint8_t>(c, keys, n, max_value, out, d_result, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" bitsort_status_t bitsort_u64(bitsort_ctx_t *c, const uint64_t *keys, uint64_t n, uint64_t max_value,
                                        uint64_t *out, bitsort_result_t *d_result, bitsort_stream_t stream) {
    bsx_range nvtx_range_("bitsort_u64");
    if (!c) c = bsx_default_ctx();
    if (!c) return BITSORT_ERR_CUDA;
    if (max_value > 0xFFFFFFFFull) return BITSORT_ERR_INVALID;
    if (n > max_value + 1) return BITSORT_ERR_INVALID;
    if (n > 0 && (!keys || !out)) return BITSORT_ERR_INVALID;
    if (((uintptr_t)keys & 7u) || ((uintptr_t)out & 7u)) return BITSORT_ERR_INVALID;
    if (n > 0 && keys != out && bsx_ranges_overlap(keys, out, n * sizeof(uint64_t))) return BITSORT_ERR_INVALID;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaSetDevice(c->device) != cudaSuccess) return BITSORT_ERR_CUDA;
    bitsort_result_t *res = d_result ? d_result : c->result;
    if (n == 0) return bsx_check(cudaMemsetAsync(res, 0, sizeof(bitsort_result_t), s));
    if (!c->wide_misc) {
        cudaError_t e = cudaMalloc(&c->wide_misc, sizeof(WideMisc));
        if (e != cudaSuccess) {
            c->wide_misc = nullptr;
            return bsx_check(e);
        }
    }
    if (c->wide_cap < n) {
        if (c->wide) {
            cudaDeviceSynchronize();
            cudaFree(c->wide);
            c->wide = nullptr;
            c->wide_cap = 0;
        }
        cudaError_t e = cudaMalloc(&c->wide, n * sizeof(uint32_t));
        if (e != cudaSuccess) {
            c->wide = nullptr;
            return bsx_check(e);
        }
        c->wide_cap = n;
    }
    WideMisc *m = reinterpret_cast<WideMisc *>(c->wide_misc);
    cudaError_t e = cudaMemsetAsync(m, 0, sizeof(WideMisc), s);
    if (e != cudaSuccess) return bsx_check(e);
    const int T = 256;
    const uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>((n + T - 1) / T, (uint64_t)c->sms * 8));
    narrow_kernel<<<(unsigned)grid, T, 0, s>>>(keys, n, max_value, c->wide, m);
    if ((e = cudaGetLastError()) != cudaSuccess) {
        bsx_note_error((int)e, "narrowing launch");
        return BITSORT_ERR_CUDA;
    }
    // the 32-bit sort of the narrowed keys, in place in the scratch copy
    bitsort_status_t st = bitsort_ex(c, c->wide, n, (uint32_t)max_value, c->wide, &m->inner, stream);
    if (st != BITSORT_OK) return st;
    widen_kernel<<<(unsigned)grid, T, 0, s>>>(c->wide, out, max_value, m, res);
    if ((e = cudaGetLastError()) != cudaSuccess) {
        bsx_note_error((int)e, "widening launch");
        return BITSORT_ERR_CUDA;
    }
    c->launches.fetch_add(2);
    return BITSORT_OK;
}
