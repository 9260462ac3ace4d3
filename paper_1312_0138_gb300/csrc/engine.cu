// engine.cu -- the sort kernels for sm_103a.
//
// The bitmap form of the paper's bitwise sort (Section V, Algorithm 1; result
// fixed by Theorem 1), split into work items (see engine.h): one persistent
// kernel runs every item type from a ticket counter in ascending order (one or
// many arrays), and one phase kernel per item type runs the phases of a single
// sort as separate launches.  Design points:
//   * keys stream through 128-bit loads with the streaming cache hint; the
//     head and tail of a range that is not 16-byte aligned are peeled;
//   * the bitmap of a bucket lives in shared memory, where the OR of a
//     shifted one (Table I, Example 2) is a native shared-memory atomic; a
//     sparse slice also keeps a summary bitmap of its non-empty words;
//   * the per-word popcount (Example 6) of a slice is summed per warp; a
//     partition-path slice starts its outputs at its bucket's known offset,
//     and only the global-bitmap path chains its slices by a decoupled
//     look-back (Merrill & Garland, "Single-pass Parallel Prefix Scan with
//     Decoupled Look-back", NVIDIA NVR-2016-002);
//   * set-bit positions are written ascending, bit 0 first inside a word
//     (Section II numbering), by neighbouring lanes (coalesced) or staged per
//     warp in shared memory and written in 16-byte stores (dense words);
//   * every wait on another CTA is bounded in time (%globaltimer) and in
//     iterations, and reports a timeout instead of hanging.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "engine.h"
#include "ptx.cuh"

namespace bsx {

constexpr unsigned kFull = 0xffffffffu;

// floor(x / S) = floor(x * magic / 2^64) with magic = ceil(2^64 / S).  For a
// 32-bit x the low half of the magic only contributes the high word of
// x * lo, a whole number (the fraction below it cannot carry): three integer
// instructions instead of a 64 x 64 multiply.
__device__ __forceinline__ uint32_t bucket_of(uint32_t x, uint64_t magic) {
    const uint64_t t = (uint64_t)x * (uint32_t)(magic >> 32) + __umulhi(x, (uint32_t)magic);
    return (uint32_t)(t >> 32);
}

__device__ __forceinline__ uint32_t warp_sum_u32(uint32_t v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
    return v;
}
__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
    return v;
}
__device__ __forceinline__ uint32_t warp_incl_scan_u32(uint32_t v, int lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, v, d);
        if (lane >= d) v += y;
    }
    return v;
}
__device__ __forceinline__ uint64_t warp_incl_scan_u64(uint64_t v, int lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint64_t y = __shfl_up_sync(kFull, v, d);
        if (lane >= d) v += y;
    }
    return v;
}

struct SharedMisc {
    uint64_t wsum[33];
    uint64_t excl;
    uint32_t wcount[32];
    uint32_t wbase[32];
    uint32_t ticket;
    uint32_t flag;
    uint32_t total;
    uint32_t summ_clean;   // the summary bitmap (start of shared memory) is all zero
    uint32_t bm_clean_w;   // the slice bitmap's first bm_clean_w words are zero
    uint64_t known;        // PARTITION: output offset of the slice's bucket (thread 0)
    uint64_t expect;       // PARTITION: keys the bucket received (thread 0)
    uint32_t defer;        // slices report their completion once per CTA, at the end of the kernel
    uint32_t done_local;   // slices this CTA finished while deferring (thread 0)
    uint32_t nonempty[32]; // slice groups: per warp, a ballot of the slices with keys
};

// Thread 0 only: wait until *p >= target.  Gives up (false) when the array's
// timeout flag is raised by another CTA, after `limit_ns` of wall time, or
// after an iteration cap that bounds the loop even if the timer misbehaves.
__device__ bool wait_geq(const uint32_t *p, uint32_t target, const uint32_t *timeout_flag, uint64_t limit_ns) {
    if (ld_acquire_u32(p) >= target) return true;
    WaitClock clk;
    clk.start();
    const uint64_t cap = limit_ns / 16 + 4096;
    uint32_t sleep = 32;
    for (uint64_t it = 0; it < cap; ++it) {
        __nanosleep(sleep);
        if (sleep < 2048) sleep <<= 1;
        if (ld_acquire_u32(p) >= target) return true;
        if ((it & 7) == 7) {
            if (ld_acquire_u32(timeout_flag) != 0) return false;
            if (clk.expired(limit_ns)) return false;
        }
    }
    return false;
}

// Exclusive prefix sums of load(0..nb) passed to store(i, prefix); returns
// the total.  Every thread of the block must call it.
template <int T, class Load, class Store>
__device__ uint64_t block_exclusive_scan(uint32_t nb, Load load, Store store, SharedMisc &m) {
    constexpr int NW = T / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t per = (nb + T - 1) / T;
    const uint32_t lo = min(nb, threadIdx.x * per), hi = min(nb, lo + per);
    uint64_t s = 0;
    for (uint32_t i = lo; i < hi; ++i) s += load(i);
    const uint64_t incl = warp_incl_scan_u64(s, lane);
    if (lane == 31) m.wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint64_t w = lane < NW ? m.wsum[lane] : 0;
        const uint64_t wi = warp_incl_scan_u64(w, lane);
        if (lane < NW) m.wsum[lane] = wi - w;
        if (lane == 31) m.wsum[32] = wi;
    }
    __syncthreads();
    uint64_t run = m.wsum[warp] + incl - s;
    for (uint32_t i = lo; i < hi; ++i) {
        const uint64_t c = load(i);
        store(i, run);
        run += c;
    }
    const uint64_t total = m.wsum[32];
    __syncthreads();
    return total;
}

// Exclusive prefix sums of the 32-bit counts c[0..nb) written to e[0..nb),
// in place allowed (e == c); returns the total.  Every thread must call it.
template <int T>
__device__ uint32_t block_exclusive_scan_u32(uint32_t nb, const uint32_t *c, uint32_t *e, SharedMisc &m) {
    constexpr int NW = T / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t per = (nb + T - 1) / T;
    const uint32_t lo = min(nb, threadIdx.x * per), hi = min(nb, lo + per);
    uint32_t s = 0;
    for (uint32_t i = lo; i < hi; ++i) s += c[i];
    const uint32_t incl = warp_incl_scan_u32(s, lane);
    if (lane == 31) m.wcount[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < NW ? m.wcount[lane] : 0;
        const uint32_t wi = warp_incl_scan_u32(w, lane);
        if (lane < NW) m.wbase[lane] = wi - w;
        if (lane == 31) m.total = wi;
    }
    __syncthreads();
    uint32_t run = m.wbase[warp] + incl - s;
    for (uint32_t i = lo; i < hi; ++i) {
        const uint32_t v = c[i];
        e[i] = run;
        run += v;
    }
    const uint32_t total = m.total;
    __syncthreads();
    return total;
}

// Calls f(key) for every key of p[lo, hi): 128-bit streaming loads for the
// 16-byte aligned body, scalar loads for the peeled head and tail.
template <int T, bool kStream, int U = 8, class F>
__device__ __forceinline__ void for_each_key(const uint32_t *p, uint64_t lo, uint64_t hi, F &&f) {
    if (lo >= hi) return;
    const uint32_t mis = (uint32_t)((reinterpret_cast<uintptr_t>(p + lo) & 15u) >> 2);
    uint64_t head = mis ? 4u - mis : 0u;
    if (head > hi - lo) head = hi - lo;
    if (threadIdx.x < head) f(kStream ? __ldcs(p + lo + threadIdx.x) : __ldcg(p + lo + threadIdx.x));
    const uint64_t b0 = lo + head;
    const uint64_t nv = (hi - b0) >> 2;
    const uint4 *v = reinterpret_cast<const uint4 *>(p + b0);
    uint64_t i = threadIdx.x;
    for (; i + (U - 1) * (uint64_t)T < nv; i += U * (uint64_t)T) {
        uint4 q[U];
#pragma unroll
        for (int u = 0; u < U; ++u) q[u] = kStream ? __ldcs(v + i + u * T) : __ldcg(v + i + u * T);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            f(q[u].x);
            f(q[u].y);
            f(q[u].z);
            f(q[u].w);
        }
    }
    for (; i < nv; i += T) {
        const uint4 q = kStream ? __ldcs(v + i) : __ldcg(v + i);
        f(q.x);
        f(q.y);
        f(q.z);
        f(q.w);
    }
    const uint64_t t0 = b0 + (nv << 2);
    if (t0 + threadIdx.x < hi) f(kStream ? __ldcs(p + t0 + threadIdx.x) : __ldcg(p + t0 + threadIdx.x));
}

// ------------------------------------------------------------- look-back
// Warp 0 of the CTA that owns slice s: publish the slice's own count, add up
// the counts of the slices before it (stopping at the nearest published
// inclusive prefix), publish the inclusive prefix and return the exclusive
// one.  Bounded: on timeout the array's timeout flag is raised and 0 is used.
__device__ uint64_t lookback(const EngineParams &P, const ArrayDesc &a, uint32_t s, uint32_t agg, int lane) {
    uint64_t *look = a.look;
    if (s == 0) {
        if (lane == 0) st_release_u64(&look[0], LB_PREFIX | agg);
        return 0;
    }
    if (lane == 0) st_release_u64(&look[s], LB_AGG | agg);
    uint64_t excl = 0;
    int64_t j = (int64_t)s - 1;
    bool expired = false;
    WaitClock clk;
    uint64_t iters = 0;
    const uint64_t cap = P.wait_limit_ns / 16 + 4096;
    while (true) {
        const int64_t idx = j - lane;
        uint64_t v = idx >= 0 ? ld_acquire_u64(&look[idx]) : LB_PREFIX;
        while (__any_sync(kFull, (v >> 62) == 0)) {
            if (iters == 0) clk.start();
            ++iters;
            if ((iters & 7) == 0) {
                bool stop = false;
                if (lane == 0)
                    stop = iters > cap || clk.expired(P.wait_limit_ns) ||
                           ld_acquire_u32(&a.sync[SY_TIMEOUT]) != 0;
                if (__shfl_sync(kFull, stop ? 1 : 0, 0)) {
                    expired = true;
                    break;
                }
            }
            __nanosleep(64);
            if ((v >> 62) == 0) v = ld_acquire_u64(&look[idx]);
        }
        if (expired) break;
        const unsigned pmask = __ballot_sync(kFull, (v >> 62) == 2);
        uint64_t val = v & LB_VALUE;
        if (pmask) {
            const int first = __ffs(pmask) - 1;  // nearest slice with a prefix
            if (lane > first) val = 0;
            excl += warp_sum_u64(val);
            break;
        }
        excl += warp_sum_u64(val);
        j -= 32;
    }
    if (expired) {
        if (lane == 0) atomicOr(&a.sync[SY_TIMEOUT], 1u);
        excl = 0;
    }
    if (lane == 0) st_release_u64(&look[s], LB_PREFIX | (excl + agg));
    return excl;
}

// Writes the set-bit positions of bm[w0, w1) in ascending order to
// out[base ...]: value = v0 + 32*word + bit (Section II numbering, bit 0
// first).  A warp step covers U groups of 32 consecutive words; lane l holds
// word l of every group, so neighbouring lanes write neighbouring outputs
// (coalesced stores), and the U warp-wide prefix sums that place the lanes'
// outputs are independent, which hides their shuffle latency.  Each lane
// writes the four lowest set bits of a word with predicated stores; only
// words with more set bits walk the rest.
template <int U>
__device__ __forceinline__ void emit_words(const uint32_t *bm, uint32_t w0, uint32_t w1, uint32_t v0, uint64_t base,
                                           uint32_t *out, uint64_t lim) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;   // lanes below this one
    for (uint32_t i0 = w0; i0 < w1; i0 += 32 * U) {
        uint32_t v[U], c[U], incl[U];
        bool single = true;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t i = i0 + u * 32 + lane;
            v[u] = i < w1 ? bm[i] : 0u;
            c[u] = __popc(v[u]);
            incl[u] = c[u];
            single &= c[u] <= 1u;
        }
        if (__all_sync(kFull, single)) {
            // sparse step: no word holds more than one set bit, so a lane's
            // output index is the number of non-empty words below it
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t nz = __ballot_sync(kFull, v[u] != 0);
                const uint64_t o = base + __popc(nz & lt);
                if (v[u] && o < lim) __stcs(out + o, v0 + (i0 + u * 32 + lane) * 32u + (__ffs(v[u]) - 1));
                base += __popc(nz);
            }
            continue;
        }
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t y = __shfl_up_sync(kFull, incl[u], d);
                if (lane >= d) incl[u] += y;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t chunk = __shfl_sync(kFull, incl[u], 31);
            const uint32_t pos = incl[u] - c[u];
            const uint32_t val = v0 + (i0 + u * 32 + lane) * 32u - 1u;
            uint32_t x = v[u];
            if (base + chunk <= lim) {   // warp-uniform: the step lies inside out[0, n)
                uint32_t *d = out + base + pos;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (c[u] > (uint32_t)j) __stcs(d + j, val + __ffs(x));
                    x &= x - 1;
                }
                if (__any_sync(kFull, x != 0)) {
                    d += 4;
                    while (x) {
                        __stcs(d++, val + __ffs(x));
                        x &= x - 1;
                    }
                }
            } else {
                uint64_t o = base + pos;
                while (x) {
                    if (o < lim) __stcs(out + o, val + __ffs(x));   // never past n, whatever the scratch held
                    ++o;
                    x &= x - 1;
                }
            }
            base += chunk;
        }
    }
}

// Staged emission: the set-bit positions of many consecutive steps gather in
// a per-warp shared-memory buffer whose index matches the output address
// modulo 16 bytes; a full buffer leaves as 16-byte vector stores of whole
// 128-byte lines (a scalar head and tail around them).  Far fewer, fuller L2
// write requests than storing each step's handful of positions.
// Index of the highest set bit of x (x != 0).
__device__ __forceinline__ uint32_t bit_high(uint32_t x) {
    uint32_t p;
    asm("bfind.u32 %0, %1;" : "=r"(p) : "r"(x));
    return p;
}

__device__ __forceinline__ void stage_flush(const uint32_t *stage, uint32_t s0, uint32_t fill, uint32_t *out,
                                            uint64_t g0, uint64_t lim) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    uint32_t head = (4u - s0) & 3u;
    if (head > fill) head = fill;
    if ((uint32_t)lane < head && g0 + lane < lim) __stcs(out + g0 + lane, stage[s0 + lane]);
    const uint32_t nvec = (fill - head) >> 2;
    const uint32_t sb = s0 + head;
    const uint64_t gb = g0 + head;
    if (gb + 4ull * nvec <= lim) {
        const uint4 *src = reinterpret_cast<const uint4 *>(stage + sb);
        uint4 *dst = reinterpret_cast<uint4 *>(out + gb);
        for (uint32_t k = lane; k < nvec; k += 32) __stcs(dst + k, src[k]);
    } else {
        for (uint32_t k = lane; k < 4 * nvec; k += 32)
            if (gb + k < lim) __stcs(out + gb + k, stage[sb + k]);
    }
    const uint32_t t0 = head + 4 * nvec;
    if ((uint32_t)lane < fill - t0 && g0 + t0 + lane < lim) __stcs(out + g0 + t0 + lane, stage[s0 + t0 + lane]);
    __syncwarp();
}

__device__ __forceinline__ void emit_words_staged(const uint32_t *bm, uint32_t w0, uint32_t w1, uint32_t v0,
                                                  uint64_t base, uint32_t *out, uint64_t lim, uint32_t *stage,
                                                  uint32_t cap) {
    const int lane = threadIdx.x & 31;
    const uintptr_t out_addr = reinterpret_cast<uintptr_t>(out);
    uint64_t g0 = base;
    uint32_t s0 = (uint32_t)(((out_addr >> 2) + g0) & 3);
    uint32_t fill = 0;
    for (uint32_t i0 = w0; i0 < w1; i0 += 32) {
        const uint32_t i = i0 + lane;
        const uint32_t v = i < w1 ? bm[i] : 0u;
        const uint32_t c = __popc(v);
        const uint32_t incl = warp_incl_scan_u32(c, lane);
        const uint32_t chunk = __shfl_sync(kFull, incl, 31);
        const uint32_t pos = incl - c;
        if (s0 + fill + chunk > cap) {   // warp-uniform: flush before this step
            stage_flush(stage, s0, fill, out, g0, lim);
            g0 += fill;
            fill = 0;
            s0 = (uint32_t)(((out_addr >> 2) + g0) & 3);
        }
        const uint32_t val = v0 + i * 32u - 1u;
        uint32_t x = v;
        if (s0 + chunk <= cap) {
            // the highest set bit first, into the word's last slot: one bfind
            // and one clear per bit, stores at fixed offsets from e, sixteen
            // slots unrolled (dense words: 16 set bits on average at density
            // 1/2; c2a's bucket phase 4.44 -> 4.36 ms against the lowest-bit
            // walk with four unrolled slots)
            uint32_t *e = stage + s0 + fill + pos + c - 1;
            const uint32_t vb = val + 1u;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                if (c > (uint32_t)j) {
                    const uint32_t p = bit_high(x);
                    e[-j] = vb + p;
                    x ^= 1u << p;
                }
            }
            if (__any_sync(kFull, c > 16u)) {
                for (int j = 16; x; ++j) {
                    const uint32_t p = bit_high(x);
                    e[-j] = vb + p;
                    x ^= 1u << p;
                }
            }
            fill += chunk;
        } else {
            // one step with more positions than the buffer holds (near-full
            // words): store it directly
            uint64_t o = g0 + pos;
            while (x) {
                if (o < lim) __stcs(out + o, val + __ffs(x));
                ++o;
                x &= x - 1;
            }
            g0 += chunk;
            s0 = (uint32_t)(((out_addr >> 2) + g0) & 3);
        }
    }
    stage_flush(stage, s0, fill, out, g0, lim);
}

// Staged emission with runs: every lane takes WPL consecutive words, so one
// warp-wide scan places 32*WPL words, and a lane walks the set bits of its run
// in one loop (reading its next word from shared memory when the current one
// is exhausted).  Positions gather in the per-warp buffer and leave through
// stage_flush.  A step with more positions than the buffer holds (dense
// words) is written directly.
template <int WPL>
__device__ __forceinline__ void emit_runs_staged(const uint32_t *bm, uint32_t w0, uint32_t w1, uint32_t v0,
                                                 uint64_t base, uint32_t *out, uint64_t lim, uint32_t *stage,
                                                 uint32_t cap) {
    const int lane = threadIdx.x & 31;
    const uintptr_t out_addr = reinterpret_cast<uintptr_t>(out);
    uint64_t g0 = base;
    uint32_t s0 = (uint32_t)(((out_addr >> 2) + g0) & 3);
    uint32_t fill = 0;
    for (uint32_t i0 = w0; i0 < w1; i0 += 32 * WPL) {
        const uint32_t i = i0 + lane * WPL;
        uint32_t c = 0;
#pragma unroll
        for (int k = 0; k < WPL; k += 4) {
            if (i + k < w1) {
                const uint4 q = *reinterpret_cast<const uint4 *>(bm + i + k);
                c += __popc(q.x) + __popc(q.y) + __popc(q.z) + __popc(q.w);
            }
        }
        const uint32_t incl = warp_incl_scan_u32(c, lane);
        const uint32_t chunk = __shfl_sync(kFull, incl, 31);
        const uint32_t pos = incl - c;
        if (s0 + fill + chunk > cap) {   // warp-uniform
            stage_flush(stage, s0, fill, out, g0, lim);
            g0 += fill;
            fill = 0;
            s0 = (uint32_t)(((out_addr >> 2) + g0) & 3);
        }
        uint32_t k = 0;
        uint32_t x = (c && i < w1) ? bm[i] : 0u;
        uint32_t val = v0 + i * 32u - 1u;
        uint32_t left = c;
        if (s0 + chunk <= cap) {
            uint32_t *d = stage + s0 + fill + pos;
            while (left) {
                if (x) {
                    *d++ = val + __ffs(x);
                    x &= x - 1;
                    --left;
                } else {
                    ++k;
                    x = bm[i + k];   // left > 0: a set bit lies ahead inside the run
                    val += 32u;
                }
            }
            fill += chunk;
        } else {
            uint64_t o = g0 + fill + pos;   // fill == 0 here: the buffer was just flushed
            while (left) {
                if (x) {
                    if (o < lim) __stcs(out + o, val + __ffs(x));
                    ++o;
                    x &= x - 1;
                    --left;
                } else {
                    ++k;
                    x = bm[i + k];
                    val += 32u;
                }
            }
            g0 += chunk;
            s0 = (uint32_t)(((out_addr >> 2) + g0) & 3);
        }
    }
    stage_flush(stage, s0, fill, out, g0, lim);
}

template <int WPL>
__device__ __forceinline__ uint32_t count_words(const uint32_t *bm, uint32_t w0, uint32_t w1) {
    const int lane = threadIdx.x & 31;
    uint32_t c = 0;
    for (uint32_t i = w0 + lane * WPL; i < w1; i += 32 * WPL) {
        if constexpr (WPL == 4) {
            const uint4 q = *reinterpret_cast<const uint4 *>(bm + i);
            c += __popc(q.x) + __popc(q.y) + __popc(q.z) + __popc(q.w);
        } else if constexpr (WPL == 2) {
            const uint2 q = *reinterpret_cast<const uint2 *>(bm + i);
            c += __popc(q.x) + __popc(q.y);
        } else {
            c += __popc(bm[i]);
        }
    }
    return warp_sum_u32(c);
}

// Count the set bits of one slice (per warp range, then the block), get the
// number of set bits of all earlier slices by look-back, and leave in shared
// memory: m.excl (first output index of the slice), m.total (its set bits),
// m.wbase[w] (set bits before warp w's range).  Returns the warp's range.
// The partition path knows where each bucket's outputs start: with distinct
// keys, a bucket's set bits equal its key count, so the slice starts at the
// bucket's histogram offset (EXACT layout) or at the sum of the fill counts
// of the buckets before it (CAPACITY layout), computed by the slice's
// thread 0 into m.known / m.expect.  The slice records (start, count) in its
// look-back word for the array's last CTA; one whose count falls short of
// its bucket's keys (repeated keys) raises the mismatch flag, and the last
// CTA then closes the gaps (slice_complete).  Without a partition (GLOBAL
// path) the slices chain through the decoupled look-back.
__device__ __forceinline__ bool known_offsets(const ArrayDesc &a) {
    return a.path == BITSORT_PATH_PARTITION && a.nslices > 1;
}

// Called by warp 0 of the CTA that owns slice s (lane 0 reads m.known).
__device__ uint64_t slice_offset(const EngineParams &P, const ArrayDesc &a, uint32_t s, uint32_t total, int lane,
                                 const SharedMisc &m) {
    if (known_offsets(a)) {
        if (lane == 0) {
            a.look[s] = (m.known << 32) | total;
            if (total != m.expect) atomicOr(&a.sync[SY_MISMATCH], 1u);
        }
        return m.known;
    }
    return a.nslices > 1 ? lookback(P, a, s, total, lane) : 0;
}

template <int T>
__device__ void slice_count(const EngineParams &P, const ArrayDesc &a, uint32_t s, const uint32_t *bm,
                            uint32_t words, uint32_t wpl, uint32_t &w0, uint32_t &w1, SharedMisc &m,
                            bool with_lookback = true) {
    constexpr int NW = T / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // warp ranges are whole multiples of 32 * max(wpl, 4) words: every
    // emitter's steps fit, and the count reads 4 words per lane
    const uint32_t step = 32u * max(wpl, 4u);
    const uint32_t wpw = (((words + NW - 1) / NW) + step - 1) / step * step;
    w0 = min(words, (uint32_t)warp * wpw);
    w1 = min(words, w0 + wpw);
    const uint32_t cnt = count_words<4>(bm, w0, w1);
    if (lane == 0) m.wcount[warp] = cnt;
    __syncthreads();
    if (warp == 0) {
        const uint32_t c = lane < NW ? m.wcount[lane] : 0;
        const uint32_t incl = warp_incl_scan_u32(c, lane);
        if (lane < NW) m.wbase[lane] = incl - c;
        const uint32_t total = __shfl_sync(kFull, incl, 31);
        uint64_t excl = 0;
        if (with_lookback) excl = slice_offset(P, a, s, total, lane, m);
        if (lane == 0) {
            m.excl = excl;
            m.total = total;
        }
    }
    __syncthreads();
}

// Look-back of slice s alone (its own count already in m.total).
template <int T>
__device__ void slice_lookback(const EngineParams &P, const ArrayDesc &a, uint32_t s, SharedMisc &m) {
    if (threadIdx.x < 32) {
        const uint64_t excl = slice_offset(P, a, s, m.total, threadIdx.x, m);
        if (threadIdx.x == 0) m.excl = excl;
    }
    __syncthreads();
}

// The CTA that finishes the array's last slice writes the outcome and
// returns the array's scratch to its zero state for the next launch.  On the
// partition path it also sums the slices' counts and, if some slice held
// fewer set bits than its bucket had keys (repeated keys), moves every
// slice's outputs down, in slice order, to close the gaps: each chunk of T
// values is read whole before it is written, and a slice never moves up.
// `count` slices are reported at once (a CTA that deferred its slices'
// reports to the end of the kernel); a CTA with nothing to report must not
// call it.
template <int T>
__device__ void complete_slices(const ArrayDesc &a, SharedMisc &m, uint32_t count) {
    // the barrier orders the block's writes before thread 0's fence, which
    // makes them visible device-wide before the completion count (and, for
    // the last CTA, the count before its reads)
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t d = atomicAdd(&a.sync[SY_SLICES_DONE], count);
        m.flag = (d + count == a.nslices) ? 1u : 0u;
        if (m.flag) __threadfence();
    }
    __syncthreads();
    if (!m.flag) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t total = m.total;
    if (known_offsets(a)) {
        uint64_t part = 0;
        for (uint32_t i = threadIdx.x; i < a.nslices; i += T) part += (uint32_t)__ldcg(&a.look[i]);
        part = warp_sum_u64(part);
        if (lane == 0) m.wsum[warp] = part;
        __syncthreads();
        total = 0;
        for (int w = 0; w < T / 32; ++w) total += m.wsum[w];
        const bool gaps = ld_acquire_u32(&a.sync[SY_MISMATCH]) != 0 && ld_acquire_u32(&a.sync[SY_TIMEOUT]) == 0;
        if (gaps) {
            uint32_t *out = a.out;
            uint64_t dst = 0;
            for (uint32_t i = 0; i < a.nslices; ++i) {
                const uint64_t v = __ldcg(&a.look[i]);
                const uint64_t src = v >> 32, cnt = (uint32_t)v;
                if (src != dst) {
                    for (uint64_t k = 0; k < cnt; k += T) {
                        const uint64_t j = k + threadIdx.x;
                        const uint32_t x = j < cnt ? __ldcg(out + src + j) : 0u;
                        __syncthreads();
                        if (j < cnt) out[dst + j] = x;
                        __syncthreads();
                    }
                }
                dst += cnt;
            }
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < a.nslices; i += T) {
            a.look[i] = 0;
            a.cursor[i] = 0;
        }
    } else {
        if (a.nslices > 1) total = ld_acquire_u64(&a.look[a.nslices - 1]) & LB_VALUE;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < a.nslices && a.nslices > 1; i += T) a.look[i] = 0;
    }
    if (threadIdx.x == 0) {
        uint32_t st = BITSORT_OK;
        if (ld_acquire_u32(&a.sync[SY_TIMEOUT]) != 0) st = BITSORT_ERR_TIMEOUT;
        else if (ld_acquire_u32(&a.sync[SY_RANGE]) != 0) st = BITSORT_ERR_KEY_RANGE;
        else if (total < a.n) st = BITSORT_ERR_DUPLICATE;
        a.result->status = st;
        a.result->reserved = 0;
        a.result->count = total;
        for (int k = 0; k < SY_COUNT; ++k) a.sync[k] = 0;
    }
}

// End of one slice: report it now, or count it for the CTA's report at the
// end of the kernel (m.defer).
template <int T>
__device__ void slice_complete(const ArrayDesc &a, SharedMisc &m) {
    if (m.defer) {
        __syncthreads();
        if (threadIdx.x == 0) ++m.done_local;
        return;
    }
    complete_slices<T>(a, m, 1u);
}

// Count, look back and write out one bitmap slice held in shared memory by
// walking its words (EMIT_WORD).  `bm` holds `words` words covering the
// values v0 .. v0 + 32*words - 1 and is zero from `words` up to the next
// multiple of 4.
template <int T>
__device__ void slice_finish(const EngineParams &P, const ArrayDesc &a, uint32_t s, const uint32_t *bm,
                             uint32_t words, uint32_t v0, uint32_t *stage_all, SharedMisc &m) {
    const int warp = threadIdx.x >> 5;
    const uint32_t wpl = a.wpl;
    uint32_t w0, w1;
    slice_count<T>(P, a, s, bm, words, wpl, w0, w1, m);
    const uint64_t base = m.excl + m.wbase[warp];
    constexpr uint32_t SW = stage_words(T);
    uint32_t *stage = stage_all + warp * SW;
    if (a.stage && wpl == 8) emit_runs_staged<8>(bm, w0, w1, v0, base, a.out, a.n, stage, SW);
    else if (a.stage && wpl == 4) emit_runs_staged<4>(bm, w0, w1, v0, base, a.out, a.n, stage, SW);
    else if (a.stage) emit_words_staged(bm, w0, w1, v0, base, a.out, a.n, stage, SW);
    else if (wpl == 4) emit_words<4>(bm, w0, w1, v0, base, a.out, a.n);
    else if (wpl == 2) emit_words<2>(bm, w0, w1, v0, base, a.out, a.n);
    else emit_words<1>(bm, w0, w1, v0, base, a.out, a.n);
    slice_complete<T>(a, m);
}

// ------------------------------------------------------------------ items
// Shared part of HIST: add the buckets of p[lo, hi) to the shared histogram
// (keys above max_value are only reported), then add it to the global counts.
// Returns true in the CTA that completed the last of `expected` contributions;
// that CTA then turns the counts into bucket offsets.
template <int T>
__device__ void hist_range(const ArrayDesc &a, uint64_t lo, uint64_t hi, uint32_t expected, char *smem,
                           SharedMisc &m) {
    const uint32_t nb = a.nslices;
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem);
    for (uint32_t i = threadIdx.x; i < nb; i += T) hist[i] = 0;
    __syncthreads();
    bool bad = false;
    const uint64_t M = a.M, magic = a.div_magic;
    const uint32_t bias = a.bias;
    for_each_key<T, false>(a.keys, lo, hi, [&](uint32_t x) {
        const uint32_t y = x - bias;
        if ((uint64_t)y < M) atomicAdd(&hist[bucket_of(y, magic)], 1u);
        else bad = true;
    });
    bad = __syncthreads_or(bad);
    if (bad && threadIdx.x == 0) atomicOr(&a.sync[SY_RANGE], 1u);
    for (uint32_t i = threadIdx.x; i < nb; i += T) {
        const uint32_t c = hist[i];
        if (c) atomicAdd(&a.counts[i], c);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t d = atomicAdd(&a.sync[SY_HIST_DONE], 1u);
        m.flag = (d == expected - 1) ? 1u : 0u;
        if (m.flag) __threadfence();
    }
    __syncthreads();
    if (m.flag) {
        block_exclusive_scan<T>(
            nb, [&](uint32_t i) -> uint64_t { return __ldcg(&a.counts[i]); },
            [&](uint32_t i, uint64_t v) { a.offsets[i] = v; }, m);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            st_release_u32(&a.sync[SY_OFFSETS_READY], 1u);
        }
    }
}

template <int T>
__device__ void item_hist(const EngineParams &P, const ArrayDesc &a, uint32_t tile, char *smem, SharedMisc &m) {
    const uint64_t lo = (uint64_t)tile * a.tile_keys;
    hist_range<T>(a, lo, min(lo + a.tile_keys, a.n), a.key_tiles, smem, m);
}

// PART: move the keys of one tile to their buckets' runs of the partition
// buffer.  Every key's bucket and rank inside the tile come from one shared
// atomic; the tile is then reordered by bucket in shared memory so that each
// bucket's run leaves in consecutive stores.  Keys above max_value go to an
// extra discard bin (index nslices) that is never written.  Positions are
// 32-bit (the buffer has at most 2^32 entries): run start minus the tile-local
// prefix is kept per bin (delta), so a key's position is delta[b] + its index
// in the reordered tile; lim[b] ends the part of the run that fits.
//
// part_tile() does everything after the keys are in registers: x[j] holds
// tile element j*T + threadIdx.x (valid while that index < nkeys).  `sorted`
// may be the buffer the keys came from: it is written only after a barrier
// that follows every thread's reads.
template <int T>
__device__ void part_tile(const ArrayDesc &a, const uint32_t (&x)[kKeysPerThread], uint32_t nkeys, uint32_t *hist,
                          uint32_t *delta, uint32_t *lim, uint32_t *sorted, uint16_t *sorted_b, SharedMisc &m) {
    constexpr int K = kKeysPerThread;
    const uint32_t nb = a.nslices;
    const uint32_t nbins = nb + 1;
    const bool capacity = a.layout == LAYOUT_CAPACITY;
    const uint64_t magic = a.div_magic;
    const uint32_t maxv = (uint32_t)(a.M - 1);
    const uint32_t bias = a.bias;   // keys are classified as x - bias; the buffer keeps x
    uint32_t br[K];   // bin << 16 | rank in the tile
    bool bad = false;
    if (nkeys == (uint32_t)a.tile_keys) {
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const uint32_t y = x[j] - bias;
            const bool in = y <= maxv;
            bad |= !in;
            const uint32_t bin = in ? bucket_of(y, magic) : nb;
            br[j] = (bin << 16) | atomicAdd(&hist[bin], 1u);
        }
    } else {
#pragma unroll
        for (int j = 0; j < K; ++j) {
            br[j] = 0xFFFFFFFFu;
            if ((uint32_t)j * T + threadIdx.x < nkeys) {
                const uint32_t y = x[j] - bias;
                const bool in = y <= maxv;
                bad |= !in;
                const uint32_t bin = in ? bucket_of(y, magic) : nb;
                br[j] = (bin << 16) | atomicAdd(&hist[bin], 1u);
            }
        }
    }
    if (capacity) {
        bad = __syncthreads_or(bad);
        if (bad && threadIdx.x == 0) atomicOr(&a.sync[SY_RANGE], 1u);
    } else {
        __syncthreads();   // (the histogram pass reports keys above max_value)
    }
    // reserve each bucket's run (needs the counts), then turn counts into
    // prefixes.  A thread owns up to kReserve bins per round and issues
    // their global atomics (and offset loads) before it uses any result, so
    // a wide fan-out waits for one atomic round trip per round, not per bin.
    constexpr int kReserve = 4;
    for (uint32_t r0 = 0; r0 < nbins; r0 += kReserve * T) {
        uint32_t cnt[kReserve], at[kReserve];
#pragma unroll
        for (int u = 0; u < kReserve; ++u) {
            const uint32_t i = r0 + u * T + threadIdx.x;
            cnt[u] = i < nb ? hist[i] : 0u;
        }
#pragma unroll
        for (int u = 0; u < kReserve; ++u)
            at[u] = cnt[u] ? atomicAdd(&a.cursor[r0 + u * T + threadIdx.x], cnt[u]) : 0u;
        uint64_t off[kReserve];
#pragma unroll
        for (int u = 0; u < kReserve; ++u)
            off[u] = (!capacity && cnt[u]) ? __ldcg(&a.offsets[r0 + u * T + threadIdx.x]) : 0ull;
#pragma unroll
        for (int u = 0; u < kReserve; ++u) {
            const uint32_t i = r0 + u * T + threadIdx.x;
            if (i >= nbins) break;
            const uint32_t c = cnt[u];
            uint32_t start = 0, fit = 0;
            if (c) {
                if (capacity) {
                    const uint64_t cap = a.cap;
                    start = (uint32_t)((uint64_t)i * cap + at[u]);
                    fit = at[u] >= cap ? 0u : (uint32_t)min((uint64_t)c, cap - at[u]);
                    if (fit < c) atomicOr(&a.sync[SY_OVERFLOW], 1u);   // only with repeated keys
                } else {
                    const uint64_t st = off[u] + at[u];
                    start = (uint32_t)st;
                    fit = st >= a.n ? 0u : (uint32_t)min((uint64_t)c, a.n - st);   // a sane scratch never clips
                }
            }
            delta[i] = start;
            lim[i] = fit;
        }
    }
    block_exclusive_scan_u32<T>(nbins, hist, hist, m);
    for (uint32_t i = threadIdx.x; i < nbins; i += T) {
        const uint32_t p = hist[i];
        delta[i] -= p;   // position = delta + index in the reordered tile (mod 2^32)
        lim[i] += p;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < K; ++j) {
        if (br[j] != 0xFFFFFFFFu) {
            const uint32_t bin = br[j] >> 16;
            const uint32_t at = hist[bin] + (br[j] & 0xFFFFu);
            sorted[at] = x[j];
            sorted_b[at] = (uint16_t)bin;
        }
    }
    __syncthreads();
    uint32_t *part = a.part;
#pragma unroll 4
    for (uint32_t i = threadIdx.x; i < nkeys; i += T) {
        const uint32_t bin = sorted_b[i];
        if (i < lim[bin]) part[delta[bin] + i] = sorted[i];
    }
}

template <int T>
__device__ void item_part(const EngineParams &P, const ArrayDesc &a, uint32_t tile, char *smem, SharedMisc &m) {
    constexpr int K = kKeysPerThread;
    const uint32_t nb = a.nslices;
    const uint32_t nbins = nb + 1;
    const bool capacity = a.layout == LAYOUT_CAPACITY;
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem);   // counts, then the tile-local exclusive prefix
    uint32_t *delta = hist + nbins;
    uint32_t *lim = delta + nbins;
    uint32_t *sorted = lim + nbins;
    uint16_t *sorted_b = reinterpret_cast<uint16_t *>(sorted + a.tile_keys);

    if (threadIdx.x == 0) {
        m.flag = 1u;
        if (!capacity && !a.phased)
            m.flag = wait_geq(&a.sync[SY_OFFSETS_READY], 1u, &a.sync[SY_TIMEOUT], P.wait_limit_ns) ? 1u : 0u;
    }
    for (uint32_t i = threadIdx.x; i < nbins; i += T) hist[i] = 0;
    __syncthreads();
    if (!m.flag) {
        if (threadIdx.x == 0) atomicOr(&a.sync[SY_TIMEOUT], 1u);
    } else {
        const uint64_t lo = (uint64_t)tile * a.tile_keys;
        const uint64_t hi = min(lo + a.tile_keys, a.n);
        const uint32_t nkeys = (uint32_t)(hi - lo);
        uint32_t x[K];
        if (nkeys == (uint32_t)a.tile_keys && (reinterpret_cast<uintptr_t>(a.keys) & 15u) == 0) {
            // full tile: K keys per thread, 128-bit loads
            const uint4 *src = reinterpret_cast<const uint4 *>(a.keys + lo);
#pragma unroll
            for (int j = 0; j < K / 4; ++j) {
                const uint4 q = __ldcs(src + j * T + threadIdx.x);
                x[4 * j] = q.x; x[4 * j + 1] = q.y; x[4 * j + 2] = q.z; x[4 * j + 3] = q.w;
            }
            // element order j*T + tid inside the tile is a permutation of the
            // (4*(j'*T + tid) + r) load order; ranks only need some order
        } else {
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const uint32_t e = (uint32_t)j * T + threadIdx.x;
                x[j] = e < nkeys ? __ldcs(a.keys + lo + e) : 0u;
            }
        }
        part_tile<T>(a, x, nkeys, hist, delta, lim, sorted, sorted_b, m);
    }
    if (!a.phased) {
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&a.sync[SY_PART_DONE], 1u);
        }
    }
}

// ------------------------------------------------- PART, phase kernel
// The partition phase of a single sort (the persistent engine and the
// streaming partition use item_part / part_stream above).  A CTA takes tiles
// t, t + G, ...; per tile:
//   1. every key's bin and its rank among the tile's keys of that bin come
//      from one shared-memory atomic;
//   2. each thread owns a contiguous range of bins: it issues the global
//      reservations of its bins' runs (an atomic on the bucket's cursor) at
//      once, and uses their results only in the second pass of the scan, so
//      that their round trip overlaps the scan's first pass and barriers;
//   3. that second pass writes the tile-local prefix of every bin and its run
//      words {start - prefix, fit + prefix};
//   4. the tile is reordered by bin in shared memory, and each bin's keys
//      leave in consecutive stores; the writer recomputes a key's bin from
//      the key instead of reading a tag array (ALU instead of two
//      shared-memory accesses per key).
// `base` (per bin, filled once per CTA) is where the bucket's range starts:
// its histogram offset (EXACT) or b * cap (CAPACITY).  Positions are 32-bit
// (the buffer has at most 2^32 entries).

// Bin of a key for the partition: value y = x - bias; with kCheck, keys above
// max_value go to the discard bin nb.  kShift: S = 2^sh.
template <bool kShift, bool kCheck>
__device__ __forceinline__ uint32_t part_bin(uint32_t x, uint32_t bias, uint32_t maxv, uint32_t sh, uint64_t magic,
                                             uint32_t nb) {
    const uint32_t y = x - bias;
    const uint32_t b = kShift ? (y >> sh) : bucket_of(y, magic);
    if (kCheck) return y <= maxv ? b : nb;
    return b;
}

constexpr int kOwnEarly = 4;   // bins per thread whose reservations are issued ahead of the scan

// Run words of bin i from its count c, tile prefix p and reservation `at`.
__device__ __forceinline__ uint2 part_run(const ArrayDesc &a, uint32_t i, uint32_t c, uint32_t p, uint32_t at,
                                          uint32_t base, bool capacity) {
    uint32_t fit;
    if (capacity) {
        const uint64_t cap = a.cap;
        fit = at >= cap ? 0u : (uint32_t)min((uint64_t)c, cap - at);
        if (fit < c) atomicOr(&a.sync[SY_OVERFLOW], 1u);   // only with repeated keys
    } else {
        const uint64_t st = (uint64_t)base + at;
        fit = st >= a.n ? 0u : (uint32_t)min((uint64_t)c, a.n - st);   // a sane scratch never clips
    }
    return make_uint2(base + at - p, fit + p);
}

// Steps 2 and 3 of a partition tile, once the tile's counts are in hist
// (all bins, the discard bin nb last): every thread reserves the runs of its
// buckets [lo_bin, hi_bin) in the partition buffer (global atomics, issued
// ahead of the scan when it owns at most kOwnEarly bins), the block scans
// the counts into tile prefixes (hist[i] = keys of the bins before i in the
// tile), and each bucket with keys gets its run words.  Ends with a barrier.
template <int T, bool kCheck>
__device__ __forceinline__ void part_scan_bins(const ArrayDesc &a, uint32_t *hist, const uint32_t *base, uint2 *run,
                                               uint32_t lo_bin, uint32_t hi_bin, SharedMisc &m) {
    constexpr int NW = T / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t nb = a.nslices;
    const bool capacity = a.layout == LAYOUT_CAPACITY;
    const bool early = hi_bin - lo_bin <= (uint32_t)kOwnEarly;
    uint32_t at[kOwnEarly];
    uint32_t own = 0;
    if (early) {
#pragma unroll
        for (int k = 0; k < kOwnEarly; ++k) {
            const uint32_t i = lo_bin + k;
            const uint32_t c = i < hi_bin ? hist[i] : 0u;
            at[k] = c ? atomicAdd(&a.cursor[i], c) : 0u;
            own += c;
        }
    } else {
        for (uint32_t i = lo_bin; i < hi_bin; ++i) own += hist[i];
    }
    const uint32_t incl = warp_incl_scan_u32(own, lane);
    if (lane == 31) m.wcount[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < NW ? m.wcount[lane] : 0u;
        const uint32_t wi = warp_incl_scan_u32(w, lane);
        if (lane < NW) m.wbase[lane] = wi - w;
        if (kCheck && lane == 31) {   // the discard bin after every bucket
            if (hist[nb]) run[nb] = make_uint2(0u, 0u);
            hist[nb] = wi;
        }
    }
    __syncthreads();

    uint32_t p = m.wbase[warp] + incl - own;
    if (early) {
#pragma unroll
        for (int k = 0; k < kOwnEarly; ++k) {
            const uint32_t i = lo_bin + k;
            if (i < hi_bin) {
                const uint32_t c = hist[i];
                hist[i] = p;
                if (c) run[i] = part_run(a, i, c, p, at[k], base[i], capacity);
                p += c;
            }
        }
    } else {
        for (uint32_t i = lo_bin; i < hi_bin; ++i) {
            const uint32_t c = hist[i];
            hist[i] = p;
            if (c) run[i] = part_run(a, i, c, p, atomicAdd(&a.cursor[i], c), base[i], capacity);
            p += c;
        }
    }
    __syncthreads();
}

// Keys of tile t into x (element j*T + threadIdx.x in x[j]): 16-byte loads
// for a whole tile of 16-byte aligned keys; returns the tile's key count.
template <int T>
__device__ __forceinline__ uint32_t part_load(const ArrayDesc &a, uint32_t t, uint32_t (&x)[kKeysPerThread]) {
    constexpr int K = kKeysPerThread;
    const uint64_t lo = (uint64_t)t * a.tile_keys;
    const uint32_t nkeys = (uint32_t)(min(lo + a.tile_keys, a.n) - lo);
    if (nkeys == a.tile_keys && (reinterpret_cast<uintptr_t>(a.keys) & 15u) == 0) {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.keys + lo);
#pragma unroll
        for (int j = 0; j < K / 4; ++j) {
            const uint4 q = __ldcs(src + j * T + threadIdx.x);
            x[4 * j] = q.x; x[4 * j + 1] = q.y; x[4 * j + 2] = q.z; x[4 * j + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const uint32_t e = (uint32_t)j * T + threadIdx.x;
            x[j] = e < nkeys ? __ldcs(a.keys + lo + e) : 0u;
        }
    }
    return nkeys;
}

// One tile: x[j] holds tile element j*T + threadIdx.x (valid while below
// nkeys; every element when kFull).  The thread owns buckets [lo_bin,
// hi_bin) (the discard bin nb, keys above max_value, comes after all of
// them and is never written); it zeroes their counts again at the end, so
// that the next tile starts with an empty histogram.  Once the reorder has
// used x, the keys of tile `next` (if below key_tiles) are loaded into it,
// so that their round trip overlaps this tile's write-out.  Ends with a
// barrier.
template <int T, bool kShift, bool kCheck, bool kFull>
__device__ void part_tile_phase(const ArrayDesc &a, uint32_t (&x)[kKeysPerThread], uint32_t nkeys, uint32_t *hist,
                                const uint32_t *base, uint2 *run, uint32_t *sorted, uint32_t lo_bin, uint32_t hi_bin,
                                SharedMisc &m, uint32_t next) {
    constexpr int K = kKeysPerThread;
    const uint32_t nb = a.nslices;
    const uint32_t bias = a.bias, maxv = (uint32_t)(a.M - 1), sh = a.s_shift;
    const uint64_t magic = a.div_magic;
    const bool capacity = a.layout == LAYOUT_CAPACITY;

    // 1. ranks inside the tile (bin << 16 | rank)
    uint32_t br[K];
    bool bad = false;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        br[j] = 0xFFFFFFFFu;
        if (kFull || (uint32_t)j * T + threadIdx.x < nkeys) {
            const uint32_t b = part_bin<kShift, kCheck>(x[j], bias, maxv, sh, magic, nb);
            if (kCheck) bad |= b == nb;
            br[j] = (b << 16) | atomicAdd(&hist[b], 1u);
        }
    }
    if (kCheck && capacity) {
        bad = __syncthreads_or(bad);
        if (bad && threadIdx.x == 0) atomicOr(&a.sync[SY_RANGE], 1u);
    } else {
        __syncthreads();   // (EXACT: the histogram pass reports keys above max_value)
    }

    // 2., 3. reservations, tile prefixes and run words of the buckets
    part_scan_bins<T, kCheck>(a, hist, base, run, lo_bin, hi_bin, m);

    // 4. reorder by bin, then each bin's keys leave in consecutive stores
#pragma unroll
    for (int j = 0; j < K; ++j) {
        if (kFull || br[j] != 0xFFFFFFFFu) sorted[hist[br[j] >> 16] + (br[j] & 0xFFFFu)] = x[j];
    }
    __syncthreads();
    // (eight keys at a time: their loads, then their run words, then their
    // stores, so that no key's shared-memory latency waits on another's)
    if (next < a.key_tiles) part_load<T>(a, next, x);
    uint32_t *part = a.part;
#pragma unroll
    for (int j0 = 0; j0 < K; j0 += 8) {
        uint32_t v[8];
        uint2 f[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const uint32_t i = (uint32_t)(j0 + u) * T + threadIdx.x;
            v[u] = (kFull || i < nkeys) ? sorted[i] : 0u;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) f[u] = run[part_bin<kShift, kCheck>(v[u], bias, maxv, sh, magic, nb)];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const uint32_t i = (uint32_t)(j0 + u) * T + threadIdx.x;
            if ((kFull || i < nkeys) && i < f[u].y) part[f[u].x + i] = v[u];
        }
    }
    for (uint32_t i = lo_bin; i < hi_bin; ++i) hist[i] = 0u;
    if (kCheck && threadIdx.x == 0) hist[nb] = 0u;
    __syncthreads();
}

template <int T>
__device__ void part_phase(const EngineParams &P, const ArrayDesc &a, char *smem, SharedMisc &m) {
    constexpr int K = kKeysPerThread;
    const uint32_t nb = a.nslices, nbins = nb + 1;
    // layout (as part_phase_smem_bytes): counts / prefixes | bucket bases | run words | tile
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem);
    uint32_t *base = hist + nbins;
    uint2 *run = reinterpret_cast<uint2 *>(smem + ((nbins * 8u + 7u) & ~7u));
    uint32_t *sorted = reinterpret_cast<uint32_t *>(run + nbins);
    const uint32_t per = (nb + T - 1) / T;
    const uint32_t lo_bin = min(nb, threadIdx.x * per), hi_bin = min(nb, lo_bin + per);
    const bool capacity = a.layout == LAYOUT_CAPACITY;
    for (uint32_t i = lo_bin; i < hi_bin; ++i) {
        hist[i] = 0u;
        base[i] = capacity ? (uint32_t)((uint64_t)i * a.cap) : (uint32_t)__ldcg(&a.offsets[i]);
    }
    if (threadIdx.x == 0) hist[nb] = 0u;
    __syncthreads();
    const bool shift = a.s_shift != 0;
    const bool check = a.M != (1ull << 32);
    const bool aligned = (reinterpret_cast<uintptr_t>(a.keys) & 15u) == 0;
    uint32_t t = blockIdx.x;
    if (t >= a.key_tiles) return;
    uint32_t x[K];
    uint32_t nkeys = part_load<T>(a, t, x);
    while (t < a.key_tiles) {
        const uint32_t next = t + gridDim.x;
        const bool full = nkeys == a.tile_keys && aligned;
        if (!full) part_tile_phase<T, false, true, false>(a, x, nkeys, hist, base, run, sorted, lo_bin, hi_bin, m, next);
        else if (shift && check) part_tile_phase<T, true, true, true>(a, x, nkeys, hist, base, run, sorted, lo_bin, hi_bin, m, next);
        else if (shift) part_tile_phase<T, true, false, true>(a, x, nkeys, hist, base, run, sorted, lo_bin, hi_bin, m, next);
        else if (check) part_tile_phase<T, false, true, true>(a, x, nkeys, hist, base, run, sorted, lo_bin, hi_bin, m, next);
        else part_tile_phase<T, false, false, true>(a, x, nkeys, hist, base, run, sorted, lo_bin, hi_bin, m, next);
        t = next;
        if (t < a.key_tiles) nkeys = (uint32_t)(min((uint64_t)(t + 1) * a.tile_keys, a.n) - (uint64_t)t * a.tile_keys);
    }
}

// ---------------------------------------------- bulk copies (TMA) + mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
                 : "memory");
}
// bytes from global src to shared dst (both 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(mbar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the given phase of an mbarrier (a bulk copy of this CTA's
// own); false after `limit_ns` (then the caller reports a timeout).
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(mbar, parity)) return true;
    WaitClock clk;
    clk.start();
    for (uint32_t it = 0; it < (1u << 30); ++it) {
        if (mbar_try_wait(mbar, parity)) return true;
        if ((it & 63) == 63 && clk.expired(limit_ns)) return false;
    }
    return false;
}

// Streaming PART (one kernel, one CTA per resident slot): a CTA takes tiles
// t, t + G, t + 2G, ...  While tile k is ranked, reserved, reordered and
// written, the bulk-copy engine already brings tile k+1 into the other
// buffer; a tile's landing buffer then serves as its reordered copy.  Tiles
// that are not whole, or keys that are not 16-byte aligned, are loaded by
// the threads instead.  The next tile's copy is issued only after the
// current tile's wait has succeeded in every thread, so after a timeout at
// most the copy that timed out is still outstanding; the CTA waits for it
// (four times the wait limit) before it exits.  That last wait is the only
// one whose expiry could leave a copy in flight at exit.
template <int T>
__device__ void part_stream(const EngineParams &P, const ArrayDesc &a, char *smem, SharedMisc &m) {
    constexpr int K = kKeysPerThread;
    const uint32_t nb = a.nslices;
    const uint32_t nbins = nb + 1;
    // layout (as part_stream_smem_bytes): bins | bucket tags | two landing buffers | two mbarriers
    const uint32_t off_tags = ((nbins * 12u) + 127u) & ~127u;
    const uint32_t off_buf = off_tags + ((a.tile_keys * 2u + 127u) & ~127u);
    const uint32_t off_mbar = off_buf + 2u * a.tile_keys * 4u;
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem);
    uint32_t *delta = hist + nbins;
    uint32_t *lim = delta + nbins;
    uint16_t *tags = reinterpret_cast<uint16_t *>(smem + off_tags);
    uint32_t *buf0 = reinterpret_cast<uint32_t *>(smem + off_buf);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + off_mbar);
    const uint32_t ntiles = a.key_tiles;
    const uint32_t G = gridDim.x;
    const uint32_t tile_bytes = a.tile_keys * 4u;
    const bool aligned = (reinterpret_cast<uintptr_t>(a.keys) & 15u) == 0;
    auto whole = [&](uint32_t t) { return aligned && (uint64_t)(t + 1) * a.tile_keys <= a.n; };

    uint32_t t = blockIdx.x;
    if (threadIdx.x == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && t < ntiles && whole(t)) {
        mbar_expect_tx(&mbar[0], tile_bytes);
        bulk_load(buf0, a.keys + (uint64_t)t * a.tile_keys, tile_bytes, &mbar[0]);
    }
    // per buffer: completed uses (mbarrier phase parity) and a copy issued
    // whose completion has not been seen
    uint32_t uses[2] = {0u, 0u};
    bool pend[2] = {t < ntiles && whole(t), false};
    for (uint32_t k = 0; t < ntiles; ++k, t += G) {
        const uint32_t b = k & 1u;
        uint32_t *cur = buf0 + (b ? a.tile_keys : 0u);
        uint32_t *nxt = buf0 + (b ? 0u : a.tile_keys);
        for (uint32_t i = threadIdx.x; i < nbins; i += T) hist[i] = 0;
        const uint64_t lo = (uint64_t)t * a.tile_keys;
        const uint32_t nkeys = (uint32_t)(min(lo + a.tile_keys, a.n) - lo);
        uint32_t x[K];
        bool ok = true;
        if (whole(t)) {
            ok = mbar_wait(&mbar[b], uses[b] & 1u, P.wait_limit_ns);
            if (ok) {
                ++uses[b];
                pend[b] = false;
                const uint4 *src = reinterpret_cast<const uint4 *>(cur);
#pragma unroll
                for (int j = 0; j < K / 4; ++j) {
                    const uint4 q = src[j * T + threadIdx.x];
                    x[4 * j] = q.x; x[4 * j + 1] = q.y; x[4 * j + 2] = q.z; x[4 * j + 3] = q.w;
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const uint32_t e = (uint32_t)j * T + threadIdx.x;
                x[j] = e < nkeys ? __ldcs(a.keys + lo + e) : 0u;
            }
        }
        // hist zeroed; every thread holds its keys (the buffer is free) or
        // some thread's wait ran out
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) atomicOr(&a.sync[SY_TIMEOUT], 1u);
            break;
        }
        const uint32_t tn = t + G;
        if (tn < ntiles && whole(tn)) {
            if (threadIdx.x == 0) {
                fence_proxy_async_smem();   // this buffer was last read and written by the threads
                mbar_expect_tx(&mbar[b ^ 1u], tile_bytes);
                bulk_load(nxt, a.keys + (uint64_t)tn * a.tile_keys, tile_bytes, &mbar[b ^ 1u]);
            }
            pend[b ^ 1u] = true;
        }
        part_tile<T>(a, x, nkeys, hist, delta, lim, cur, tags, m);
        __syncthreads();
    }
    // no bulk copy of this CTA may still be in flight when it exits: only a
    // copy whose wait ran out can be outstanding here
    for (int q = 0; q < 2; ++q)
        if (pend[q]) mbar_wait(&mbar[q], uses[q] & 1u, 4 * P.wait_limit_ns);
}

// Sparse slice (few keys for its words): the scatter also set one summary
// bit per non-empty word (summ), so counting and emission visit only the
// non-empty words: a lane takes one summary word (32 bitmap words) per step.
// Every word read is cleared behind (bitmap and summary), so the slice is zero
// again for this CTA's next sparse slice without a full clear.
// ------------------------------------------------- PART with wide tiles
// The phase kernel's partition at 32 keys a thread: tiles of 32 Ki keys at
// 1024 threads, 16 Ki at 512.  Against part_tile_phase's 16 keys a thread,
// the per-bucket work
// of a tile (reservations, prefixes, run words) is spread over twice the
// keys, and with thousands of buckets each run the tile leaves in the
// partition buffer is twice as long (fewer, fuller L2 writes).  Keys and
// their ranks would not both fit the registers, so the tile is a counting
// sort: pass 1 counts the keys per bin, the prefixes and reservations
// follow, and pass 2 takes each key's slot from its bin's running prefix
// (a shared-memory atomic; the order of a bucket's keys inside its run is
// arbitrary, and the bucket phase does not depend on it).  The next tile
// arrives while this one leaves: the write-out goes in four chunks, and
// behind each of the first three the matching quarter of the next tile is
// copied into the freed part of the tile buffer (cp.async, 16 bytes a
// thread); the last quarter comes into registers.

// Tile offset of a thread's element j: 16-byte group j/4 of the thread's
// eight, groups of the block interleaved (group g of thread i at g*T + i).
template <int T>
__device__ __forceinline__ uint32_t wide_elem(int j) {
    return 4u * ((uint32_t)(j >> 2) * T + threadIdx.x) + (uint32_t)(j & 3);
}

// Elements [J0, J1) of the tile of nkeys keys at a.keys + lo into x (vec:
// a whole tile of 16-byte aligned keys, read in 16-byte loads).
template <int T, int J0, int J1>
__device__ __forceinline__ void wide_load(const ArrayDesc &a, uint64_t lo, uint32_t nkeys, bool vec,
                                          uint32_t (&x)[kWideKeysPerThread]) {
    if (vec) {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.keys + lo);
#pragma unroll
        for (int g = J0 / 4; g < J1 / 4; ++g) {
            const uint4 q = __ldcs(src + g * T + threadIdx.x);
            x[4 * g] = q.x; x[4 * g + 1] = q.y; x[4 * g + 2] = q.z; x[4 * g + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int j = J0; j < J1; ++j) {
            const uint32_t e = wide_elem<T>(j);
            x[j] = e < nkeys ? __ldcs(a.keys + lo + e) : 0u;
        }
    }
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// One wide tile: x[j] holds tile element wide_elem(j) (valid while below
// nkeys; every element when kFull).  Bucket ownership, the discard bin and
// the zeroed histogram at the end are as in part_tile_phase.  stage_next:
// tile `next` is whole and its keys 16-byte aligned; its groups 0..5 are
// then copied into this thread's slots of the tile buffer (to be read by
// this thread after cp_async_wait_all) and its groups 6, 7 loaded into
// x[24..31].  Ends with a barrier.
template <int T, bool kShift, bool kCheck, bool kFull>
__device__ __forceinline__ void part_tile_wide(const ArrayDesc &a, uint32_t (&x)[kWideKeysPerThread], uint32_t nkeys,
                                               uint32_t *hist, const uint32_t *base, uint2 *run, uint32_t *sorted,
                                               uint32_t lo_bin, uint32_t hi_bin, SharedMisc &m, uint32_t next,
                                               bool stage_next) {
    constexpr int K = kWideKeysPerThread;
    static_assert(T * K / 8 / T == 4, "four write-out chunks of eight keys a thread");
    const uint32_t nb = a.nslices;
    const uint32_t bias = a.bias, maxv = (uint32_t)(a.M - 1), sh = a.s_shift;
    const uint64_t magic = a.div_magic;
    const bool capacity = a.layout == LAYOUT_CAPACITY;

    // 1. counts per bin
    bool bad = false;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        if (kFull || wide_elem<T>(j) < nkeys) {
            const uint32_t b = part_bin<kShift, kCheck>(x[j], bias, maxv, sh, magic, nb);
            if (kCheck) bad |= b == nb;
            atomicAdd(&hist[b], 1u);
        }
    }
    if (kCheck && capacity) {
        bad = __syncthreads_or(bad);
        if (bad && threadIdx.x == 0) atomicOr(&a.sync[SY_RANGE], 1u);
    } else {
        __syncthreads();   // (EXACT: the histogram pass reports keys above max_value)
    }

    // 2., 3. reservations, tile prefixes and run words of the buckets
    part_scan_bins<T, kCheck>(a, hist, base, run, lo_bin, hi_bin, m);

    // 4. every key to the next slot of its bin
#pragma unroll
    for (int j = 0; j < K; ++j) {
        if (kFull || wide_elem<T>(j) < nkeys) {
            const uint32_t b = part_bin<kShift, kCheck>(x[j], bias, maxv, sh, magic, nb);
            sorted[atomicAdd(&hist[b], 1u)] = x[j];
        }
    }
    __syncthreads();

    // 5. write-out, chunk c = sorted[8cT, 8(c+1)T): eight keys a thread, their
    // loads, then their run words, then their stores
    const uint64_t nlo = (uint64_t)next * a.tile_keys;
    if (stage_next) wide_load<T, 24, 32>(a, nlo, a.tile_keys, true, x);
    uint32_t *part = a.part;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uint32_t v[8];
        uint2 f[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const uint32_t i = (uint32_t)(8 * c + u) * T + threadIdx.x;
            v[u] = (kFull || i < nkeys) ? sorted[i] : 0u;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) f[u] = run[part_bin<kShift, kCheck>(v[u], bias, maxv, sh, magic, nb)];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const uint32_t i = (uint32_t)(8 * c + u) * T + threadIdx.x;
            if ((kFull || i < nkeys) && i < f[u].y) part[f[u].x + i] = v[u];
        }
        if (c < 3) {
            __syncthreads();   // chunk c is read: the next tile's groups 2c, 2c+1 may land there
            if (stage_next) {
                const uint32_t *src = a.keys + nlo;
#pragma unroll
                for (int g = 2 * c; g < 2 * c + 2; ++g) {
                    const uint32_t e = 4u * ((uint32_t)g * T + threadIdx.x);
                    cp_async16(sorted + e, src + e);
                }
                cp_async_commit();
            }
        }
    }
    for (uint32_t i = lo_bin; i < hi_bin; ++i) hist[i] = 0u;
    if (kCheck && threadIdx.x == 0) hist[nb] = 0u;
    __syncthreads();
}

// PART phase with wide tiles (T = 512 or 1024, a.tile_keys = 32 * T): a CTA takes
// tiles t, t + G, t + 2G, ...  Shared memory as part_phase.  A tile that is
// not whole, or keys that are not 16-byte aligned, are loaded by the threads
// at the start of the tile instead of behind the previous one.  Every copy
// a thread issues is waited for by that thread before its next tile, so none
// is in flight when the CTA exits.
template <int T>
__device__ void part_wide(const EngineParams &P, const ArrayDesc &a, char *smem, SharedMisc &m) {
    constexpr int K = kWideKeysPerThread;
    const uint32_t nb = a.nslices, nbins = nb + 1;
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem);
    uint32_t *base = hist + nbins;
    uint2 *run = reinterpret_cast<uint2 *>(smem + ((nbins * 8u + 7u) & ~7u));
    uint32_t *sorted = reinterpret_cast<uint32_t *>(run + nbins);
    const uint32_t per = (nb + T - 1) / T;
    const uint32_t lo_bin = min(nb, threadIdx.x * per), hi_bin = min(nb, lo_bin + per);
    const bool capacity = a.layout == LAYOUT_CAPACITY;
    for (uint32_t i = lo_bin; i < hi_bin; ++i) {
        hist[i] = 0u;
        base[i] = capacity ? (uint32_t)((uint64_t)i * a.cap) : (uint32_t)__ldcg(&a.offsets[i]);
    }
    if (threadIdx.x == 0) hist[nb] = 0u;
    __syncthreads();
    const bool shift = a.s_shift != 0;
    const bool check = a.M != (1ull << 32);
    const bool aligned = (reinterpret_cast<uintptr_t>(a.keys) & 15u) == 0;
    const uint32_t TK = a.tile_keys;
    auto keys_of = [&](uint32_t t) { return (uint32_t)(min((uint64_t)(t + 1) * TK, a.n) - (uint64_t)t * TK); };
    uint32_t t = blockIdx.x;
    if (t >= a.key_tiles) return;
    uint32_t x[K];
    uint32_t nkeys = keys_of(t);
    wide_load<T, 0, K>(a, (uint64_t)t * TK, nkeys, aligned && nkeys == TK, x);
    bool staged = false;
    while (t < a.key_tiles) {
        const uint32_t next = t + gridDim.x;
        const bool stage_next = next < a.key_tiles && aligned && keys_of(next) == TK;
        if (staged) {   // groups 0..5 copied by this thread behind the previous tile
            cp_async_wait_all();
            const uint4 *st4 = reinterpret_cast<const uint4 *>(sorted);
#pragma unroll
            for (int g = 0; g < 6; ++g) {
                const uint4 q = st4[g * T + threadIdx.x];
                x[4 * g] = q.x; x[4 * g + 1] = q.y; x[4 * g + 2] = q.z; x[4 * g + 3] = q.w;
            }
        }
        if (nkeys != TK) part_tile_wide<T, false, true, false>(a, x, nkeys, hist, base, run, sorted, lo_bin, hi_bin, m, next, stage_next);
        else if (shift && check) part_tile_wide<T, true, true, true>(a, x, nkeys, hist, base, run, sorted, lo_bin, hi_bin, m, next, stage_next);
        else if (shift) part_tile_wide<T, true, false, true>(a, x, nkeys, hist, base, run, sorted, lo_bin, hi_bin, m, next, stage_next);
        else if (check) part_tile_wide<T, false, true, true>(a, x, nkeys, hist, base, run, sorted, lo_bin, hi_bin, m, next, stage_next);
        else part_tile_wide<T, false, false, true>(a, x, nkeys, hist, base, run, sorted, lo_bin, hi_bin, m, next, stage_next);
        t = next;
        if (t >= a.key_tiles) break;
        nkeys = keys_of(t);
        if (!stage_next) wide_load<T, 0, K>(a, (uint64_t)t * TK, nkeys, aligned && nkeys == TK, x);
        staged = stage_next;
    }
}

template <int T>
__device__ void slice_finish_sparse(const EngineParams &P, const ArrayDesc &a, uint32_t s, uint32_t *bm,
                                    uint32_t *summ, uint32_t words, uint32_t v0, SharedMisc &m) {
    constexpr int NW = T / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t nsw = (words + 31) / 32;
    const uint32_t spw = (((nsw + NW - 1) / NW) + 31u) & ~31u;
    const uint32_t s0 = min(nsw, (uint32_t)warp * spw), s1 = min(nsw, s0 + spw);
    uint32_t cnt = 0;
    for (uint32_t j = s0 + lane; j < s1; j += 32) {
        uint32_t sm = summ[j];
        while (sm) {
            cnt += __popc(bm[j * 32 + (__ffs(sm) - 1)]);
            sm &= sm - 1;
        }
    }
    cnt = warp_sum_u32(cnt);
    if (lane == 0) m.wcount[warp] = cnt;
    __syncthreads();
    if (warp == 0) {
        const uint32_t c = lane < NW ? m.wcount[lane] : 0;
        const uint32_t incl = warp_incl_scan_u32(c, lane);
        if (lane < NW) m.wbase[lane] = incl - c;
        const uint32_t total = __shfl_sync(kFull, incl, 31);
        const uint64_t excl = slice_offset(P, a, s, total, lane, m);
        if (lane == 0) {
            m.excl = excl;
            m.total = total;
        }
    }
    __syncthreads();
    uint64_t base = m.excl + m.wbase[warp];
    const uint64_t lim = a.n;
    uint32_t *out = a.out;
    for (uint32_t j0 = s0; j0 < s1; j0 += 32) {
        const uint32_t j = j0 + lane;
        const uint32_t sm0 = j < s1 ? summ[j] : 0u;
        uint32_t c = 0;
        for (uint32_t sm = sm0; sm; sm &= sm - 1) c += __popc(bm[j * 32 + (__ffs(sm) - 1)]);
        const uint32_t incl = warp_incl_scan_u32(c, lane);
        const uint32_t chunk = __shfl_sync(kFull, incl, 31);
        uint64_t o = base + incl - c;
        for (uint32_t sm = sm0; sm; sm &= sm - 1) {
            const uint32_t w = j * 32 + (__ffs(sm) - 1);
            uint32_t x = bm[w];
            bm[w] = 0u;
            const uint32_t val = v0 + w * 32u - 1u;
            while (x) {
                if (o < lim) __stcs(out + o, val + __ffs(x));   // never past n
                ++o;
                x &= x - 1;
            }
        }
        if (sm0) summ[j] = 0u;
        base += chunk;
    }
    slice_complete<T>(a, m);
}

template <int T, int U = 8>
__device__ void bucket_slice(const EngineParams &P, const ArrayDesc &a, uint32_t b, char *smem, SharedMisc &m) {
    constexpr int NW = T / 32;
    const bool rank = a.emit == EMIT_RANK;
    const uint64_t v0 = (uint64_t)b * a.S;
    const uint64_t vals = min((uint64_t)a.S, a.M - v0);
    const uint32_t words = (uint32_t)((vals + 31) >> 5);
    const uint32_t w4 = (words + 3u) & ~3u;
    // shared memory: [summary bitmap] then EMIT_WORD [stage (optional) | bitmap]
    // or EMIT_RANK [bitmap | prefix | outputs]
    uint32_t *summ = reinterpret_cast<uint32_t *>(smem);
    uint32_t *stage = summ + kSummaryWords;
    uint32_t *bm = (!rank && a.stage) ? stage + NW * stage_words(T) : stage;
    uint32_t *pre = bm + w4;
    uint32_t *outs = pre + w4;
    const bool partitioned = a.path == BITSORT_PATH_PARTITION;

    if (threadIdx.x == 0) {
        m.flag = 1u;
        if (partitioned && !a.phased)
            m.flag = wait_geq(&a.sync[SY_PART_DONE], a.key_tiles + a.stall, &a.sync[SY_TIMEOUT], P.wait_limit_ns)
                         ? 1u : 0u;
    }
    __syncthreads();

    // where the slice's keys are: a range of the partition buffer, or the
    // whole input (fused path, or a capacity bucket that overflowed)
    const uint32_t *src = a.keys;
    uint64_t lo = 0, hi = a.n;
    bool filter_range = !partitioned;   // input keys above max_value are skipped and reported
    if (partitioned && a.layout == LAYOUT_CAPACITY) {
        const uint64_t filled = __ldcg(&a.cursor[b]);
        if (filled <= a.cap) {
            src = a.part;
            lo = (uint64_t)b * a.cap;
            hi = lo + filled;
        }
        if (known_offsets(a)) {   // the slice starts after the keys of the buckets before it
            uint64_t before = 0;
            for (uint32_t i = threadIdx.x; i < b; i += T) before += __ldcg(&a.cursor[i]);
            before = warp_sum_u64(before);
            if ((threadIdx.x & 31) == 0) m.wsum[threadIdx.x >> 5] = before;
            if (threadIdx.x == 0) m.expect = filled;
        }
    } else if (partitioned) {
        src = a.part;
        lo = min(__ldcg(&a.offsets[b]), a.n);
        hi = lo + min((uint64_t)__ldcg(&a.counts[b]), a.n - lo);
        if (threadIdx.x == 0) {
            m.known = lo;
            m.expect = hi - lo;
        }
    }
    if (!m.flag) hi = lo;
    if (known_offsets(a) && hi == lo && m.flag) {
        // a bucket that received no keys (most buckets of a few keys over a
        // wide range): no bitmap to build or read; the slice records a count
        // of zero at its offset and leaves the shared memory as it was
        __syncthreads();   // (the warps' sums of the CAPACITY offset)
        if (threadIdx.x == 0) {
            uint64_t known = m.known;
            if (a.layout == LAYOUT_CAPACITY) {
                known = 0;
                for (int w = 0; w < NW; ++w) known += m.wsum[w];
            }
            a.look[b] = known << 32;
            if (m.expect != 0) atomicOr(&a.sync[SY_MISMATCH], 1u);
        }
        slice_complete<T>(a, m);
        return;
    }
    // sparse slice: at most one key per four bitmap words (summary bitmap)
    const bool sparse = !rank && a.summary && (hi - lo) * 4 <= (uint64_t)words;
    if (!m.summ_clean) {
        for (uint32_t i = threadIdx.x; i < kSummaryWords; i += T) summ[i] = 0u;
    }
    if (!sparse || m.bm_clean_w < w4) {
        uint4 *bm4 = reinterpret_cast<uint4 *>(bm);
        for (uint32_t i = threadIdx.x; i < w4 / 4; i += T) bm4[i] = make_uint4(0, 0, 0, 0);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        m.summ_clean = 1u;
        if (partitioned && a.layout == LAYOUT_CAPACITY && known_offsets(a)) {
            uint64_t before = 0;
            for (int w = 0; w < NW; ++w) before += m.wsum[w];
            m.known = before;
        }
    }

    const uint32_t bias = a.bias;
    const uint32_t base = (uint32_t)v0 + bias, span = (uint32_t)vals;   // slice values: x - base in [0, span)
    bool bad = false;
    if (sparse) {
        auto set_bits = [&](uint32_t l) {
            const uint32_t w = l >> 5;
            atomicOr(&bm[w], 1u << (l & 31));
            atomicOr(&summ[w >> 5], 1u << (w & 31));
        };
        if (filter_range) {
            const uint64_t M = a.M;
            for_each_key<T, false, U>(src, lo, hi, [&](uint32_t x) {
                const uint32_t y = x - bias;
                if ((uint64_t)y < M) set_bits(y);
                else bad = true;
            });
        } else {
            for_each_key<T, false, U>(src, lo, hi, [&](uint32_t x) {
                const uint32_t l = x - base;
                if (l < span) set_bits(l);
            });
        }
    } else if (filter_range) {
        const uint64_t M = a.M;
        for_each_key<T, false, U>(src, lo, hi, [&](uint32_t x) {
            const uint32_t y = x - bias;
            if ((uint64_t)y < M) atomicOr(&bm[y >> 5], 1u << (y & 31));
            else bad = true;
        });
    } else {
        for_each_key<T, false, U>(src, lo, hi, [&](uint32_t x) {
            const uint32_t l = x - base;
            if (l < span) atomicOr(&bm[l >> 5], 1u << (l & 31));
        });
    }
    if (!m.flag && threadIdx.x == 0) atomicOr(&a.sync[SY_TIMEOUT], 1u);
    bad = __syncthreads_or(bad);
    if (bad && threadIdx.x == 0) atomicOr(&a.sync[SY_RANGE], 1u);
    if (partitioned && threadIdx.x == 0) {
        a.counts[b] = 0;
        if (a.nslices == 1) a.cursor[b] = 0;   // else the last CTA clears the cursors (known offsets)
    }
    if (sparse) {
        slice_finish_sparse<T>(P, a, b, bm, summ, words, base, m);
        if (threadIdx.x == 0) m.bm_clean_w = max(m.bm_clean_w, w4);   // every word read was cleared
        return;
    }
    if (threadIdx.x == 0) m.bm_clean_w = 0u;
    if (!rank) {
        slice_finish<T>(P, a, b, bm, words, base, stage, m);
        return;
    }

    // EMIT_RANK.  The slice reads its keys a second time below, so it must
    // not announce its count to later slices before that: a later slice that
    // knows its output offset may already be writing the output buffer, which
    // can hold this slice's keys (exact layout).  Ranks inside the slice need
    // no global offset, so the look-back comes after the second read.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t w0, w1;
    slice_count<T>(P, a, b, bm, words, 1, w0, w1, m, false);
    const uint32_t total = m.total;
    if (total > a.stage_cap) {
        // more outputs than the staging room (skewed keys): walk the words instead
        slice_lookback<T>(P, a, b, m);
        emit_words<1>(bm, w0, w1, base, m.excl + m.wbase[warp], a.out, a.n);
        slice_complete<T>(a, m);
        return;
    }
    {   // exclusive prefix of the set bits before every word of the slice
        uint32_t run = m.wbase[warp];
        for (uint32_t i0 = w0; i0 < w1; i0 += 32) {
            const uint32_t i = i0 + lane;
            const uint32_t c = i < w1 ? __popc(bm[i]) : 0u;
            const uint32_t incl = warp_incl_scan_u32(c, lane);
            if (i < w1) pre[i] = run + incl - c;
            run += __shfl_sync(kFull, incl, 31);
        }
    }
    __syncthreads();
    // every key writes itself at its index among the set bits
    if (filter_range) {
        const uint64_t M = a.M;
        for_each_key<T, true>(src, lo, hi, [&](uint32_t x) {
            const uint32_t y = x - bias;
            if ((uint64_t)y < M) {
                const uint32_t w = y >> 5;
                outs[pre[w] + __popc(bm[w] & ((1u << (y & 31)) - 1u))] = x;
            }
        });
    } else {
        for_each_key<T, true>(src, lo, hi, [&](uint32_t x) {
            const uint32_t l = x - base;
            if (l < span) {
                const uint32_t w = l >> 5;
                outs[pre[w] + __popc(bm[w] & ((1u << (l & 31)) - 1u))] = x;
            }
        });
    }
    __syncthreads();
    slice_lookback<T>(P, a, b, m);
    {   // the slice's outputs leave in consecutive stores
        uint32_t *out = a.out;
        const uint64_t o = m.excl;
        const uint32_t cnt = (o + total <= a.n) ? total : (o < a.n ? (uint32_t)(a.n - o) : 0u);
        for (uint32_t i = threadIdx.x; i < cnt; i += T) __stcs(out + o + i, outs[i]);
    }
    slice_complete<T>(a, m);
}

// A BUCKET item: one slice, or (sgroup > 1: a batch array of the exact
// layout, whose slices know their offsets and do not wait on one another)
// a run of sgroup consecutive slices.  A sparse array over a wide range has
// far more slices than keys; as a group, one item classifies its slices in
// parallel (a thread each), writes the zero-count look-back word of every
// empty slice, builds and emits only the slices with keys, and reports the
// whole group's completion at once.
// (compiled on its own, not inlined: its copy of the slice code then does
// not weigh on the register allocation of the one-slice path)
template <int T, int U>
__device__ __noinline__ void bucket_group(const EngineParams &P, const ArrayDesc &a, uint32_t idx, char *smem,
                                          SharedMisc &m) {
    const uint32_t g = a.sgroup;
    constexpr int NW = T / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t b0 = idx * g, b1 = min(b0 + g, a.nslices);
    const uint32_t was = m.defer;
    if (threadIdx.x == 0) {
        // the counts and offsets are final once the array's partition is done
        m.flag = 1u;
        if (!a.phased)
            m.flag = wait_geq(&a.sync[SY_PART_DONE], a.key_tiles + a.stall, &a.sync[SY_TIMEOUT], P.wait_limit_ns)
                         ? 1u : 0u;
    }
    __syncthreads();
    const bool ok = m.flag != 0;
    if (threadIdx.x == 0) {
        if (!ok) atomicOr(&a.sync[SY_TIMEOUT], 1u);
        m.defer = 1u;
        if (!was) m.done_local = 0u;
    }
    uint32_t built = 0;   // slices with keys handed to bucket_slice (thread 0's count)
    for (uint32_t c0 = b0; c0 < b1; c0 += T) {
        const uint32_t b = c0 + threadIdx.x;
        bool keys = false;
        if (b < b1) {
            keys = ok && __ldcg(&a.counts[b]) != 0u;
            if (!keys) a.look[b] = (uint64_t)__ldcg(&a.offsets[b]) << 32;   // an empty slice
        }
        const unsigned bal = __ballot_sync(kFull, keys);
        if (lane == 0) m.nonempty[warp] = bal;
        __syncthreads();
        for (int w = 0; w < NW; ++w) {
            uint32_t bits = m.nonempty[w];
            while (bits) {
                const uint32_t bb = c0 + (uint32_t)w * 32u + (uint32_t)(__ffs(bits) - 1);
                bits &= bits - 1u;
                bucket_slice<T, U>(P, a, bb, smem, m);
                ++built;
                __syncthreads();
            }
        }
        __syncthreads();   // (m.nonempty is rewritten for the next chunk)
    }
    // every slice of the group is done: the built ones counted themselves
    // while deferring, the empty ones are added here
    if (!was) {
        __syncthreads();
        if (threadIdx.x == 0) {
            m.defer = 0u;
            m.done_local = 0u;
        }
        complete_slices<T>(a, m, b1 - b0);
    } else {
        __syncthreads();
        if (threadIdx.x == 0) m.done_local += (b1 - b0) - built;
        __syncthreads();
    }
}

template <int T, int U = 8>
__device__ __forceinline__ void item_bucket(const EngineParams &P, const ArrayDesc &a, uint32_t idx, char *smem,
                                            SharedMisc &m) {
    if (a.sgroup > 1) bucket_group<T, U>(P, a, idx, smem, m);
    else bucket_slice<T, U>(P, a, idx, smem, m);
}

// GSCATTER: OR the keys of p[lo, hi) into the global bitmap (L2 atomics).
template <int T>
__device__ void gscatter_range(const ArrayDesc &a, uint64_t lo, uint64_t hi) {
    const uint64_t M = a.M;
    uint32_t *bitmap = a.bitmap;
    bool bad = false;
    const uint32_t bias = a.bias;
    for_each_key<T, true>(a.keys, lo, hi, [&](uint32_t x) {
        const uint32_t y = x - bias;
        if ((uint64_t)y < M) atomicOr(&bitmap[y >> 5], 1u << (y & 31));
        else bad = true;
    });
    bad = __syncthreads_or(bad);
    if (bad && threadIdx.x == 0) atomicOr(&a.sync[SY_RANGE], 1u);
}

template <int T>
__device__ void item_gscatter(const EngineParams &P, const ArrayDesc &a, uint32_t tile, SharedMisc &m) {
    const uint64_t lo = (uint64_t)tile * a.tile_keys;
    gscatter_range<T>(a, lo, min(lo + a.tile_keys, a.n));
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&a.sync[SY_PART_DONE], 1u);
    }
}

template <int T>
__device__ void item_gscan(const EngineParams &P, const ArrayDesc &a, uint32_t s, char *smem, SharedMisc &m) {
    constexpr int NW = T / 32;
    uint32_t *stage = reinterpret_cast<uint32_t *>(smem) + kSummaryWords;
    uint32_t *bm = a.stage ? stage + NW * stage_words(T) : stage;
    const uint64_t v0 = (uint64_t)s * a.S;
    const uint64_t vals = min((uint64_t)a.S, a.M - v0);
    const uint32_t words = (uint32_t)((vals + 31) >> 5);
    const uint32_t w4 = (words + 3u) & ~3u;
    if (threadIdx.x == 0) {
        m.flag = 1u;
        if (!a.phased)
            m.flag = wait_geq(&a.sync[SY_PART_DONE], a.key_tiles + a.stall, &a.sync[SY_TIMEOUT], P.wait_limit_ns)
                         ? 1u : 0u;
    }
    __syncthreads();
    uint4 *bm4 = reinterpret_cast<uint4 *>(bm);
    uint4 *src = reinterpret_cast<uint4 *>(a.bitmap + (v0 >> 5));
    if (m.flag) {
        for (uint32_t i = threadIdx.x; i < w4 / 4; i += T) {
            bm4[i] = __ldcg(src + i);
            __stcg(src + i, make_uint4(0, 0, 0, 0));  // clean behind: zero for the next call
        }
    } else {
        for (uint32_t i = threadIdx.x; i < w4 / 4; i += T) bm4[i] = make_uint4(0, 0, 0, 0);
        if (threadIdx.x == 0) atomicOr(&a.sync[SY_TIMEOUT], 1u);
    }
    __syncthreads();
    // words past the array's last value are zero in the bitmap (padding)
    slice_finish<T>(P, a, s, bm, words, (uint32_t)v0 + a.bias, stage, m);
}

// ----------------------------------------------------------------- kernel
template <int T>
__global__ void __launch_bounds__(T, 1024 / T) engine_kernel(const __grid_constant__ EngineParams P) {
    extern __shared__ __align__(16) char smem[];
    __shared__ SharedMisc m;
    const Segment *segs = P.segments ? P.segments : P.seg;
    if (threadIdx.x == 0) {
        m.summ_clean = 0u;
        m.bm_clean_w = 0u;
        m.defer = 0u;
        m.done_local = 0u;
    }
    for (;;) {
        if (threadIdx.x == 0) m.ticket = atomicAdd(&P.ticket[0], 1u);
        __syncthreads();
        const uint32_t t = m.ticket;
        __syncthreads();
        if (t >= P.total_items) break;
        uint32_t lo = 0, hi = P.nseg;  // last segment with start <= t
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (segs[mid].start <= t) lo = mid;
            else hi = mid;
        }
        const Segment sg = segs[lo];
        const ArrayDesc &a = P.arrays ? P.arrays[sg.array] : P.one;
        const uint32_t idx = sg.first + (t - sg.start);
        switch (sg.type) {
            case IT_HIST: item_hist<T>(P, a, idx, smem, m); break;
            case IT_PART: item_part<T>(P, a, idx, smem, m); break;
            case IT_BUCKET: item_bucket<T>(P, a, idx, smem, m); break;
            case IT_GSCATTER: item_gscatter<T>(P, a, idx, m); break;
            case IT_GSCAN: item_gscan<T>(P, a, idx, smem, m); break;
            default: break;
        }
        __syncthreads();
        if (threadIdx.x == 0 && sg.type != IT_BUCKET) {
            // other items use the shared memory their own way
            m.bm_clean_w = 0u;
            if (sg.type != IT_GSCAN) m.summ_clean = 0u;
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&P.ticket[1], 1u) == gridDim.x - 1) {
            P.ticket[0] = 0;
            P.ticket[1] = 0;
            __threadfence();
        }
    }
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while the previous kernel of the stream drains;
// griddepcontrol.wait blocks until that kernel has completed and its writes
// are visible (a no-op when there is no such dependency).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// One phase of the sort of a single array (P.one) as its own kernel, so that
// each phase runs with the occupancy its shared memory allows.  Slice phases
// take their slices in ticket order (the look-back needs it); tile phases use
// a grid-stride loop.
// MINB = 1024 / T: at most 64 registers per thread, so that 1024 threads
// (four CTAs of 256, two of 512) fit one SM.  MINB = 1 (a "solo" kernel) is
// launched when the phase's shared memory leaves room for one CTA per SM
// only: the CTA then gets the whole register file (up to 255 registers a
// thread at 256 threads, 128 at 512), and the bucket scatter keeps 16
// 16-byte loads in flight per thread instead of 8.
template <int T, int TYPE, int MINB = 1024 / T>
__global__ void __launch_bounds__(T, MINB) phase_kernel(const __grid_constant__ EngineParams P) {
    constexpr int U = (MINB == 1 && T <= 512) ? 16 : 8;
    extern __shared__ __align__(16) char smem[];
    __shared__ SharedMisc m;
    if (threadIdx.x == 0) {
        m.summ_clean = 0u;
        m.bm_clean_w = 0u;
        m.defer = 0u;
        m.done_local = 0u;
    }
    pdl_wait();
    const ArrayDesc &a = P.one;
    if constexpr (TYPE == IT_BUCKET || TYPE == IT_GSCAN) {
      if (TYPE == IT_BUCKET && (known_offsets(a) || a.nslices == 1)) {
        // the slices do not wait on one another: a fixed share per CTA, one
        // completion report per CTA
        if (threadIdx.x == 0) m.defer = 1u;
        __syncthreads();
        for (uint32_t t = blockIdx.x; t < P.total_items; t += gridDim.x) {
            item_bucket<T, U>(P, a, t, smem, m);
            __syncthreads();
        }
        pdl_trigger();
        const uint32_t done = m.done_local;
        if (threadIdx.x == 0) m.defer = 0u;
        if (done) complete_slices<T>(a, m, done);
      } else {
        for (;;) {
            if (threadIdx.x == 0) m.ticket = atomicAdd(&P.ticket[0], 1u);
            __syncthreads();
            const uint32_t t = m.ticket;
            __syncthreads();
            if (t >= P.total_items) break;
            if constexpr (TYPE == IT_BUCKET) item_bucket<T, U>(P, a, t, smem, m);
            else item_gscan<T>(P, a, t, smem, m);
            __syncthreads();
        }
        pdl_trigger();
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicAdd(&P.ticket[1], 1u) == gridDim.x - 1) {
                P.ticket[0] = 0;
                P.ticket[1] = 0;
                __threadfence();
            }
        }
      }
    } else if constexpr (TYPE == IT_PARTS) {
        part_stream<T>(P, a, smem, m);
        pdl_trigger();

    } else if constexpr (TYPE == IT_PART) {
        part_phase<T>(P, a, smem, m);
        pdl_trigger();
    } else if constexpr (TYPE == IT_PARTW) {
        part_wide<T>(P, a, smem, m);
        pdl_trigger();
    } else {
        // HIST / GSCATTER stream one contiguous chunk of keys per CTA (one
        // flush of the shared histogram, one completion count per CTA)
        const uint64_t chunk = ((a.n + gridDim.x - 1) / gridDim.x + 3) & ~3ull;
        const uint64_t lo = min((uint64_t)blockIdx.x * chunk, a.n);
        const uint64_t hi = min(lo + chunk, a.n);
        if constexpr (TYPE == IT_HIST) hist_range<T>(a, lo, hi, gridDim.x, smem, m);
        else gscatter_range<T>(a, lo, hi);
        pdl_trigger();
    }
}

// ------------------------------------------------------------------- host
using KernelFn = void (*)(EngineParams);

// A phase whose dynamic shared memory is above this leaves room for one CTA
// per SM (of the 228 KiB of an SM), so its solo kernel (MINB = 1) is used.
constexpr uint32_t kSoloSmemBytes = 114u * 1024u - 1024u;

// kind: -1 = persistent engine, else an ItemType (one phase); solo: the
// MINB = 1 instance of a phase kernel (256 / 512 threads)
static KernelFn kernel_for(int kind, int threads, bool solo = false) {
    if (threads == 256) {
        if (solo) {
            switch (kind) {
                case IT_PART: return phase_kernel<256, IT_PART, 1>;
                case IT_BUCKET: return phase_kernel<256, IT_BUCKET, 1>;
                case IT_GSCAN: return phase_kernel<256, IT_GSCAN, 1>;
                case IT_PARTS: return phase_kernel<256, IT_PARTS, 1>;
            }
        }
        switch (kind) {
            case -1: return engine_kernel<256>;
            case IT_HIST: return phase_kernel<256, IT_HIST>;
            case IT_PART: return phase_kernel<256, IT_PART>;
            case IT_BUCKET: return phase_kernel<256, IT_BUCKET>;
            case IT_GSCATTER: return phase_kernel<256, IT_GSCATTER>;
            case IT_GSCAN: return phase_kernel<256, IT_GSCAN>;
            case IT_PARTS: return phase_kernel<256, IT_PARTS>;
        }
    } else if (threads == 512) {
        if (solo) {
            switch (kind) {
                case IT_PART: return phase_kernel<512, IT_PART, 1>;
                case IT_BUCKET: return phase_kernel<512, IT_BUCKET, 1>;
                case IT_GSCAN: return phase_kernel<512, IT_GSCAN, 1>;
                case IT_PARTS: return phase_kernel<512, IT_PARTS, 1>;
            }
        }
        switch (kind) {
            case -1: return engine_kernel<512>;
            case IT_HIST: return phase_kernel<512, IT_HIST>;
            case IT_PART: return phase_kernel<512, IT_PART>;
            case IT_BUCKET: return phase_kernel<512, IT_BUCKET>;
            case IT_GSCATTER: return phase_kernel<512, IT_GSCATTER>;
            case IT_GSCAN: return phase_kernel<512, IT_GSCAN>;
            case IT_PARTS: return phase_kernel<512, IT_PARTS>;
            case IT_PARTW: return phase_kernel<512, IT_PARTW>;
        }
    } else if (threads == 1024) {
        // one CTA per SM for the phase kernels of a single sort (the
        // persistent engine stays at 256 / 512 threads)
        switch (kind) {
            case IT_HIST: return phase_kernel<1024, IT_HIST>;
            case IT_PART: return phase_kernel<1024, IT_PART>;
            case IT_BUCKET: return phase_kernel<1024, IT_BUCKET>;
            case IT_GSCATTER: return phase_kernel<1024, IT_GSCATTER>;
            case IT_GSCAN: return phase_kernel<1024, IT_GSCAN>;
            case IT_PARTS: return phase_kernel<1024, IT_PARTS>;
            case IT_PARTW: return phase_kernel<1024, IT_PARTW>;
        }
    }
    return nullptr;
}

// the kernel a phase launches with `smem_bytes` of dynamic shared memory
static KernelFn kernel_for_smem(int kind, int threads, uint32_t smem_bytes) {
    const bool solo = kind >= 0 && threads < 1024 && smem_bytes > kSoloSmemBytes;
    KernelFn f = solo ? kernel_for(kind, threads, true) : nullptr;
    return f ? f : kernel_for(kind, threads);
}

int engine_set_smem_limit(int threads, uint32_t smem_bytes) {
    for (int kind : {-1, (int)IT_HIST, (int)IT_PART, (int)IT_BUCKET, (int)IT_GSCATTER, (int)IT_GSCAN, (int)IT_PARTS,
                     (int)IT_PARTW}) {
        if (kind == -1 && threads == 1024) continue;   // no persistent engine at 1024 threads
        if (kind == IT_PARTW && threads == 256) continue;   // wide tiles at 512 and 1024 threads
        KernelFn f = kernel_for(kind, threads);
        if (!f) return (int)cudaErrorInvalidValue;
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
        if (e != cudaSuccess) return (int)e;
        KernelFn g = threads < 1024 ? kernel_for(kind, threads, true) : nullptr;
        if (g && g != f) {
            e = cudaFuncSetAttribute(g, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
            if (e != cudaSuccess) return (int)e;
        }
    }
    return 0;
}

int engine_max_blocks_per_sm(int threads, uint32_t smem_bytes, int *blocks) {
    return kernel_max_blocks_per_sm(-1, threads, smem_bytes, blocks);
}

int kernel_max_blocks_per_sm(int kind, int threads, uint32_t smem_bytes, int *blocks) {
    KernelFn f = kernel_for_smem(kind, threads, smem_bytes);
    if (!f) return (int)cudaErrorInvalidValue;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, f, threads, smem_bytes);
}

int engine_launch(const EngineParams &p, int threads, uint32_t smem_bytes, int grid, void *stream) {
    return kernel_launch(-1, p, threads, smem_bytes, grid, stream, false);
}

int kernel_launch(int kind, const EngineParams &p, int threads, uint32_t smem_bytes, int grid, void *stream,
                  bool pdl) {
    KernelFn f = kernel_for_smem(kind, threads, smem_bytes);
    if (!f) return (int)cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem_bytes;
    cfg.stream = reinterpret_cast<cudaStream_t>(stream);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaSuccess;
    if (pdl) {
        e = cudaLaunchKernelEx(&cfg, f, p);
        if (e == cudaSuccess) return 0;
        // a stream or driver that does not take programmatic serialization:
        // launch in plain stream order instead
        if (getenv("BITSORT_VERBOSE"))
            fprintf(stderr, "bitsort: programmatic launch refused (%s); plain launch\n", cudaGetErrorString(e));
        cudaGetLastError();
    }
    f<<<grid, threads, smem_bytes, cfg.stream>>>(p);
    return (int)cudaGetLastError();
}

}  // namespace bsx
