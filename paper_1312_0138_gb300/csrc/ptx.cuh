// ptx.cuh -- memory-model and timer helpers in inline PTX shared by the
// kernels of the library: acquire loads and release stores at GPU scope (the
// publication of look-back words and flags between CTAs) and the global
// nanosecond timer that bounds every wait.
#pragma once
#include <stdint.h>

namespace bsx {

__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u64(uint64_t *p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wall-clock bound of one wait.  The wait has expired once two consecutive
// windows of half the limit have passed, each measured from a fresh timer
// read: a single step of the global timer (the driver may adjust it, forwards
// or back) then cannot end a wait early, and a timer read that lies before
// the window's start restarts the window instead of wrapping the unsigned
// difference.  Every caller also caps its number of polls, so a timer that
// stops or runs backwards still ends the wait.
struct WaitClock {
    uint64_t t0 = 0;
    uint32_t windows = 0;
    __device__ __forceinline__ void start() {
        t0 = now_ns();
        windows = 0;
    }
    __device__ __forceinline__ bool expired(uint64_t limit_ns) {
        const uint64_t t = now_ns();
        if (t < t0) {
            t0 = t;
        } else if (t - t0 > limit_ns / 2) {
            t0 = t;
            ++windows;
        }
        return windows >= 2;
    }
};

}  // namespace bsx
