/*
 * Seeded synthetic input generators shared by the CPU oracle's tests and the
 * GPU library's tests and benchmark.
 *
 * This file holds only pseudo-random number generation and sampling; none of
 * the sort's arithmetic (no bitmap, no popcount, no ordering) lives here.
 *
 *   splitmix64      Steele, Lea & Flood, "Fast splittable pseudorandom number
 *                   generators", OOPSLA 2014 (the 64-bit finaliser variant
 *                   used to seed other generators).
 *   xoshiro256**    Blackman & Vigna, "Scrambled linear pseudorandom number
 *                   generators", ACM TOMS 2021.
 *   bounded draws   Lemire, "Fast random integer generation in an interval",
 *                   ACM TOMACS 2019 (multiply, then reject the biased slice).
 *   Floyd sampling  Bentley & Floyd, "A sample of brilliance", CACM 1987:
 *                   n distinct values from [0, M) in O(n) draws.  Membership
 *                   is an open-addressing hash set (no bitmap).
 *   Fisher-Yates    Durstenfeld, CACM 1964 (algorithm 235), in-place shuffle.
 *   Feistel         a keyed balanced Feistel network on d = 2h bits with
 *                   cycle walking (Black & Rogaway, "Ciphers with arbitrary
 *                   finite domains", CT-RSA 2002) gives a bijection of
 *                   [0, M); keys[i] = pi(i) for i < n are n distinct values in
 *                   pseudo-random order.  The round function is the
 *                   "lowbias32" integer hash published by C. Wellons (2018).
 *
 * Everything is deterministic given the seed and builds identically on x86-64
 * and aarch64 (fixed-width types only, no intrinsics).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct { uint64_t s[4]; } xoshiro_t;

static uint64_t splitmix64_next(uint64_t *state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static void xoshiro_seed(xoshiro_t *g, uint64_t seed) {
    uint64_t sm = seed;
    for (int i = 0; i < 4; ++i) g->s[i] = splitmix64_next(&sm);
}

static inline uint64_t xoshiro_next(xoshiro_t *g) {
    uint64_t *s = g->s;
    const uint64_t result = rotl64(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}

/* Uniform integer in [0, range) for 1 <= range <= 2^32 (Lemire's method). */
static inline uint64_t bounded(xoshiro_t *g, uint64_t range) {
    uint64_t x = xoshiro_next(g) >> 32;          /* 32 random bits */
    uint64_t m = x * range;                      /* < 2^64 since range <= 2^32 */
    uint64_t low = m & 0xFFFFFFFFull;
    if (low < range) {
        uint64_t thresh = ((1ull << 32) - range) % range;   /* 2^32 mod range */
        while (low < thresh) {
            x = xoshiro_next(g) >> 32;
            m = x * range;
            low = m & 0xFFFFFFFFull;
        }
    }
    return m >> 32;
}

/* Uniform double in [0, 1) with 53 random bits. */
static inline double unit_f64(xoshiro_t *g) {
    return (double)(xoshiro_next(g) >> 11) * (1.0 / 9007199254740992.0);
}

/* ---------------------------------------------------------------- hash set */
typedef struct { uint64_t *slot; uint64_t mask; } hset_t;   /* 0 = empty, v+1 stored */

static int hset_init(hset_t *h, uint64_t n) {
    uint64_t cap = 16;
    while (cap < 2 * n + 16) cap <<= 1;
    h->slot = (uint64_t *)calloc(cap, sizeof(uint64_t));
    h->mask = cap - 1;
    return h->slot ? 0 : -1;
}

/* Returns 1 if v was inserted, 0 if it was already present. */
static int hset_insert(hset_t *h, uint64_t v) {
    uint64_t i = ((v + 1) * 0x9E3779B97F4A7C15ull) >> 20;
    for (;;) {
        i &= h->mask;
        uint64_t cur = h->slot[i];
        if (cur == 0) { h->slot[i] = v + 1; return 1; }
        if (cur == v + 1) return 0;
        ++i;
    }
}

/* ------------------------------------------------------------ public calls */

/* n distinct values from [0, M) by Floyd's algorithm, then Fisher-Yates
 * shuffled.  Requires n <= M, M <= 2^32.  Returns 0 on success. */
int gen_floyd_shuffled(uint64_t seed, uint64_t n, uint64_t M, uint32_t *out) {
    if (n > M || M > (1ull << 32) || M == 0) return n == 0 ? 0 : -1;
    if (n == 0) return 0;
    xoshiro_t g; xoshiro_seed(&g, seed);
    hset_t h; if (hset_init(&h, n)) return -2;
    uint64_t k = 0;
    for (uint64_t j = M - n; j < M; ++j) {
        uint64_t t = bounded(&g, j + 1);          /* uniform in [0, j] */
        if (hset_insert(&h, t)) out[k++] = (uint32_t)t;
        else { hset_insert(&h, j); out[k++] = (uint32_t)j; }
    }
    free(h.slot);
    for (uint64_t i = n - 1; i > 0; --i) {
        uint64_t j = bounded(&g, i + 1);
        uint32_t tmp = out[i]; out[i] = out[j]; out[j] = tmp;
    }
    return 0;
}

/* Fisher-Yates shuffle of an existing array in place. */
void gen_shuffle_u32(uint64_t seed, uint32_t *a, uint64_t n) {
    if (n < 2) return;
    xoshiro_t g; xoshiro_seed(&g, seed);
    for (uint64_t i = n - 1; i > 0; --i) {
        uint64_t j = bounded(&g, i + 1);
        uint32_t tmp = a[i]; a[i] = a[j]; a[j] = tmp;
    }
}

/* n uniform draws from [0, M) WITH replacement (duplicates likely): used to
 * build inputs that break the distinct-key contract on purpose. */
int gen_uniform_u32(uint64_t seed, uint64_t n, uint64_t M, uint32_t *out) {
    if (M == 0 || M > (1ull << 32)) return -1;
    xoshiro_t g; xoshiro_seed(&g, seed);
    for (uint64_t i = 0; i < n; ++i) out[i] = (uint32_t)bounded(&g, M);
    return 0;
}

/* count uniform doubles in [0, 1). */
void gen_unit_f64(uint64_t seed, uint64_t count, double *out) {
    xoshiro_t g; xoshiro_seed(&g, seed);
    for (uint64_t i = 0; i < count; ++i) out[i] = unit_f64(&g);
}

/* ----------------------------------------------------------------- Feistel */
typedef struct { uint32_t key[8]; int half; uint32_t mask; uint64_t M; int rounds; } feistel_t;

static inline uint32_t lowbias32(uint32_t x) {
    x ^= x >> 16; x *= 0x7feb352dU;
    x ^= x >> 15; x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

static void feistel_init(feistel_t *f, uint64_t seed, uint64_t M) {
    int d = 2;
    while (d < 64 && (1ull << d) < M) ++d;
    if (d & 1) ++d;
    f->half = d / 2;
    f->mask = (uint32_t)((1ull << f->half) - 1);
    f->M = M;
    f->rounds = 6;
    uint64_t sm = seed ^ 0xF2E15E1Dull;
    for (int i = 0; i < 8; ++i) f->key[i] = (uint32_t)splitmix64_next(&sm);
}

static inline uint64_t feistel_enc_once(const feistel_t *f, uint64_t x) {
    uint32_t L = (uint32_t)(x >> f->half) & f->mask, R = (uint32_t)x & f->mask;
    for (int r = 0; r < f->rounds; ++r) {
        uint32_t nl = R;
        uint32_t nr = L ^ (lowbias32(R ^ f->key[r]) & f->mask);
        L = nl; R = nr;
    }
    return ((uint64_t)L << f->half) | R;
}

static inline uint64_t feistel_dec_once(const feistel_t *f, uint64_t y) {
    uint32_t L = (uint32_t)(y >> f->half) & f->mask, R = (uint32_t)y & f->mask;
    for (int r = f->rounds - 1; r >= 0; --r) {
        uint32_t pr = L;
        uint32_t pl = R ^ (lowbias32(L ^ f->key[r]) & f->mask);
        L = pl; R = pr;
    }
    return ((uint64_t)L << f->half) | R;
}

/* keys[i] = pi(start + i), pi a bijection of [0, M) (cycle-walked Feistel). */
int gen_feistel_perm(uint64_t seed, uint64_t M, uint64_t start, uint64_t count, uint32_t *out) {
    if (M == 0 || M > (1ull << 32) || start + count > M) return -1;
    feistel_t f; feistel_init(&f, seed, M);
    #pragma omp parallel for schedule(static)
    for (uint64_t i = 0; i < count; ++i) {
        uint64_t y = feistel_enc_once(&f, start + i);
        while (y >= M) y = feistel_enc_once(&f, y);
        out[i] = (uint32_t)y;
    }
    return 0;
}

/* out[i] = pi^{-1}(y[i]) for the same permutation as gen_feistel_perm. */
int gen_feistel_inverse(uint64_t seed, uint64_t M, const uint32_t *y, uint64_t count, uint64_t *out) {
    if (M == 0 || M > (1ull << 32)) return -1;
    feistel_t f; feistel_init(&f, seed, M);
    #pragma omp parallel for schedule(static)
    for (uint64_t i = 0; i < count; ++i) {
        uint64_t x = feistel_dec_once(&f, y[i]);
        while (x >= M) x = feistel_dec_once(&f, x);
        out[i] = x;
    }
    return 0;
}
