/*
 * CPU oracle for the bitwise sort of an integer array.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline / reference leg load this library.  The GPU
 * library never links, includes or calls it, and this file includes nothing
 * from the GPU library: the two share no code.
 *
 * Plain, slow, obviously correct C.  Every function restates a passage of
 * the paper (K. Yordzhev, "The bitwise operations related to a fast sorting
 * algorithm"):
 *
 *   oracle_bit_value      Example 1 (value of bit i of x via x & 1<<i), with
 *                         the bit numbering of Section II (bit 0 rightmost).
 *   oracle_bin_repl_i16   Example 4 (bit pattern of a short, most significant
 *                         bit first); pinned by Table II.
 *   oracle_bitmap_sort    the bit-set form of the bitwise sort: every key x
 *                         sets bit (x mod 32) of word floor(x / 32) with OR
 *                         (Table I) and a shifted one (Example 2); the words
 *                         are then read in index order and, inside a word,
 *                         from bit 0 upwards (Section II numbering), and every
 *                         set bit is written out.  For distinct keys the
 *                         result is the ascending order of Theorem 1.
 *   oracle_paper_sort_u32 Algorithm 1, first function: one stable split of
 *                         the array per bit, zeros before ones, bits taken
 *                         from 0 upwards; `nbits` passes.  The paper stops
 *                         before the sign bit (t-1 passes for a t-bit type);
 *                         an unsigned 32-bit key needs all 32.
 *   oracle_paper_sort_i32 Algorithm 1, second function: negatives and
 *                         non-negatives separated (order kept), each sorted
 *                         by the first function over bits 0..t-2, negatives
 *                         written first.
 *   oracle_bitmap_sort_i32  the bit-set form for signed keys in
 *                         [min_value, max_value] (offsets from min_value).
 *   oracle_bitmap_sort_u64  the bit-set form for 64-bit keys (Algorithm 1 is
 *                         written for any integer type T).
 *
 * Status codes (same numbering as the GPU library's public header, written
 * out again here on purpose):
 *   0 OK, 2 KEY_RANGE (a key above max_value was skipped),
 *   3 DUPLICATE (fewer distinct keys than n), 4 NOMEM.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_KEY_RANGE 2
#define ORACLE_DUPLICATE 3
#define ORACLE_NOMEM 4

/* Example 1: 1 if bit i of x is set, else 0 (i in 0..31, bit 0 rightmost). */
int oracle_bit_value(uint32_t x, unsigned i) {
    return (x & (1u << i)) != 0 ? 1 : 0;
}

/* Table I, column "z = x | y", applied bitwise: exposed so that the truth
 * table can be checked against the operation the oracle's bitmap uses. */
uint32_t oracle_bit_or(uint32_t x, uint32_t y) { return x | y; }

/* Example 4: the 16 bits of a short, most significant first, as '0'/'1'
 * characters; out must hold 17 bytes (NUL-terminated). */
void oracle_bin_repl_i16(int16_t v, char *out) {
    uint16_t bits = (uint16_t)v;            /* the stored two's-complement pattern */
    for (int d = 15; d >= 0; --d)
        out[15 - d] = ((bits >> d) & 1u) ? '1' : '0';
    out[16] = '\0';
}

/*
 * Bitmap sort of n keys bounded by max_value.
 *
 * M = max_value + 1 values are possible, so the bitmap has ceil(M / 32)
 * words (M is computed in 64 bits: max_value may be 2^32 - 1).
 *   1. all words start at zero;
 *   2. for every key x <= max_value: word[x / 32] |= 1 << (x mod 32);
 *      a key above max_value is skipped and reported (KEY_RANGE);
 *   3. for word w = 0, 1, ... and bit b = 0..31 inside it: if the bit is set,
 *      append 32 w + b to out.
 * *count receives the number of values written.  If it is smaller than n
 * while every key was in range, some key occurred twice (DUPLICATE): out then
 * holds the ascending distinct keys.  out needs room for n values.
 */
int oracle_bitmap_sort(const uint32_t *keys, uint64_t n, uint32_t max_value,
                       uint32_t *out, uint64_t *count) {
    uint64_t M = (uint64_t)max_value + 1u;
    uint64_t words = (M + 31u) / 32u;
    uint32_t *bitmap = (uint32_t *)calloc(words, sizeof(uint32_t));
    if (bitmap == NULL) return ORACLE_NOMEM;

    int out_of_range = 0;
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t x = keys[i];
        if (x > max_value) { out_of_range = 1; continue; }
        bitmap[x / 32u] = bitmap[x / 32u] | (1u << (x % 32u));
    }

    uint64_t k = 0;
    for (uint64_t w = 0; w < words; ++w) {
        if (bitmap[w] == 0) continue;          /* no bit set in this word */
        for (unsigned b = 0; b < 32u; ++b) {
            if (bitmap[w] & (1u << b)) {
                out[k] = (uint32_t)(w * 32u + b);
                ++k;
            }
        }
    }
    free(bitmap);
    *count = k;
    if (out_of_range) return ORACLE_KEY_RANGE;
    if (k < n) return ORACLE_DUPLICATE;
    return ORACLE_OK;
}

/* Algorithm 1, first function: for k = 0 .. nbits-1, split the array into
 * the elements whose bit k is 0 and those whose bit k is 1, each part keeping
 * the order it had, and write the zeros back first, then the ones. */
static int paper_split_passes_u32(uint32_t *a, uint64_t n, int nbits) {
    if (n == 0) return ORACLE_OK;
    uint32_t *zeros = (uint32_t *)malloc(n * sizeof(uint32_t));
    uint32_t *ones = (uint32_t *)malloc(n * sizeof(uint32_t));
    if (zeros == NULL || ones == NULL) { free(zeros); free(ones); return ORACLE_NOMEM; }
    for (int k = 0; k < nbits; ++k) {
        uint64_t n0 = 0, n1 = 0;
        for (uint64_t i = 0; i < n; ++i) {
            if (a[i] & (1u << k)) { ones[n1] = a[i]; ++n1; }
            else                  { zeros[n0] = a[i]; ++n0; }
        }
        for (uint64_t i = 0; i < n0; ++i) a[i] = zeros[i];
        for (uint64_t i = 0; i < n1; ++i) a[n0 + i] = ones[i];
    }
    free(zeros);
    free(ones);
    return ORACLE_OK;
}

/* Algorithm 1 for unsigned 32-bit keys, in place, with `nbits` passes
 * (32 sorts every uint32; 31 is the paper's t-1 bound, which leaves bit 31
 * unexamined). */
int oracle_paper_sort_u32(uint32_t *a, uint64_t n, int nbits) {
    if (nbits < 0 || nbits > 32) return -1;
    return paper_split_passes_u32(a, n, nbits);
}

/* Algorithm 1, second function, for signed 32-bit keys, in place:
 * negatives and non-negatives are separated in their input order, each part
 * is sorted by the first function over bits 0 .. t-2 (t = 32; two's
 * complement, so the low 31 bits of a negative value order it among the
 * negatives), and the negatives are written before the non-negatives. */
int oracle_paper_sort_i32(int32_t *a, uint64_t n) {
    if (n == 0) return ORACLE_OK;
    uint32_t *neg = (uint32_t *)malloc(n * sizeof(uint32_t));
    uint32_t *pos = (uint32_t *)malloc(n * sizeof(uint32_t));
    if (neg == NULL || pos == NULL) { free(neg); free(pos); return ORACLE_NOMEM; }
    uint64_t nm = 0, np = 0;
    for (uint64_t i = 0; i < n; ++i) {
        if (a[i] < 0) { neg[nm] = (uint32_t)a[i]; ++nm; }
        else          { pos[np] = (uint32_t)a[i]; ++np; }
    }
    int rc = paper_split_passes_u32(neg, nm, 31);
    if (rc == ORACLE_OK) rc = paper_split_passes_u32(pos, np, 31);
    if (rc == ORACLE_OK) {
        for (uint64_t i = 0; i < nm; ++i) a[i] = (int32_t)neg[i];
        for (uint64_t i = 0; i < np; ++i) a[nm + i] = (int32_t)pos[i];
    }
    free(neg);
    free(pos);
    return rc;
}

/* Bitmap sort of signed 32-bit keys in [min_value, max_value]: every key is
 * moved to the unsigned offset x - min_value (computed in 64 bits), sorted by
 * oracle_bitmap_sort, and moved back.  Negative values come first, as in
 * Algorithm 1's second function. */
int oracle_bitmap_sort_i32(const int32_t *keys, uint64_t n, int32_t min_value, int32_t max_value,
                           int32_t *out, uint64_t *count) {
    if (max_value < min_value) return -1;
    uint32_t *shifted = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
    if (shifted == NULL) return ORACLE_NOMEM;
    int below = 0;
    for (uint64_t i = 0; i < n; ++i) {
        int64_t d = (int64_t)keys[i] - (int64_t)min_value;
        if (d < 0) { below = 1; d = (int64_t)max_value - (int64_t)min_value + 1; } /* skipped below */
        shifted[i] = d > (int64_t)UINT32_MAX ? UINT32_MAX : (uint32_t)d;
    }
    uint32_t span = (uint32_t)((int64_t)max_value - (int64_t)min_value);
    int rc = oracle_bitmap_sort(shifted, n, span, (uint32_t *)out, count);
    for (uint64_t i = 0; i < *count; ++i)
        out[i] = (int32_t)((int64_t)((uint32_t *)out)[i] + (int64_t)min_value);
    free(shifted);
    if (rc == ORACLE_NOMEM) return rc;
    if (below) return ORACLE_KEY_RANGE;
    return rc;
}

/* Bitmap sort of n 64-bit keys bounded by max_value: the same three steps
 * as oracle_bitmap_sort over M = max_value + 1 values, with 64-bit keys and
 * outputs (the bitmap has ceil(M / 32) words; max_value < 2^40 keeps it
 * below 16 GiB, larger bounds are refused with -1). */
int oracle_bitmap_sort_u64(const uint64_t *keys, uint64_t n, uint64_t max_value,
                           uint64_t *out, uint64_t *count) {
    if (max_value >= (1ull << 40)) return -1;
    uint64_t M = max_value + 1u;
    uint64_t words = (M + 31u) / 32u;
    uint32_t *bitmap = (uint32_t *)calloc(words, sizeof(uint32_t));
    if (bitmap == NULL) return ORACLE_NOMEM;
    int out_of_range = 0;
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t x = keys[i];
        if (x > max_value) { out_of_range = 1; continue; }
        bitmap[x / 32u] = bitmap[x / 32u] | (1u << (x % 32u));
    }
    uint64_t k = 0;
    for (uint64_t w = 0; w < words; ++w) {
        if (bitmap[w] == 0) continue;
        for (unsigned b = 0; b < 32u; ++b) {
            if (bitmap[w] & (1u << b)) {
                out[k] = w * 32u + b;
                ++k;
            }
        }
    }
    free(bitmap);
    *count = k;
    if (out_of_range) return ORACLE_KEY_RANGE;
    if (k < n) return ORACLE_DUPLICATE;
    return ORACLE_OK;
}
