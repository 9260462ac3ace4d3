"""Checks that pin the CPU oracle to facts fixed by the paper and by plain
mathematics, independently of the oracle itself.

Each ``check_*`` function takes an :class:`oracle.Oracle` and raises
``AssertionError`` on a mismatch.  ``test_oracle_pins.py`` runs them on the
real oracle; ``test_oracle_mutants.py`` runs them on copies of the oracle with
a planted mistake and requires that at least one check fails for every copy.

What pins what:
* Table I (golden file)            -> the OR used to set bits; Example 1 bit test.
* Table II (golden file)           -> the two's-complement pattern (Example 4)
                                      behind the signed split of Algorithm 1.
* brute force over every subset    -> the bitmap sort, all bit/word positions,
  of [0, M), M <= 12, several orders  expected value built from the subset mask
                                      by enumeration, no sort involved.
* closed form                      -> a permutation of [0, M) sorts to 0..M-1.
* library sort (numpy)             -> large random inputs, incl. keys >= 2^31
                                      and max_value = 2^32 - 1.
* invariants                       -> strictly increasing, length, membership.
* Theorem 1's induction invariant  -> after pass s of Algorithm 1 the values
                                      mod 2^(s+1) are non-decreasing.
* error semantics                  -> duplicates / out-of-range keys.
"""
from __future__ import annotations

import itertools

import numpy as np

import gen
from conftest import read_golden

OK, KEY_RANGE, DUPLICATE = 0, 2, 3
U32MAX = (1 << 32) - 1


def check_table1_or(o):
    for xb, yb, _and, orr, _xor, _notx in read_golden("table1_bitwise_ops.txt"):
        xb, yb, orr = int(xb), int(yb), int(orr)
        for i in (0, 1, 5, 17, 30, 31):
            z = o.bit_or(xb << i, yb << i)
            assert o.bit_value(z, i) == orr, ("Table I OR", xb, yb, i)
            assert z == (orr << i), ("OR leaked into other bits", xb, yb, i, z)


def check_bit_value_positions(o):
    # Section II numbering: bit 0 is the rightmost one; 2^i has only bit i set.
    for i in range(32):
        x = 1 << i
        for j in range(32):
            assert o.bit_value(x, j) == (1 if i == j else 0), (i, j)
    assert o.bit_value(0b1011, 0) == 1 and o.bit_value(0b1011, 2) == 0


def check_table2_patterns(o):
    for value, pattern in read_golden("table2_short_patterns.txt"):
        v = int(value)
        if v > 32767:              # stored as a short it wraps (printed that way)
            v -= 65536
        assert o.bin_repl_i16(v) == pattern, (value, pattern, o.bin_repl_i16(v))


def _expected_from_mask(mask: int, M: int):
    return [v for v in range(M) if (mask >> v) & 1]


def check_brute_force_subsets(o, max_M: int = 10, orders: int = 3):
    for M in range(1, max_M + 1):
        for mask in range(1 << M):
            members = _expected_from_mask(mask, M)
            for r in range(orders):
                keys = gen.shuffle(1000 * M + 7 * mask + r, np.array(members, dtype=np.uint32))
                st, out = o.bitmap_sort(keys, M - 1)
                assert st == OK, (M, mask, r, st)
                assert out.tolist() == members, (M, mask, r, keys.tolist(), out.tolist())


def check_all_permutations_small(o):
    for members in ([0], [3, 1], [0, 5, 2], [7, 0, 31, 32], [1, 33, 64, 95, 2], [0, 1, 2, 3, 4, 63]):
        want = sorted(members)
        mv = max(members)
        for perm in itertools.permutations(members):
            st, out = o.bitmap_sort(np.array(perm, dtype=np.uint32), mv)
            assert st == OK and out.tolist() == want, (perm, out.tolist())


def check_closed_form_permutation(o):
    for M in (1, 2, 31, 32, 33, 63, 64, 65, 1000, 4096, 1 << 20):
        keys = gen.feistel(M, M, M)            # a permutation of [0, M)
        st, out = o.bitmap_sort(keys, M - 1)
        assert st == OK
        assert np.array_equal(out, np.arange(M, dtype=np.uint32)), M


def check_against_library_sort(o):
    cases = [(1000, 1 << 12), (100_000, 1 << 20), (50_000, 1 << 32), (3, 1 << 32),
             (4096, 4096), (777, 1 << 31), (20_000, (1 << 31) + 12345)]
    for i, (n, M) in enumerate(cases):
        keys = gen.floyd(17 + i, n, M)
        st, out = o.bitmap_sort(keys, M - 1)
        assert st == OK, (n, M, st)
        assert np.array_equal(out, np.sort(keys)), (n, M)


def check_invariants(o):
    for i, (n, M) in enumerate([(1, 1), (10, 10), (5000, 1 << 16), (30_000, 1 << 32)]):
        keys = gen.floyd(99 + i, n, M)
        st, out = o.bitmap_sort(keys, M - 1)
        assert st == OK
        assert out.size == n
        assert np.all(out[1:] > out[:-1])
        assert np.all(np.isin(out, keys))


def check_edge_cases(o):
    st, out = o.bitmap_sort(np.array([], dtype=np.uint32), 0)
    assert st == OK and out.size == 0
    st, out = o.bitmap_sort(np.array([0], dtype=np.uint32), 0)
    assert st == OK and out.tolist() == [0]
    st, out = o.bitmap_sort(np.array([5], dtype=np.uint32), 5)
    assert st == OK and out.tolist() == [5]
    top = np.array([U32MAX, 0, 1 << 31, (1 << 31) - 1, U32MAX - 1], dtype=np.uint32)
    st, out = o.bitmap_sort(top, U32MAX)
    assert st == OK and out.tolist() == [0, (1 << 31) - 1, 1 << 31, U32MAX - 1, U32MAX]
    # keys exactly at max_value are in range; max_value + 1 is not
    st, out = o.bitmap_sort(np.array([9, 0, 10, 4], dtype=np.uint32), 9)
    assert st == KEY_RANGE and out.tolist() == [0, 4, 9]
    st, out = o.bitmap_sort(np.array([9, 0, 4], dtype=np.uint32), 9)
    assert st == OK and out.tolist() == [0, 4, 9]


def check_duplicates(o):
    keys = gen.uniform_with_replacement(5, 20_000, 1 << 14)
    st, out = o.bitmap_sort(keys, (1 << 14) - 1)
    uniq = np.unique(keys)
    assert uniq.size < keys.size
    assert st == DUPLICATE
    assert np.array_equal(out, uniq)
    st, out = o.bitmap_sort(np.array([3, 3], dtype=np.uint32), 3)
    assert st == DUPLICATE and out.tolist() == [3]
    # a key out of range outranks a duplicate in the status
    st, out = o.bitmap_sort(np.array([3, 3, 8], dtype=np.uint32), 7)
    assert st == KEY_RANGE and out.tolist() == [3]


def check_paper_algorithm(o):
    for i, (n, M) in enumerate([(1, 2), (100, 1 << 8), (20_000, 1 << 32), (5000, 1 << 20)]):
        keys = gen.floyd(300 + i, n, M)
        b = o.paper_sort_u32(keys, 32)
        assert np.array_equal(b, np.sort(keys))
        st, a = o.bitmap_sort(keys, M - 1)
        assert np.array_equal(a, b)
    # Algorithm 1 keeps duplicates: it sorts the multiset
    keys = gen.uniform_with_replacement(6, 5000, 300)
    assert np.array_equal(o.paper_sort_u32(keys, 32), np.sort(keys))


def check_theorem1_invariant(o):
    keys = gen.uniform_with_replacement(8, 3000, 1 << 32)
    for s in range(32):
        a = o.paper_sort_u32(keys, s + 1)     # the array after pass s
        low = a.astype(np.uint64) % (1 << (s + 1))
        assert np.all(low[1:] >= low[:-1]), s
        assert np.array_equal(np.sort(a), np.sort(keys))   # a permutation


def check_paper_signed(o):
    vals = gen.uniform_with_replacement(9, 20_000, 1 << 32).view(np.int32)
    vals = np.concatenate([vals, np.array([-(1 << 31), (1 << 31) - 1, 0, -1], dtype=np.int32)])
    assert np.array_equal(o.paper_sort_i32(vals), np.sort(vals))
    distinct = gen.floyd(10, 10_000, 1 << 32).view(np.int32)
    st, out = o.bitmap_sort_i32(distinct, -(1 << 31), (1 << 31) - 1)
    assert st == OK and np.array_equal(out, np.sort(distinct))
    st, out = o.bitmap_sort_i32(np.array([-5, 7, -3, 2], dtype=np.int32), -4, 7)
    assert st == KEY_RANGE and out.tolist() == [-3, 2, 7]


def check_bitmap_u64(o):
    # brute force over every subset of [0, M) for small M, in shuffled order
    for M in range(1, 9):
        for mask in range(1 << M):
            keys = np.array([v for v in range(M) if mask >> v & 1], dtype=np.uint64)
            keys = gen.shuffle(mask + 77, keys.astype(np.uint32)).astype(np.uint64)
            st, out = o.bitmap_sort_u64(keys, M - 1)
            assert st == OK and out.tolist() == _expected_from_mask(mask, M)
    # values above 2^32: the library sort of distinct keys
    base = gen.floyd(11, 20_000, 1 << 32).astype(np.uint64)
    keys = (base << np.uint64(2)) | (base & np.uint64(3))          # distinct values below 2^34
    st, out = o.bitmap_sort_u64(keys, (1 << 34) - 1)
    assert st == OK and np.array_equal(out, np.sort(keys))
    assert int(out[-1]) >= (1 << 32)
    # a key above max_value is skipped and reported, also one that only
    # differs above bit 31
    st, out = o.bitmap_sort_u64(np.array([5, (1 << 32) + 5, 7], dtype=np.uint64), 100)
    assert st == KEY_RANGE and out.tolist() == [5, 7]
    st, out = o.bitmap_sort_u64(np.array([3, 3, 1], dtype=np.uint64), 3)
    assert st == DUPLICATE and out.tolist() == [1, 3]
    # below 2^32 it agrees with the 32-bit form
    k32 = gen.floyd(12, 5_000, 1 << 20)
    st32, o32 = o.bitmap_sort(k32, (1 << 20) - 1)
    st64, o64 = o.bitmap_sort_u64(k32.astype(np.uint64), (1 << 20) - 1)
    assert st32 == st64 == OK and np.array_equal(o32.astype(np.uint64), o64)


ALL_CHECKS = [
    check_table1_or, check_bit_value_positions, check_table2_patterns,
    check_brute_force_subsets, check_all_permutations_small, check_closed_form_permutation,
    check_against_library_sort, check_invariants, check_edge_cases, check_duplicates,
    check_paper_algorithm, check_theorem1_invariant, check_paper_signed, check_bitmap_u64,
]
