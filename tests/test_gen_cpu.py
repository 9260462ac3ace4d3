"""The seeded input generators (gen/), which the oracle side and the GPU side
both draw from, checked on the CPU against what their recipes promise:
distinct keys in range, bijections with working inverses, reproducibility,
uniformity within loose statistical bounds, and the workload recipes'
bounds."""
import math

import numpy as np
import pytest

import gen


def test_floyd_distinct_in_range_reproducible():
    for n, M in [(1, 1), (5, 5), (1000, 1000), (1000, 1 << 20), (100_000, 1 << 20), (4097, 1 << 32)]:
        a = gen.floyd(7, n, M)
        assert a.size == n and np.unique(a).size == n, (n, M)
        assert int(a.max()) < M
        assert np.array_equal(a, gen.floyd(7, n, M))
    assert not np.array_equal(gen.floyd(7, 1000, 1 << 20), gen.floyd(8, 1000, 1 << 20))
    # n = M draws every value: a permutation, and a shuffled one
    p = gen.floyd(3, 4096, 4096)
    assert np.array_equal(np.sort(p), np.arange(4096, dtype=np.uint32))
    assert not np.array_equal(p, np.arange(4096, dtype=np.uint32))
    with pytest.raises(ValueError):
        gen.floyd(1, 11, 10)


def test_floyd_is_uniform_over_values():
    # 2^16 draws from [0, 2^20): every 1/16 of the range holds 1/16 of the keys
    a = gen.floyd(11, 1 << 16, 1 << 20)
    counts = np.bincount(a >> 16, minlength=16)
    expect = (1 << 16) / 16
    chi2 = float(((counts - expect) ** 2 / expect).sum())
    assert chi2 < 50.0, counts        # 15 degrees of freedom: P(chi2 > 50) < 1e-5


@pytest.mark.parametrize("M", [1, 2, 3, 7, 1000, (1 << 16) + 1, 1 << 20])
def test_feistel_is_a_bijection_with_inverse(M):
    p = gen.feistel(5, M, M)
    assert np.array_equal(np.sort(p), np.arange(M, dtype=np.uint32))
    inv = gen.feistel_inverse(5, M, p)
    assert np.array_equal(inv, np.arange(M, dtype=np.uint64))


def test_feistel_prefix_start_and_seeds():
    M = 1 << 24
    full = gen.feistel(9, 1 << 16, M)
    assert np.unique(full).size == full.size and int(full.max()) < M
    # a window starting at `start` is the same slice of the one sequence
    assert np.array_equal(gen.feistel(9, 1000, M, start=5000), full[5000:6000])
    assert not np.array_equal(full[:1000], gen.feistel(10, 1000, M))
    # keys of the full 32-bit range, inverted
    big = gen.feistel(2, 4096, 1 << 32)
    assert np.array_equal(gen.feistel_inverse(2, 1 << 32, big), np.arange(4096, dtype=np.uint64))
    with pytest.raises(ValueError):
        gen.feistel(1, 10, 9)


def test_shuffle_is_a_permutation():
    a = np.arange(10_000, dtype=np.uint32) * 3
    b = gen.shuffle(4, a)
    assert np.array_equal(np.sort(b), a) and not np.array_equal(a, b)
    assert np.array_equal(b, gen.shuffle(4, a))


def test_uniform_with_replacement():
    a = gen.uniform_with_replacement(12, 200_000, 10)
    assert int(a.max()) <= 9
    counts = np.bincount(a, minlength=10)
    chi2 = float(((counts - 20_000) ** 2 / 20_000).sum())
    assert chi2 < 40.0, counts        # 9 degrees of freedom
    full = gen.uniform_with_replacement(13, 1 << 16, 1 << 32)
    assert int(full.max()) >= 1 << 31  # the top bit is drawn too


def test_unit_doubles():
    u = gen.unit(14, 100_000)
    assert float(u.min()) >= 0.0 and float(u.max()) < 1.0
    assert abs(float(u.mean()) - 0.5) < 0.01
    assert np.array_equal(u, gen.unit(14, 100_000))


def test_keys_recipe_dispatch():
    assert np.array_equal(gen.keys(1, 100, 1000), gen.floyd(1, 100, 1000))
    assert np.array_equal(gen.keys(1, 100, 1000, "feistel"), gen.feistel(1, 100, 1000))
    with pytest.raises(ValueError):
        gen.keys(1, 10, 100, "other")


def test_batch_spec_bounds():
    spec = gen.batch_spec(0x13120138 + 3, 4096)
    assert len(spec) == 4096
    for n, M in spec:
        assert (1 << 10) <= n <= (1 << 22)
        assert max(1 << 12, 2 * n) <= M <= min(1 << 26, 64 * n), (n, M)
    ns = np.array([n for n, _ in spec], dtype=np.float64)
    # log-uniform over [2^10, 2^22]: the mean of log2 n is near 16
    assert abs(float(np.log2(ns).mean()) - 16.0) < 0.3
    assert 1.9e9 < ns.sum() < 2.3e9


def test_serve_spec_bounds():
    reqs = gen.serve_spec(0x13120138 + 4, 300, 200.0)
    times = [t for t, _, _ in reqs]
    assert all(b > a for a, b in zip(times, times[1:]))
    for _, n, M in reqs:
        assert (1 << 10) <= n <= (1 << 26) and (1 << 16) <= M <= (1 << 32) and n <= M // 2
    # Poisson arrivals at 200/s: 300 requests take about 1.5 s
    assert 1.0 < times[-1] < 2.0
    assert math.isclose(gen.log_uniform_int(0.0, 4, 64), 4) and gen.log_uniform_int(0.9999999, 4, 64) == 63
