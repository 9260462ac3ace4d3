"""Host logic of the planner on the CPU, through the C ABI entry point
bitsort_plan_rule (no GPU, no context): the plan rules for the benchmark's
sizes, invariants of every plan over a sweep of sizes, and argument checks."""
import pytest

import paper_1312_0138_gb300 as bs

SMS, SMEM = 152, 232448     # GB300: SMs, opt-in shared memory per block (227 KiB)
GIB = 1 << 30


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_1312_0138_gb300 import builder
    return bs.load(builder.build())


def plan(n, M, sms=SMS, smem=SMEM):
    return bs.plan_rule(sms, smem, n, M - 1)


def test_small_range_global_l2_bitmap():
    # n = 10^5 keys over 2^20 values: the bitmap (128 KiB) stays in L2, keys
    # are OR-ed straight into it and it is scanned in 16 Ki-value slices
    cfg, sh = plan(100_000, 1 << 20)
    assert cfg["path"] == "global" and cfg["slice_values"] == 1 << 14 and sh["slices"] == 64
    assert cfg["threads"] == 512 and sh["scratch_bytes"] == 0


def test_tiny_range_fused():
    for n, M in [(1, 1), (100, 4096), (5000, 1 << 17), (1 << 16, 1 << 20)]:
        cfg, sh = plan(n, M)
        assert cfg["path"] == "fused" and sh["slices"] == 1 and cfg["slice_values"] >= M, (n, M)


def test_dense_2e24_over_2e28_two_slices_per_sm():
    # 2^24 keys over 2^28 values: partition, capacity layout, 2 x 152 slices
    cfg, sh = plan(1 << 24, 1 << 28)
    assert cfg["path"] == "partition" and cfg["layout"] == "capacity"
    assert sh["slices"] == 2 * SMS
    assert cfg["slice_values"] == 883_072     # ceil(2^28 / 304) rounded up to 128
    assert cfg["stage"] == 0                   # density 1/16: lanes store their own positions
    # wide partition tiles of 16 Ki keys at 512 threads (1024 tiles, four or more per SM)
    assert sh["part_threads"] == 512 and sh["bucket_threads"] == 512 and sh["tile_keys"] == 16384
    assert sh["scratch_bytes"] == 304 * 883_072 * 4


def test_sparse_full_range_exact_layout_wide_phases():
    # 2^24 keys over 2^32 values: 4096 slices of 2^20 values; a capacity
    # buffer (16 GiB) would exceed 4 GiB and twice the keys' bytes, so the
    # partition runs in the exact layout; both wide phases run at 1024 threads
    cfg, sh = plan(1 << 24, 1 << 32)
    assert cfg["path"] == "partition" and cfg["layout"] == "exact" and sh["scratch_bytes"] == 0
    assert cfg["slice_values"] == 1 << 20 and sh["slices"] == 4096
    assert sh["part_threads"] == 1024 and sh["tile_keys"] == 32768   # wide tiles: 512, 3.4 per SM
    assert sh["bucket_threads"] == 1024


def test_dense_full_range_capacity_layout():
    # 2^31 keys over 2^32 values (density 1/2): the 16 GiB capacity buffer is
    # twice the keys' bytes, which the rule allows; positions are staged
    cfg, sh = plan(1 << 31, 1 << 32)
    assert cfg["path"] == "partition" and cfg["layout"] == "capacity"
    assert sh["scratch_bytes"] == 16 * GIB
    assert cfg["stage"] == 1 and sh["part_threads"] == 1024 and sh["bucket_threads"] == 512
    assert sh["tile_keys"] == 32768   # wide partition tiles


NS = [1, 2, 31, 32, 33, 1000, 4097, 65_536, 65_537, 100_000, 1 << 20, (1 << 20) + 1, 1 << 22, 1 << 24, 1 << 26,
      1 << 28, 1 << 31, 1 << 32]
MS = [1, 2, 100, 4096, 1 << 17, (1 << 17) + 1, 1 << 20, (1 << 20) + 1, 1 << 22, (1 << 22) + 3, 1 << 24, 1 << 28,
      1 << 31, 1 << 32]


@pytest.mark.parametrize("sms", [1, 8, SMS])
def test_plan_invariants(sms):
    seen = set()
    for M in MS:
        for n in NS:
            if n > M:
                continue
            cfg, sh = plan(n, M, sms=sms)
            S = cfg["slice_values"]
            seen.add(cfg["path"])
            where = (n, M, sms, cfg, sh)
            assert sh["smem_bytes"] <= SMEM, where
            assert S % 128 == 0 and S >= 128, where
            assert cfg["threads"] in (256, 512, 1024), where
            assert sh["part_threads"] in (256, 512, 1024) and sh["bucket_threads"] in (256, 512, 1024), where
            # wide partition tiles (32 keys a thread) at 512 or 1024 threads
            # where they fit the shared memory and give every SM four (512)
            # or three (1024) or more
            pt = sh["part_threads"]
            wide = (cfg["path"] == "partition" and pt in (512, 1024)
                    and -(-n // (32 * pt)) >= (3 if pt == 1024 else 4) * sms
                    and ((sh["slices"] + 4) & ~3) * 16 + 32 * pt * 4 + 16 <= SMEM)
            assert sh["tile_keys"] == (32 if wide else 16) * pt, where
            if cfg["path"] == "fused":
                assert M <= 1 << 20 and S >= M and sh["slices"] == 1, where
                continue
            assert S <= 1 << 20, where
            assert sh["slices"] == -(-M // S) <= 8192, where
            if cfg["path"] == "partition":
                cap_bytes = sh["slices"] * min(S, n) * 4
                if cfg["layout"] == "capacity":
                    assert sh["scratch_bytes"] == cap_bytes <= max(4 * GIB, 8 * n), where
                else:
                    assert sh["scratch_bytes"] == 0 and cap_bytes > max(4 * GIB, 8 * n), where
                assert cfg["stage"] <= int(10 * n >= M), where   # no staging below one key per ten values
            else:
                assert cfg["path"] == "global" and M <= 1 << 22 and n <= 1 << 20, where
    assert seen == {"fused", "global", "partition"}


def test_invalid_arguments():
    for args in [(0, SMEM, 10, 99), (SMS, 0, 10, 99), (SMS, SMEM, 101, 99)]:
        with pytest.raises(bs.BitsortError) as e:
            bs.plan_rule(*args)
        assert e.value.status == bs.ERR_INVALID, args
