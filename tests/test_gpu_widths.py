"""Parity of the bitmap sort for 16-, 8- and 64-bit keys (bitsort_u16,
bitsort_u8, bitsort_u64) with the CPU oracle, through the C ABI."""
import numpy as np
import pytest

import gen
import oracle
import paper_1312_0138_gb300 as bs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    bs.load()
    c = bs.Context(0)
    yield c
    c.close()


TORCH_VIEW = {np.uint16: np.int16, np.uint8: np.uint8, np.uint64: np.int64}


def gpu_width(ctx, keys, max_value, inplace=False):
    import torch
    dt = keys.dtype.type
    d = torch.from_numpy(np.ascontiguousarray(keys).view(TORCH_VIEW[dt]).copy()).cuda()
    out = d if inplace else torch.empty_like(d)
    st, cnt, out = ctx.sort_width(d, max_value, out=out)
    assert st != bs.ERR_TIMEOUT
    return st, cnt, out.cpu().numpy().view(dt)[:cnt]


def check(ctx, keys, max_value, inplace=False):
    if keys.dtype == np.uint64:
        want_st, want = oracle.default().bitmap_sort_u64(keys, max_value)
    else:   # the same bitmap sort of the same values, stored in 32 bits
        want_st, want = oracle.bitmap_sort(keys.astype(np.uint32), max_value)
    st, cnt, got = gpu_width(ctx, keys, max_value, inplace)
    assert st == want_st, (st, want_st)
    assert cnt == want.size
    assert np.array_equal(got.astype(np.uint64), want.astype(np.uint64))
    return st


@pytest.mark.parametrize("n,max_value", [(1, 0), (300, 65535), (40_000, 65535), (65_536, 65535), (5_000, 9_999),
                                         (33, 40)])
@pytest.mark.parametrize("inplace", [False, True])
def test_u16(ctx, n, max_value, inplace):
    keys = gen.keys(gen.SEED_BASE + 500 + n, n, max_value + 1).astype(np.uint16)
    assert check(ctx, keys, max_value, inplace) == bs.OK


@pytest.mark.parametrize("n,max_value", [(1, 0), (256, 255), (100, 255), (17, 30)])
def test_u8(ctx, n, max_value):
    keys = gen.keys(gen.SEED_BASE + 600 + n, n, max_value + 1).astype(np.uint8)
    assert check(ctx, keys, max_value) == bs.OK


def test_small_width_errors(ctx):
    keys = np.array([5, 9, 5, 1], np.uint16)
    assert check(ctx, keys, 10) == bs.ERR_DUPLICATE
    keys = np.array([5, 900, 1], np.uint16)
    assert check(ctx, keys, 100) == bs.ERR_KEY_RANGE
    keys = np.array([200, 3, 7], np.uint8)
    assert check(ctx, keys, 150) == bs.ERR_KEY_RANGE
    import torch
    with pytest.raises(bs.BitsortError):   # 5 keys cannot be distinct among 4 values
        ctx.sort_width_async(torch.zeros(5, dtype=torch.int16, device="cuda"), 3)


@pytest.mark.parametrize("n,max_value", [(1000, (1 << 20) - 1), (1 << 20, (1 << 28) - 1),
                                         (300_001, (1 << 32) - 1), (7, 6)])
@pytest.mark.parametrize("inplace", [False, True])
def test_u64(ctx, n, max_value, inplace):
    keys = gen.keys(gen.SEED_BASE + 700 + n, n, max_value + 1).astype(np.uint64)
    assert check(ctx, keys, max_value, inplace) == bs.OK


def test_u64_range_above_32_bits(ctx):
    # a key that differs from an in-range value only above bit 31 is out of range
    base = gen.keys(gen.SEED_BASE + 801, 10_000, 1 << 24).astype(np.uint64)
    keys = base.copy()
    keys[17] = base[17] + (1 << 32)
    assert check(ctx, keys, (1 << 24) - 1) == bs.ERR_KEY_RANGE
    # full 32-bit bound: replaced keys must not show up as 2^32 - 1
    keys = gen.keys(gen.SEED_BASE + 802, 10_000, 1 << 32).astype(np.uint64)
    keys[5] = (1 << 40) + 3
    keys[9] = 1 << 33
    assert check(ctx, keys, (1 << 32) - 1) == bs.ERR_KEY_RANGE
    keys[100] = (1 << 32) - 1   # and a genuine top key stays
    assert check(ctx, keys, (1 << 32) - 1) == bs.ERR_KEY_RANGE
    keys = np.array([3, 3, 1], np.uint64)
    assert check(ctx, keys, 10) == bs.ERR_DUPLICATE


def test_u64_host_errors(ctx):
    import torch
    d = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(bs.BitsortError) as e:
        ctx.sort_width_async(d, 1 << 32)   # bound above 2^32 - 1
    assert e.value.status == bs.ERR_INVALID
    st, cnt, _ = ctx.sort_width(d[:0], 10)
    assert st == bs.OK and cnt == 0
