"""Environment read at context creation (BITSORT_FORCE_PATH,
BITSORT_TUNE_CACHE), checked through the C ABI with parity against the
oracle on the sorts it steers."""
import numpy as np
import pytest

import gen
import oracle
import paper_1312_0138_gb300 as bs
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu


def sorted_ok(ctx, keys, max_value):
    st, cnt, out = ctx.sort(to_dev(keys), max_value)
    want_st, want = oracle.bitmap_sort(keys, max_value)
    assert st == want_st == bs.OK and cnt == want.size
    assert np.array_equal(to_host(out)[:cnt], want)


def test_force_path(monkeypatch):
    keys = gen.floyd(gen.SEED_BASE + 61, 300_000, 1 << 24)
    monkeypatch.setenv("BITSORT_FORCE_PATH", "global")
    c = bs.Context(0)
    try:
        assert c.get_config(1 << 24, (1 << 28) - 1)["path"] == "global"
        assert c.get_config(300_000, (1 << 24) - 1)["path"] == "global"
        sorted_ok(c, keys, (1 << 24) - 1)
    finally:
        c.close()
    # fused is kept only where one shared-memory slice covers the range
    monkeypatch.setenv("BITSORT_FORCE_PATH", "fused")
    c = bs.Context(0)
    try:
        assert c.get_config(300_000, (1 << 24) - 1)["path"] == "partition"
        assert c.get_config(100_000, (1 << 20) - 1)["path"] == "fused"   # the rule's choice: global
        sorted_ok(c, keys, (1 << 24) - 1)
        sorted_ok(c, gen.floyd(gen.SEED_BASE + 62, 100_000, 1 << 20), (1 << 20) - 1)
    finally:
        c.close()
    monkeypatch.setenv("BITSORT_FORCE_PATH", "no-such-path")   # ignored: the rule applies
    c = bs.Context(0)
    try:
        assert c.get_config(1 << 24, (1 << 28) - 1)["path"] == "partition"
    finally:
        c.close()


def test_tune_cache(monkeypatch, tmp_path):
    n, mv = 300_000, (1 << 24) - 1
    path = tmp_path / "tuned.json"
    c = bs.Context(0)
    try:
        c.set_config(n, mv, bs.PATH_GLOBAL, slice_values=1 << 16, threads=256)
        c.tune_save(str(path))
    finally:
        c.close()
    monkeypatch.setenv("BITSORT_TUNE_CACHE", str(path))
    c = bs.Context(0)
    try:
        cfg = c.get_config(n, mv)
        assert cfg["path"] == "global" and cfg["slice_values"] == 1 << 16 and cfg["threads"] == 256
        sorted_ok(c, gen.floyd(gen.SEED_BASE + 63, n, mv + 1), mv)
    finally:
        c.close()
    # a missing file leaves the rule in place and is noted
    monkeypatch.setenv("BITSORT_TUNE_CACHE", str(tmp_path / "missing.json"))
    c = bs.Context(0)
    try:
        assert b"BITSORT_TUNE_CACHE" in bs.load().bitsort_last_error()
        assert c.get_config(n, mv)["path"] == "partition"
    finally:
        c.close()
