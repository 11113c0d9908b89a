"""Host-side logic of the batched form: autotune cache keys and the cache
file round trip (no GPU needed)."""
from __future__ import annotations

import json

import pytest

B = pytest.importorskip("paper_2605_03208_gb300.batch")


def test_size_class_buckets():
    a = B.size_class([256, 1024, 64 << 20] * 1365)
    b = B.size_class([300, 1000, 60 << 20] * 1400)
    assert a == b                                    # same powers of two
    assert B.size_class([4096]) != B.size_class([4096] * 4096)
    assert B.size_class([1 << 20]) != B.size_class([1 << 30])


def test_cache_round_trip(tmp_path):
    p = str(tmp_path / "sub" / "tune.json")
    assert B.load_cache(p) == {}
    c = {"GB300|digest+compare|x": {"page_bytes": 65536, "warps": 8, "stages": 3, "chunk": 1024, "ms": 1.5}}
    B.save_cache(c, p)
    assert B.load_cache(p) == c
    with open(p, "w") as f:
        f.write("{not json")
    assert B.load_cache(p) == {}                    # a damaged cache is ignored, not fatal
    B.save_cache(c, p)
    assert json.load(open(p)) == c


def test_search_grid():
    assert B.PAGE_SIZES[0] == 4096 and B.PAGE_SIZES[-1] == 2 << 20 and len(B.PAGE_SIZES) == 10
    assert all(32 * w in (128, 256, 512) for w in B.WARPS)
