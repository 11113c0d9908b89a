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


def test_plan_carves_disjoint_per_job_outputs():
    """make_plan (host marshalling only): each job's page digests start at
    the exclusive scan of the page counts, its record at 64 bytes per job,
    and its descriptor carries the job's own addresses, size and dtype."""
    import numpy as np
    import torch
    from paper_2605_03208_gb300 import kc
    from paper_2605_03208_gb300 import workloads as W
    sizes = [1, 4096, 4097, 65536 * 3 + 17, 256]
    dtypes = [kc.U8, kc.F32, kc.F16, kc.BF16, kc.I32]
    offsets = list(np.concatenate([[0], np.cumsum([(s + 255) // 256 * 256 for s in sizes])])[:-1])
    total = int(offsets[-1]) + (sizes[-1] + 255) // 256 * 256
    js = W.JobSet(sizes, dtypes, offsets, torch.zeros(total, dtype=torch.uint8),
                  torch.zeros(total, dtype=torch.uint8))
    page = 4096
    plan = B.make_plan(js, page, device="cpu")
    npages = [(s + page - 1) // page for s in sizes]
    assert plan.npages == npages
    assert list(plan.pfirst) == [0] + list(np.cumsum(npages))
    hb, zb, cb = plan.hash.data_ptr(), plan.zero.data_ptr(), plan.cmp.data_ptr()
    for k, j in enumerate(plan.jobs):
        assert j.got_va == js.got.data_ptr() + offsets[k] and j.want_va == js.want.data_ptr() + offsets[k]
        assert j.bytes == sizes[k] and j.dtype == dtypes[k]
        assert j.flags == kc.JOB_DIGEST | kc.JOB_COMPARE
        assert j.d_hash == hb + 8 * int(plan.pfirst[k]) and j.d_zero == zb + int(plan.pfirst[k])
        assert j.d_cmp == cb + 64 * k and j.d_done == 0 and j.d_cmp_copy == 0
    assert plan.hash.numel() == plan.total_pages == sum(npages)
    # got and want read once each (the fused pass hashes and compares one read of got)
    assert B.algorithmic_bytes(plan) == 2 * sum(sizes) + 9 * sum(npages) + 64 * len(sizes)
