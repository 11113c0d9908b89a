"""kc_census_static -- the census for callers that cannot allocate memory.

Some callers (a hook inside the application's allocator, a post-failure
snapshot handler, a process whose device memory is fully reserved) cannot
call cudaMalloc.  kc_census_static serves them with all scratch in one static
device array.  These tests call it through the C ABI twice in a row and
check that each call gives exactly what the regular, context-based
kc_census gives on the same regions (hits and counts are integers: exact
equality), so a stale array from the previous call cannot go unnoticed; and
that requests beyond its stated limits are refused before any work.

This file is named to be collected last.
"""
import numpy as np
import pytest
import torch

from paper_2605_03208_gb300 import kc
from paper_2605_03208_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _snapshot(seed, p_ptr):
    layout = W.tiny_layout(seed, n=12, total=6 * W.MiB)
    dev = [torch.empty(int(s), dtype=torch.uint8, device="cuda") for s in layout.sizes]
    snap = W.tiny_fill(layout, [t.data_ptr() for t in dev], seed, p_ptr=p_ptr)
    for t, r in zip(dev, snap.regions):
        t.copy_(torch.from_numpy(r))
    torch.cuda.synchronize()
    return snap, dev


def _run(fn, snap, dev, cap):
    b = kc.bufs([(t.data_ptr(), t.numel(), kc.RAW, 0) for t in dev])
    win = W.default_window(snap.bases, snap.sizes)
    hits = torch.full((max(cap, 1) * 24,), 0x5A, dtype=torch.uint8, device="cuda")
    counts = torch.full((2,), -1, dtype=torch.int64, device="cuda")
    st = fn(b, win, hits, cap, counts)
    torch.cuda.synchronize()
    c = counts.cpu().numpy().view(np.uint64)
    n = int(c[0] + c[1])
    return st, (int(c[0]), int(c[1])), hits.cpu().numpy().view(kc.HIT_DTYPE)[: min(n, cap)]


def test_static_census_matches_context_census_twice():
    kc.load()
    ctx = kc.Context(0)
    regular = lambda b, w, h, cap, c: ctx.census(b, w[0], w[1], h, cap, c)    # noqa: E731
    static = lambda b, w, h, cap, c: kc.census_static(b, w[0], w[1], h, cap, c)  # noqa: E731
    # two different snapshots in a row: the second call must not see the first's state
    for seed, p_ptr in ((0, 0.3), (1, 0.05)):
        snap, dev = _snapshot(seed, p_ptr)
        cap = sum(int(s) // 8 for s in snap.sizes)
        st_r, cnt_r, hits_r = _run(regular, snap, dev, cap)
        assert ctx.sync() == kc.OK
        st_s, cnt_s, hits_s = _run(static, snap, dev, cap)
        assert st_r == kc.OK and st_s == kc.OK
        assert cnt_s == cnt_r and sum(cnt_r) > 1000
        assert hits_s.tobytes() == hits_r.tobytes()
        # truncated list: true counts, first `cap` hits
        st_s, cnt_t, hits_t = _run(static, snap, dev, 100)
        assert st_s == kc.OK and cnt_t == cnt_r
        assert hits_t.tobytes() == hits_r[:100].tobytes()
    ctx.close()


def test_static_census_refuses_requests_beyond_its_limits():
    kc.load()
    counts = torch.zeros(2, dtype=torch.int64, device="cuda")
    base = torch.empty(4096, dtype=torch.uint8, device="cuda")
    # 1025 regions (limit 1024); nothing is launched
    too_many = kc.bufs([(base.data_ptr() + 0, 16)] * 1025)
    assert kc.census_static(too_many, 0, 0, None, 0, counts) == kc.EINVAL
    # more than 65536 chunks of 64 KiB: a 5 GiB descriptor is rejected on the host
    huge = kc.bufs([(base.data_ptr(), 5 * W.GiB)])
    assert kc.census_static(huge, 0, 0, None, 0, counts) == kc.EINVAL
