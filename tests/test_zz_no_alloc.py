"""kc_census_static -- the census for callers that cannot allocate memory.

Some callers (a hook inside the application's allocator, a post-failure
snapshot handler, a process whose device memory is fully reserved) cannot
call cudaMalloc.  kc_census_static serves them with all scratch in one static
device array.  These tests call it through the C ABI twice in a row and check
each call's hits and counts exactly against the CPU oracle and against the
regular, context-based kc_census on the same regions (so a stale array from
the previous call cannot go unnoticed); that after the one-time set-up the
calls leave the device's free memory unchanged; that a lost region, a
window-only snapshot and the largest accepted size give the oracle's
answer; that requests beyond the stated limits are refused before any work
(the over-limit descriptor is backed by a real allocation, so even a
regressed check could not read outside it); and that a call inside a stream
capture is refused.

This file is named to be collected last.
"""
import numpy as np
import pytest
import torch

import oracle
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


def _outputs(cap):
    hits = torch.full((max(cap, 1) * 24,), 0x5A, dtype=torch.uint8, device="cuda")
    counts = torch.full((2,), -1, dtype=torch.int64, device="cuda")
    return hits, counts


def _read(hits, counts, cap):
    torch.cuda.synchronize()
    c = counts.cpu().numpy().view(np.uint64)
    n = int(c[0] + c[1])
    return (int(c[0]), int(c[1])), hits.cpu().numpy().view(kc.HIT_DTYPE)[: min(n, cap)]


def test_static_census_matches_oracle_and_context_twice_without_allocating():
    kc.load()
    assert kc.census_static(None, 0, 0, None, 0, None) == kc.OK   # set-up of this device
    ctx = kc.Context(0)
    snaps = [_snapshot(0, 0.3), _snapshot(1, 0.05)]
    caps = [sum(int(s) // 8 for s in snap.sizes) for snap, _ in snaps]
    outs = [_outputs(cap) for cap in caps] + [_outputs(100), _outputs(100)]
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    # two different snapshots in a row: the second call must not see the first's state;
    # then each again with a list cut at 100 hits
    got = []
    for k, ((snap, dev), cap) in enumerate(list(zip(snaps, caps)) + [(snaps[0], 100), (snaps[1], 100)]):
        b = kc.bufs([(t.data_ptr(), t.numel(), kc.RAW, 0) for t in dev])
        win = W.default_window(snap.bases, snap.sizes)
        hits, counts = outs[k]
        st = kc.census_static(b, win[0], win[1], hits, cap, counts)
        assert st == kc.OK
        got.append(_read(hits, counts, cap))
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes across static calls"
    for k, (snap, dev) in enumerate(snaps):
        win = W.default_window(snap.bases, snap.sizes)
        ohits, nin, nout, _ = oracle.census(snap.regions, snap.bases, *win)
        cnt, hits = got[k]
        assert cnt == (nin, nout) and nin + nout > 1000
        assert hits.tobytes() == ohits.tobytes()
        cnt_t, hits_t = got[k + 2]
        assert cnt_t == (nin, nout)
        assert hits_t.tobytes() == ohits[:100].tobytes()
        # and the context-based census on the same regions
        b = kc.bufs([(t.data_ptr(), t.numel(), kc.RAW, 0) for t in dev])
        hits_r, counts_r = _outputs(caps[k])
        ctx.census(b, win[0], win[1], hits_r, caps[k], counts_r)
        assert ctx.sync() == kc.OK
        cnt_r, hr = _read(hits_r, counts_r, caps[k])
        assert cnt_r == cnt and hr.tobytes() == hits.tobytes()
    ctx.close()


def test_static_census_lost_region_and_window_only_hits():
    kc.load()
    snap, dev = _snapshot(2, 0.3)
    win = W.default_window(snap.bases, snap.sizes)
    cap = sum(int(s) // 8 for s in snap.sizes)
    # region 3 lost: not scanned, still a target
    flags = [kc.BUF_LOST if i == 3 else 0 for i in range(len(dev))]
    b = kc.bufs([(t.data_ptr(), t.numel(), kc.RAW, f) for t, f in zip(dev, flags)])
    hits, counts = _outputs(cap)
    assert kc.census_static(b, win[0], win[1], hits, cap, counts) == kc.EBUF
    cnt, h = _read(hits, counts, cap)
    images = [r if i != 3 else r[:0] for i, r in enumerate(snap.regions)]
    ohits, nin, nout, _ = oracle.census(images, snap.bases, *win, sizes=snap.sizes)
    assert cnt == (nin, nout) and nin > 0
    assert h.tobytes() == ohits.tobytes()
    assert not np.any(h["src_alloc"] == 3) and np.any(h["target"] == 3)
    # the largest region rewritten with words that all lie in the window's
    # margins below the captured span (the other regions lost): outside hits only
    lo, hi = win
    span_lo = min(snap.bases)
    k = int(np.argmax(snap.sizes))
    nv = min(4096, int(snap.sizes[k]) // 8)
    vals = np.linspace(lo, span_lo - 8, nv, dtype=np.uint64) // np.uint64(8) * np.uint64(8)
    dev[k][: nv * 8].copy_(torch.from_numpy(vals.view(np.uint8)))
    sizes = [nv * 8 if i == k else int(s) for i, s in enumerate(snap.sizes)]
    images = [snap.regions[k][:0].copy() for _ in snap.regions]
    images[k] = vals.view(np.uint8).copy()
    b = kc.bufs([(t.data_ptr(), sizes[i], kc.RAW, 0 if i == k else kc.BUF_LOST) for i, t in enumerate(dev)])
    hits, counts = _outputs(cap)
    assert kc.census_static(b, lo, hi, hits, cap, counts) == kc.EBUF
    cnt, h = _read(hits, counts, cap)
    ohits, nin, nout, _ = oracle.census(images, snap.bases, lo, hi, sizes=sizes)
    assert cnt == (nin, nout) == (0, nv)
    assert h.tobytes() == ohits.tobytes() and np.all(h["target"] == -1)


def test_static_census_largest_size_and_limits():
    """Exactly 65536 chunks of 64 KiB (4 GiB) are accepted and match the
    oracle; one chunk more, and 1025 regions, are refused with KC_EINVAL
    before any work.  Both refused requests describe real device memory."""
    kc.load()
    big = torch.zeros(4 * W.GiB + 64 * W.KiB, dtype=torch.uint8, device="cuda")
    base = big.data_ptr()
    rng = np.random.default_rng(5)
    offs = np.unique(rng.integers(0, (4 * W.GiB) // 8, 3000)) * 8
    vals = (base + rng.integers(0, 4 * W.GiB // 8, offs.size) * 8).astype(np.uint64)
    vals[::7] = np.uint64(base - 4096)                 # in the window, below the region: outside hits
    big_w = big[: 4 * W.GiB].view(torch.int64)
    big_w[torch.from_numpy(offs // 8).cuda()] = torch.from_numpy(vals.view(np.int64)).cuda()
    win = W.default_window([base], [4 * W.GiB])
    cap = offs.size + 16
    hits, counts = _outputs(cap)
    b = kc.bufs([(base, 4 * W.GiB, kc.RAW, 0)])
    assert kc.census_static(b, win[0], win[1], hits, cap, counts) == kc.OK
    cnt, h = _read(hits, counts, cap)
    host = big[: 4 * W.GiB].cpu().numpy()
    ohits, nin, nout, _ = oracle.census([host], [base], *win)
    del host
    assert cnt == (nin, nout) and nin + nout == offs.size
    assert h.tobytes() == ohits.tobytes()
    # one 64 KiB chunk more than the static counters hold
    b = kc.bufs([(base, 4 * W.GiB + 64 * W.KiB, kc.RAW, 0)])
    assert kc.census_static(b, win[0], win[1], hits, cap, counts) == kc.EINVAL
    # 1025 disjoint regions (the limit is 1024)
    b = kc.bufs([(base + 4096 * i, 4096, kc.RAW, 0) for i in range(1025)])
    assert kc.census_static(b, win[0], win[1], hits, cap, counts) == kc.EINVAL
    del big


def test_static_census_refused_inside_a_stream_capture():
    kc.load()
    snap, dev = _snapshot(3, 0.1)
    win = W.default_window(snap.bases, snap.sizes)
    b = kc.bufs([(t.data_ptr(), t.numel(), kc.RAW, 0) for t in dev])
    hits, counts = _outputs(1000)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    st = None
    with torch.cuda.graph(g, stream=s):
        st = kc.census_static(b, win[0], win[1], hits, 1000, counts, stream=s)
        counts.add_(0)   # the capture holds some work of its own
    assert st == kc.EINVAL
    g.replay()
    torch.cuda.synchronize()
    # outside the capture the same call works
    assert kc.census_static(b, win[0], win[1], hits, 1000, counts) == kc.OK
    cnt, h = _read(hits, counts, 1000)
    ohits, nin, nout, _ = oracle.census(snap.regions, snap.bases, *win)
    assert cnt == (nin, nout) and h.tobytes() == ohits[:1000].tobytes()
