"""Helpers for the GPU parity tests: place synthetic snapshots in device
memory, run the CUDA path through the C ABI, and fetch results to the host."""
from __future__ import annotations

import numpy as np
import torch

from paper_2605_03208_gb300 import kc
from paper_2605_03208_gb300 import workloads as W


def device_snapshot(snap_layout, fill, seed=0, **kw):
    """Allocate every region on cuda:0, fill it on the host with its real VA,
    upload it.  Returns (snapshot with host regions, list of device tensors)."""
    dev = [torch.empty(int(s), dtype=torch.uint8, device="cuda") for s in snap_layout.sizes]
    bases = [t.data_ptr() for t in dev]
    snap = fill(snap_layout, bases, seed, **kw)
    for t, r in zip(dev, snap.regions):
        t.copy_(torch.from_numpy(r))
    torch.cuda.synchronize()
    return snap, dev


def region_bufs(snap, dev, flags=None):
    items = []
    for i, (t, dt) in enumerate(zip(dev, snap.dtypes or [kc.RAW] * len(dev))):
        f = 0 if flags is None else flags[i]
        items.append((t.data_ptr(), t.numel(), dt, f))
    return kc.bufs(items)


def to_np(t: torch.Tensor, dtype=None) -> np.ndarray:
    a = t.cpu().numpy()
    return a.view(dtype) if dtype is not None else a


def empty_u8(n):
    return torch.empty(max(int(n), 1), dtype=torch.uint8, device="cuda")


def run_digest(ctx, snap, dev, page_bytes=None, flags=None):
    S = page_bytes or snap.page_bytes
    b = region_bufs(snap, dev, flags)
    P = kc.page_count(b, S)
    h = torch.empty(max(P, 1), dtype=torch.int64, device="cuda")
    z = torch.empty(max(P, 1), dtype=torch.uint8, device="cuda")
    pf = torch.empty(len(dev) + 1, dtype=torch.int64, device="cuda")
    st = ctx.digest(b, S, h, z, pf)
    torch.cuda.synchronize()
    return st, to_np(h)[:P].view(np.uint64), to_np(z)[:P], to_np(pf).view(np.uint64)


def run_scan(ctx, snap, dev, win, cap=None, page_bytes=None, flags=None):
    S = page_bytes or snap.page_bytes
    b = region_bufs(snap, dev, flags)
    P = kc.page_count(b, S)
    if cap is None:
        cap = sum(int(s) // 8 for s in snap.sizes)
    h = torch.empty(max(P, 1), dtype=torch.int64, device="cuda")
    z = torch.empty(max(P, 1), dtype=torch.uint8, device="cuda")
    pf = torch.empty(len(dev) + 1, dtype=torch.int64, device="cuda")
    hits = empty_u8(max(cap, 1) * 24)
    counts = torch.full((2,), 0x5A5A5A5A, dtype=torch.int64, device="cuda")   # the call resets them
    st = ctx.scan(b, S, h, z, pf, win[0], win[1], hits, cap, counts)
    return st, dict(hash=to_np(h)[:P].view(np.uint64), zero=to_np(z)[:P],
                    page_first=to_np(pf).view(np.uint64), hits=to_np(hits).view(kc.HIT_DTYPE),
                    counts=to_np(counts).view(np.uint64))


def run_census(ctx, snap, dev, win, cap=None, flags=None):
    b = region_bufs(snap, dev, flags)
    if cap is None:
        cap = sum(int(s) // 8 for s in snap.sizes)
    hits = empty_u8(max(cap, 1) * 24)
    counts = torch.zeros(2, dtype=torch.int64, device="cuda")
    st = ctx.census(b, win[0], win[1], hits if cap else None, cap, counts)
    return st, to_np(hits).view(kc.HIT_DTYPE), to_np(counts).view(np.uint64)


def hits_tuples(h):
    return [(int(x["src_alloc"]), int(x["src_offset"]), int(x["value"]), int(x["target"])) for x in h]


def run_dedup(ctx, snap, dev, h_dev, z_dev, page_bytes=None, arena_cap=None):
    S = page_bytes or snap.page_bytes
    b = region_bufs(snap, dev)
    P = kc.page_count(b, S)
    table = empty_u8(max(P, 1) * 16)
    if arena_cap is None:
        arena_cap = P * S
    arena = empty_u8(arena_cap) if arena_cap else None
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = ctx.dedup(b, S, h_dev, z_dev, table, arena, arena_cap, nb)
    torch.cuda.synchronize()
    n_blobs = int(to_np(nb).view(np.uint64)[0])
    t = to_np(table).view(kc.PAGE_DTYPE)[:P]
    return st, t, arena, n_blobs
