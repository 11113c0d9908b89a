"""Snapshots on disk: save a captured address space (deduplicated) and load
it back at the same VA offsets.

The paper streams every tracked region to host memory in large chunks and
writes it, with a manifest of the regions (base VA, size, kind), next to the
reproducer; replay copies the bytes back at the same VAs ("Memory Capture",
"VA-Faithful HSA Replay").  Here the snapshot is reduced on the device first
(kc_scan: page digests and the pointer census; kc_dedup: page table and the
packed arena of unique non-zero pages), and only the arena crosses to the
host, in chunks through two pinned buffers so that writing one chunk to the
file overlaps copying the next.  Loading reverses it: chunks of the arena
file are read into pinned buffers and copied to a device arena, again
overlapped, and kc_restore writes every page at its VA offset (zero pages
are written as zeros, they are not stored).

Layout of a snapshot directory:
  memory_regions.json  manifest: format version, page size, regions (index,
                       base VA, bytes, dtype, first page, page count), blob
                       count, census counts, file names and sizes
  pages.bin            the page table, 16 bytes per page (va_offset u64,
                       alloc_id u32, blob u32), little-endian
  digest.bin           per page: XXH64 (u64) then, after all hashes, the
                       zero flags (u8); a loader can check pages against them
  arena.bin            n_blobs pages of page_bytes each (unique non-zero
                       pages, the last page of a region zero-filled to S)
  census.bin           the census hits, 24 bytes each (src_offset u64, value
                       u64, src_alloc u32, target i32)
"""
from __future__ import annotations

import json
import os
import time

import numpy as np
import torch

from . import kc
from . import workloads as W

FORMAT = "kc-snapshot-1"
CHUNK = 64 * W.MiB


def _regions_of(bufs) -> list:
    return [dict(index=i, base_va=int(b.base_va), bytes=int(b.bytes), dtype=int(b.dtype)) for i, b in enumerate(bufs)]


def save(ctx: kc.Context, bufs, page_bytes: int, path: str, win=None, census_cap: int = 1 << 20,
         chunk_bytes: int = CHUNK, stream=None) -> dict:
    """Snapshot the regions `bufs` (a kc_buf array of device regions) into
    directory `path`.  Returns the manifest with timings."""
    os.makedirs(path, exist_ok=True)
    st = stream or torch.cuda.current_stream()
    dev = torch.device("cuda", torch.cuda.current_device())
    P = kc.page_count(bufs, page_bytes)
    S = page_bytes
    if win is None:
        bases = [int(b.base_va) for b in bufs]
        win = W.default_window(bases, [int(b.bytes) for b in bufs])
    t0 = time.perf_counter()
    h = torch.empty(max(P, 1), dtype=torch.int64, device=dev)
    z = torch.empty(max(P, 1), dtype=torch.uint8, device=dev)
    pf = torch.empty(len(bufs) + 1, dtype=torch.int64, device=dev)
    hits = torch.empty(max(census_cap, 1) * 24, dtype=torch.uint8, device=dev)
    counts = torch.zeros(2, dtype=torch.int64, device=dev)
    table = torch.empty(max(P, 1) * 16, dtype=torch.uint8, device=dev)
    arena = torch.empty(max(P, 1) * S, dtype=torch.uint8, device=dev)
    nb = torch.zeros(1, dtype=torch.int64, device=dev)
    s1 = ctx.scan(bufs, S, h, z, pf, win[0], win[1], hits, census_cap, counts, st,
                  allow=(kc.OK, kc.EBUF, kc.ETRUNC))
    s2 = ctx.dedup(bufs, S, h, z, table, arena, P * S, nb, st)
    status = ctx.sync(st)
    if status not in (kc.OK, kc.ETRUNC):
        raise kc.KcError(status, "snapshot reduction failed on the device")
    n_blobs = int(nb.cpu().numpy().view(np.uint64)[0])
    cnt = counts.cpu().numpy().view(np.uint64)
    n_hits = int(min(int(cnt[0]) + int(cnt[1]), census_cap))
    t_dev = time.perf_counter() - t0

    # small outputs in one piece
    with open(os.path.join(path, "pages.bin"), "wb") as f:
        f.write(table[:P * 16].cpu().numpy().tobytes())
    with open(os.path.join(path, "digest.bin"), "wb") as f:
        f.write(h[:P].cpu().numpy().tobytes())
        f.write(z[:P].cpu().numpy().tobytes())
    with open(os.path.join(path, "census.bin"), "wb") as f:
        f.write(hits[:n_hits * 24].cpu().numpy().tobytes())

    # the arena, streamed through two pinned buffers
    t1 = time.perf_counter()
    arena_bytes = n_blobs * S
    pinned = [torch.empty(chunk_bytes, dtype=torch.uint8, pin_memory=True) for _ in range(2)]
    done = [torch.cuda.Event(), torch.cuda.Event()]
    copy_stream = torch.cuda.Stream(device=dev)
    copy_stream.wait_stream(st)
    nchunks = (arena_bytes + chunk_bytes - 1) // chunk_bytes
    with open(os.path.join(path, "arena.bin"), "wb") as f:
        pending = None
        for i in range(nchunks + 1):
            if i < nchunks:
                k = i % 2
                o = i * chunk_bytes
                n = min(chunk_bytes, arena_bytes - o)
                with torch.cuda.stream(copy_stream):
                    pinned[k][:n].copy_(arena[o:o + n], non_blocking=True)
                done[k].record(copy_stream)
            if pending is not None:
                k0, n0 = pending
                done[k0].synchronize()
                f.write(memoryview(pinned[k0][:n0].numpy()))
            pending = (i % 2, min(chunk_bytes, arena_bytes - i * chunk_bytes)) if i < nchunks else None
    t_stream = time.perf_counter() - t1
    del arena
    manifest = dict(
        format=FORMAT, page_bytes=S, pages=P, regions=_regions_of(bufs),
        page_first=pf.cpu().numpy().astype(np.int64).tolist(), n_blobs=n_blobs,
        census=dict(inside=int(cnt[0]), outside=int(cnt[1]), stored=n_hits, window=[int(win[0]), int(win[1])],
                    truncated=bool(s1 == kc.ETRUNC or int(cnt[0]) + int(cnt[1]) > census_cap)),
        lost_regions=[i for i in range(len(bufs)) if ctx.buf_status(i) == kc.EBUF] if s2 == kc.EBUF else [],
        files=dict(pages="pages.bin", digest="digest.bin", arena="arena.bin", census="census.bin"),
        sizes=dict(pages=P * 16, digest=P * 9, arena=arena_bytes, census=n_hits * 24),
        timings=dict(device_s=t_dev, arena_stream_s=t_stream,
                     arena_GBps=arena_bytes / t_stream / 1e9 if t_stream > 0 else None),
    )
    with open(os.path.join(path, "memory_regions.json"), "w") as f:
        json.dump(manifest, f, indent=1)
    return manifest


def read_manifest(path: str) -> dict:
    """The manifest of snapshot directory `path`, checked for consistency."""
    with open(os.path.join(path, "memory_regions.json")) as f:
        m = json.load(f)
    if m.get("format") != FORMAT:
        raise ValueError(f"{path}: not a {FORMAT} snapshot (format {m.get('format')!r})")
    S, P = int(m["page_bytes"]), int(m["pages"])
    if S <= 0 or S & (S - 1):
        raise ValueError(f"{path}: page size {S} is not a power of two")
    pf = m["page_first"]
    regs = m["regions"]
    if len(pf) != len(regs) + 1 or pf[0] != 0 or pf[-1] != P:
        raise ValueError(f"{path}: page offsets do not match the regions")
    for i, r in enumerate(regs):
        if pf[i + 1] - pf[i] != -(-int(r["bytes"]) // S):
            raise ValueError(f"{path}: region {i} has the wrong page count")
    for key, size in m["sizes"].items():
        fp = os.path.join(path, m["files"][key])
        if os.path.getsize(fp) != size:
            raise ValueError(f"{path}: {m['files'][key]} holds {os.path.getsize(fp)} bytes, manifest says {size}")
    if m["sizes"]["arena"] != int(m["n_blobs"]) * S:
        raise ValueError(f"{path}: arena size does not match the blob count")
    return m


def load(ctx: kc.Context, path: str, targets=None, chunk_bytes: int = CHUNK, stream=None) -> dict:
    """Restore snapshot `path` into `targets` (a kc_buf array of device
    regions with the manifest's sizes; None = the captured VAs themselves,
    which must be allocated in this process).  Returns timings."""
    m = read_manifest(path)
    S, P = int(m["page_bytes"]), int(m["pages"])
    st = stream or torch.cuda.current_stream()
    dev = torch.device("cuda", torch.cuda.current_device())
    if targets is None:
        targets = kc.bufs([(r["base_va"], r["bytes"], r["dtype"], 0) for r in m["regions"]])
    if len(targets) != len(m["regions"]) or any(int(t.bytes) != int(r["bytes"])
                                                for t, r in zip(targets, m["regions"])):
        raise ValueError("targets do not match the snapshot's regions")
    t0 = time.perf_counter()
    table = torch.from_numpy(np.fromfile(os.path.join(path, m["files"]["pages"]), dtype=np.uint8)).to(dev)
    arena_bytes = int(m["sizes"]["arena"])
    arena = torch.empty(max(arena_bytes, 16), dtype=torch.uint8, device=dev)
    pinned = [torch.empty(chunk_bytes, dtype=torch.uint8, pin_memory=True) for _ in range(2)]
    free = [torch.cuda.Event(), torch.cuda.Event()]
    copy_stream = torch.cuda.Stream(device=dev)
    nchunks = (arena_bytes + chunk_bytes - 1) // chunk_bytes
    with open(os.path.join(path, m["files"]["arena"]), "rb") as f:
        for i in range(nchunks):
            k = i % 2
            o = i * chunk_bytes
            n = min(chunk_bytes, arena_bytes - o)
            if i >= 2:
                free[k].synchronize()          # the copy out of this buffer has finished
            got = f.readinto(memoryview(pinned[k][:n].numpy()))
            if got != n:
                raise IOError(f"{path}: short read of the arena at {o}")
            with torch.cuda.stream(copy_stream):
                arena[o:o + n].copy_(pinned[k][:n], non_blocking=True)
            free[k].record(copy_stream)
    st.wait_stream(copy_stream)
    t_stream = time.perf_counter() - t0
    ctx.restore(targets, S, table, P, arena, arena_bytes, st)
    status = ctx.sync(st)
    if status != kc.OK:
        raise kc.KcError(status, "restore reported malformed rows or a failed region")
    return dict(arena_stream_s=t_stream, arena_GBps=arena_bytes / t_stream / 1e9 if t_stream > 0 else None,
                total_s=time.perf_counter() - t0)
