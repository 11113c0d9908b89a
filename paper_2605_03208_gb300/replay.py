"""Multi-iteration replay with the snapshot re-copied before each iteration.

A kernel under test that writes to its own inputs (in-place updates,
accumulators, counters) sees different inputs on every run unless the
captured state is put back first; the paper's replay re-copies the snapshot
before each iteration and offers a switch to skip it ("VA-Faithful HSA
Replay").  Here the deduplicated snapshot (page table + arena of unique
pages, both resident in device memory) is written back over the regions by
kc_restore -- a device-to-device scatter at memory bandwidth, with zero
pages written as zeros -- before each iteration, unless `recopy` is off.
Outputs are checked against golden buffers with kc_compare after every
iteration.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from . import kc


@dataclass
class Resident:
    """A snapshot kept on the device: page table and arena."""
    bufs: object            # kc_buf array of the regions (their VAs)
    page_bytes: int
    pages: int
    table: torch.Tensor
    arena: torch.Tensor
    n_blobs: int


def capture(ctx: kc.Context, bufs, page_bytes: int, stream=None) -> Resident:
    """Digest, deduplicate and pack the regions into a resident snapshot."""
    dev = torch.device("cuda", torch.cuda.current_device())
    P = kc.page_count(bufs, page_bytes)
    h = torch.empty(max(P, 1), dtype=torch.int64, device=dev)
    z = torch.empty(max(P, 1), dtype=torch.uint8, device=dev)
    table = torch.empty(max(P, 1) * 16, dtype=torch.uint8, device=dev)
    arena = torch.empty(max(P, 1) * page_bytes, dtype=torch.uint8, device=dev)
    nb = torch.zeros(1, dtype=torch.int64, device=dev)
    ctx.digest(bufs, page_bytes, h, z, None, stream)
    ctx.dedup(bufs, page_bytes, h, z, table, arena, P * page_bytes, nb, stream)
    if ctx.sync(stream) != kc.OK:
        raise kc.KcError(kc.ECUDA, "capture failed on the device")
    n_blobs = int(nb.cpu().numpy().view(np.uint64)[0])
    return Resident(bufs, page_bytes, P, table, arena[:max(n_blobs, 1) * page_bytes].clone(), n_blobs)


def recopy(ctx: kc.Context, snap: Resident, stream=None) -> None:
    """Put the captured bytes back at their VAs."""
    ctx.restore(snap.bufs, snap.page_bytes, snap.table, snap.pages, snap.arena, snap.n_blobs * snap.page_bytes,
                stream)


@dataclass
class ReplayReport:
    iterations: int
    recopy: bool
    records: list = field(default_factory=list)   # per iteration: kc_cmp_result per output
    recopy_ms: list = field(default_factory=list)
    run_ms: list = field(default_factory=list)

    @property
    def all_match(self) -> bool:
        return all(int(r["mismatches"]) == 0 for rec in self.records for r in rec)


def run(ctx: kc.Context, snap: Resident, kernel, outputs, golden, iterations: int, do_recopy: bool = True,
        atol: float = 0.0, rtol: float = 0.0, stream=None) -> ReplayReport:
    """Replay `kernel()` (which reads and may write the snapshot's regions
    and writes `outputs`) `iterations` times; before each iteration the
    snapshot is re-copied unless `do_recopy` is False (the first iteration
    always starts from the captured state).  After each iteration the
    outputs -- (tensor, dtype) pairs -- are compared with `golden` (tensors)."""
    st = stream or torch.cuda.current_stream()
    gb = kc.bufs([(o.data_ptr(), o.numel() * o.element_size(), dt, 0) for o, dt in outputs])
    wb = kc.bufs([(g.data_ptr(), g.numel() * g.element_size(), dt, 0) for g, (_, dt) in zip(golden, outputs)])
    rec = torch.empty(len(outputs) * 64, dtype=torch.uint8, device=st.device)
    rep = ReplayReport(iterations, do_recopy)
    E = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    for i in range(iterations):
        e0, e1, e2 = E(), E(), E()
        e0.record(st)
        if do_recopy or i == 0:
            recopy(ctx, snap, st)
        e1.record(st)
        with torch.cuda.stream(st):
            kernel()
        e2.record(st)
        ctx.compare(gb, wb, atol, rtol, rec, st)
        if ctx.sync(st) != kc.OK:
            raise kc.KcError(kc.ECUDA, "replay iteration failed on the device")
        rep.recopy_ms.append(e0.elapsed_time(e1))
        rep.run_ms.append(e1.elapsed_time(e2))
        rep.records.append(rec.cpu().numpy().view(kc.CMP_DTYPE).copy())
    return rep
