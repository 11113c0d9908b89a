"""Batched form on the host side: job plans for kc_batch_run, the plain
one-launch-per-buffer form it replaces, and the autotuner that picks the
page size and the persistent kernel's CTA shape.

A validation job is a (got, want) buffer pair: the digest of got (XXH64 per
page, zero flags) and the comparison of got against want by dtype.  The
plain form calls kc_digest and kc_compare once per job; the batched form
hands every job to one kc_batch_run launch, which can be captured in a CUDA
graph.  Both write byte-identical outputs at the same page size.

The autotuner times kc_batch_run over page sizes 4 KiB .. 2 MiB and CTA
shapes (warps per CTA, pipeline stages = loads in flight per page, chunk
bytes per stage) on the caller's own jobs, and keeps the winner in a JSON
cache keyed by GPU name, operation and a size class of the job set.  The
page size it picks is part of the result (page hashes depend on it), so
the cache entry records it and a caller that has stored digests pins it.
"""
from __future__ import annotations

import json
import math
import os
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import kc

PAGE_SIZES = [4096 << i for i in range(10)]          # 4 KiB .. 2 MiB
WARPS = [4, 8, 16]                                    # CTA size 128 / 256 / 512 threads
STAGES = [2, 3, 4, 6]                                 # chunks in flight per page
CHUNKS = [512, 1024]
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


@dataclass
class Plan:
    """Output buffers and the kc_job array for one job set at page size S."""
    page: int
    npages: list
    pfirst: np.ndarray
    hash: torch.Tensor
    zero: torch.Tensor
    cmp: torch.Tensor
    jobs: object                       # ctypes array of kc_job
    got: list = field(default_factory=list)    # (va, bytes, dtype) per job
    want: list = field(default_factory=list)

    @property
    def total_pages(self) -> int:
        return int(self.pfirst[-1])


def make_plan(js, page: int, flags: int = kc.JOB_DIGEST | kc.JOB_COMPARE, device="cuda") -> Plan:
    """Plan over a workloads.JobSet: per-job outputs carved from three
    device tensors (hash u64[P], zero u8[P], records 64 B per job)."""
    npages = [(b + page - 1) // page for b in js.sizes]
    pfirst = np.concatenate([[0], np.cumsum(npages)]).astype(np.int64)
    P = int(pfirst[-1])
    h = torch.empty(max(P, 1), dtype=torch.int64, device=device)
    z = torch.empty(max(P, 1), dtype=torch.uint8, device=device)
    c = torch.empty(max(len(js.sizes), 1) * 64, dtype=torch.uint8, device=device)
    gb, wb = js.got.data_ptr(), js.want.data_ptr()
    hb, zb, cb = h.data_ptr(), z.data_ptr(), c.data_ptr()
    items, got, want = [], [], []
    for k, (b, dt, o) in enumerate(zip(js.sizes, js.dtypes, js.offsets)):
        items.append(dict(got=gb + o, want=wb + o, bytes=b, dtype=dt, flags=flags,
                          hash=hb + 8 * int(pfirst[k]), zero=zb + int(pfirst[k]), cmp=cb + 64 * k))
        got.append((gb + o, b, dt))
        want.append((wb + o, b, dt))
    return Plan(page, npages, pfirst, h, z, c, kc.jobs(items), got, want)


def algorithmic_bytes(plan: Plan) -> int:
    """Bytes a digest + compare pass over every job must move: got and want
    read once each (the fused pass hashes and compares the same read of
    got), 9 bytes written per page (hash + zero flag) and a 64-byte record
    per job."""
    n = sum(b for _, b, _ in plan.got)
    return 2 * n + 9 * plan.total_pages + 64 * len(plan.got)


def run_batched(ctx: kc.Context, plan: Plan, atol=0.0, rtol=0.0, stream=None) -> int:
    return ctx.batch_run(plan.jobs, plan.page, atol, rtol, stream=stream)


def run_plain(ctx: kc.Context, plan: Plan, atol=0.0, rtol=0.0, stream=None) -> int:
    """One kc_digest and one kc_compare call per job (each a launch per
    buffer), writing into the same output layout as the batched plan."""
    hb, zb, cb = plan.hash.data_ptr(), plan.zero.data_ptr(), plan.cmp.data_ptr()
    worst = kc.OK
    for k, (g, w) in enumerate(zip(plan.got, plan.want)):
        gb = kc.bufs([(g[0], g[1], g[2], 0)])
        wb = kc.bufs([(w[0], w[1], w[2], 0)])
        s1 = ctx.digest(gb, plan.page, hb + 8 * int(plan.pfirst[k]), zb + int(plan.pfirst[k]), None, stream)
        s2 = ctx.compare(gb, wb, atol, rtol, cb + 64 * k, stream)
        worst = max(worst, s1, s2)
    return worst


def results(plan: Plan):
    """(hash u64[P], zero u8[P], records[jobs]) on the host."""
    torch.cuda.synchronize()
    P = plan.total_pages
    return (plan.hash[:P].cpu().numpy().view(np.uint64), plan.zero[:P].cpu().numpy(),
            plan.cmp.cpu().numpy().view(kc.CMP_DTYPE)[:len(plan.got)])


def same_results(a: Plan, b: Plan) -> bool:
    ha, za, ra = results(a)
    hb, zb, rb = results(b)
    return np.array_equal(ha, hb) and np.array_equal(za, zb) and ra.tobytes() == rb.tobytes()


# ---------------------------------------------------------------- autotuner

def _gpu_name() -> str:
    try:
        return torch.cuda.get_device_name(torch.cuda.current_device())
    except Exception:
        return "unknown"


def size_class(sizes) -> str:
    """Coarse key of a job set: job count and total bytes, each to the
    nearest power of two, and the log2 of the largest job."""
    n = len(sizes)
    tot = int(sum(sizes))
    big = int(max(sizes)) if n else 0
    return f"jobs2^{round(math.log2(max(n, 1)))}_bytes2^{round(math.log2(max(tot, 1)))}" \
           f"_max2^{round(math.log2(max(big, 1)))}"


def load_cache(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str = DEFAULT_CACHE) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time_ms(fn, reps: int, stream) -> float:
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def autotune(ctx: kc.Context, js, op: str = "digest+compare", pages=None, cache_path: str = DEFAULT_CACHE,
             reps: int = 3, pin_page: int | None = None, force: bool = False, budget_s: float = 60.0) -> dict:
    """Pick (page size, warps, stages, chunk) for kc_batch_run on the job set
    `js`.  A cached entry for the same GPU, op and size class is returned as
    is unless `force`.  `pin_page` fixes the page size (stored digests were
    made with it) and tunes the shape alone.  The search is exhaustive over
    the grid, page sizes in increasing order, and stops early once
    `budget_s` seconds are spent.  The context's forced shape is reset to
    the winner on return."""
    key = f"{_gpu_name()}|{op}|{size_class(js.sizes)}" + (f"|page{pin_page}" if pin_page else "")
    cache = load_cache(cache_path)
    if not force and key in cache:
        best = cache[key]
        ctx.set_digest_shape(best["warps"], best["stages"], best["chunk"], 1)
        return dict(best, cached=True, key=key)
    stream = torch.cuda.current_stream()
    grid = [pin_page] if pin_page else list(pages or PAGE_SIZES)
    flags = kc.JOB_DIGEST | (kc.JOB_COMPARE if "compare" in op else 0)
    sweep = []
    best = None
    t_start = time.time()
    for S in grid:
        plan = make_plan(js, S, flags)
        for w in WARPS:
            for st in STAGES:
                for ch in CHUNKS:
                    if ch > S:
                        continue
                    if ctx.lib.kc_set_digest_shape(ctx.h, w, st, ch, 1) != kc.OK:
                        continue                 # needs more shared memory than a CTA has
                    ms = _time_ms(lambda: run_batched(ctx, plan, stream=stream), reps, stream)
                    rec = dict(page_bytes=S, warps=w, stages=st, chunk=ch, ms=ms)
                    sweep.append(rec)
                    if best is None or ms < best["ms"]:
                        best = rec
        del plan
        if time.time() - t_start > budget_s:
            break
    ctx.set_digest_shape()
    if best is None:
        raise RuntimeError("autotune: no shape could be launched")
    # confirmation: the best few of the sweep re-timed with more repetitions
    # (one sweep timing is a few launches and can be off by several percent)
    top = sorted(sweep, key=lambda r: r["ms"])[:6]
    plans = {}
    for rec in top:
        S = rec["page_bytes"]
        if S not in plans:
            plans[S] = make_plan(js, S, flags)
        ctx.set_digest_shape(rec["warps"], rec["stages"], rec["chunk"], 1)
        rec["ms_confirm"] = min(_time_ms(lambda: run_batched(ctx, plans[S], stream=stream), max(reps, 5), stream)
                                for _ in range(2))
    del plans
    ctx.set_digest_shape()
    best = dict(min(top, key=lambda r: r["ms_confirm"]))
    best = dict(best, gpu=_gpu_name(), op=op, size_class=size_class(js.sizes), swept=len(sweep),
                tuned_at=time.strftime("%Y-%m-%dT%H:%M:%S"))
    cache[key] = best
    cache.setdefault("_sweeps", {})[key] = sweep
    save_cache(cache, cache_path)
    ctx.set_digest_shape(best["warps"], best["stages"], best["chunk"], 1)
    return dict(best, cached=False, key=key)
