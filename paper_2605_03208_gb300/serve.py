"""Served form: a request loop that validates candidate buffers against
golden snapshots kept resident on the device.

Tuning or kernel-generating agents submit candidate replays; each request
asks for the digest of its candidate (XXH64 per page and zero flags, which
the host diffs against the golden's stored page digests) or for the dtype
comparison of the candidate against the golden.  The loop

  * keeps the goldens and their page digests resident,
  * admits a request only when the device memory it needs (its candidate
    and outputs) fits, with the goldens, under an HBM budget, and when a
    slot is free,
  * runs admitted requests by continuous batching: every tick is one
    kc_batch_run launch holding a piece of work from every active request
    (shortest remaining work first, each piece at most a quantum), so a
    request that arrives while a 2 GiB one is on the device starts at the
    next tick instead of waiting for it to finish; results of requests
    whose last piece ran are read back as soon as their tick completes.

The plain arm handles the same stream first-in first-out, one request at a
time, with one kc_digest or kc_compare call per request.  Both arms call
only the library's kernels; the host work is planning and bookkeeping.
All results are exact, so a request's result is the same alone, in the
mix, and in either arm.
"""
from __future__ import annotations

import collections
import hashlib
import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import kc
from . import workloads as W

DIGEST, COMPARE = "digest", "compare"


# ---------------------------------------------------------------- requests

@dataclass
class Request:
    rid: int
    kind: str                 # DIGEST or COMPARE
    gid: int                  # golden buffer
    t_arrival: float          # seconds after the stream starts
    n_perturb: int            # elements changed in the candidate (0 = identical)
    seed: int
    # filled while serving
    t_start: float = 0.0      # client began handling it (seconds after the stream starts)
    admit_wait: float = 0.0   # seconds spent waiting for admission
    t_ready: float = 0.0      # candidate exists, request submitted
    t_launch: float = 0.0     # its last piece of work was enqueued on the device
    t_done: float = 0.0
    result: dict = field(default_factory=dict)
    planted: np.ndarray | None = None


def request_stream(seed: int, n: int, rate: float, n_goldens: int, frac_compare: float = 0.5,
                   frac_bad: float = 0.3) -> list:
    """n requests with Poisson arrivals at `rate` per second, each a digest
    or a comparison of a uniformly chosen golden; a `frac_bad` share carries
    1..64 changed elements."""
    rng = np.random.default_rng(seed + 909)
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    t -= t[0]
    out = []
    for i in range(n):
        kind = COMPARE if rng.random() < frac_compare else DIGEST
        bad = int(rng.integers(1, 65)) if rng.random() < frac_bad else 0
        out.append(Request(i, kind, int(rng.integers(0, n_goldens)), float(t[i]), bad,
                           int(rng.integers(0, 2**31))))
    return out


class Goldens:
    """Resident golden buffers and their page digests at page size S."""

    def __init__(self, ctx: kc.Context, data: torch.Tensor, sizes, dtypes, offsets, page: int = 65536):
        self.data, self.sizes, self.dtypes, self.offsets, self.page = data, sizes, dtypes, offsets, page
        b = kc.bufs([(data.data_ptr() + o, s, dt, 0) for s, dt, o in zip(sizes, dtypes, offsets)])
        P = kc.page_count(b, page)
        h = torch.empty(P, dtype=torch.int64, device=data.device)
        z = torch.empty(P, dtype=torch.uint8, device=data.device)
        pf = torch.empty(len(sizes) + 1, dtype=torch.int64, device=data.device)
        ctx.digest(b, page, h, z, pf)
        torch.cuda.synchronize()
        pf = pf.cpu().numpy().astype(np.int64)
        hh, zz = h.cpu().numpy().view(np.uint64), z.cpu().numpy()
        self.hash = [hh[pf[i]:pf[i + 1]].copy() for i in range(len(sizes))]
        self.zero = [zz[pf[i]:pf[i + 1]].copy() for i in range(len(sizes))]

    @property
    def resident_bytes(self) -> int:
        return int(self.data.numel()) + sum(h.nbytes + z.nbytes for h, z in zip(self.hash, self.zero))

    def view(self, gid: int) -> torch.Tensor:
        o = self.offsets[gid]
        return self.data[o:o + self.sizes[gid]]


def request_bytes(req: Request, g: Goldens) -> int:
    """Device memory a request holds while admitted: its candidate and its outputs."""
    n = g.sizes[req.gid]
    pages = (n + g.page - 1) // g.page
    return n + (9 * pages if req.kind == DIGEST else 64)


def algorithmic_bytes(req: Request, g: Goldens) -> int:
    n = g.sizes[req.gid]
    pages = (n + g.page - 1) // g.page
    return n + 9 * pages if req.kind == DIGEST else 2 * n + 64


def make_candidate(req: Request, g: Goldens, stream) -> torch.Tensor:
    """The candidate a replay produced: a device copy of the golden with
    req.n_perturb elements changed (not part of the timed service work)."""
    with torch.cuda.stream(stream):
        cand = torch.empty_like(g.view(req.gid))
        cand.copy_(g.view(req.gid))
        req.planted = np.zeros(0, np.int64)
        if req.n_perturb:
            req.planted = W.plant(cand, g.dtypes[req.gid], req.n_perturb, np.random.default_rng(req.seed))
    return cand


def finish(req: Request, g: Goldens, host_hash, host_zero, host_cmp) -> None:
    """Result of a request from its outputs on the host."""
    if req.kind == DIGEST:
        h = host_hash.view(np.uint64)
        z = host_zero
        diff = np.nonzero((h != g.hash[req.gid]) | (z != g.zero[req.gid]))[0]
        req.result = dict(pages_differ=diff.astype(np.int64).tolist(),
                          digest_sha1=hashlib.sha1(h.tobytes() + z.tobytes()).hexdigest())
    else:
        rec = host_cmp.view(kc.CMP_DTYPE)[0]
        req.result = dict(record=rec.tobytes().hex(), mismatches=int(rec["mismatches"]),
                          first=int(rec["first"]))


def expected_ok(req: Request, g: Goldens) -> bool:
    """The result agrees with what was planted in the candidate."""
    if req.kind == DIGEST:
        es = W.ESIZE[g.dtypes[req.gid]]
        pages = sorted(set((req.planted * es // g.page).tolist()))
        return req.result["pages_differ"] == pages
    first = int(req.planted[0]) if len(req.planted) else -1
    return req.result["mismatches"] == len(req.planted) and req.result["first"] == first


# ---------------------------------------------------------------- admission

class Budget:
    """Bytes of device memory under a cap, and a number of slots."""

    def __init__(self, cap_bytes: int, slots: int):
        self.cap, self.slots = int(cap_bytes), int(slots)
        self.used, self.busy = 0, 0
        self.peak_used, self.waits = 0, 0
        self.cv = threading.Condition()

    def acquire(self, n: int, stop=None) -> bool:
        if n > self.cap:
            raise ValueError(f"request of {n} bytes exceeds the admission budget of {self.cap}")
        with self.cv:
            if self.used + n > self.cap or self.busy >= self.slots:
                self.waits += 1
            while self.used + n > self.cap or self.busy >= self.slots:
                if stop is not None and stop.is_set():
                    return False
                self.cv.wait(0.05)
            self.used += n
            self.busy += 1
            self.peak_used = max(self.peak_used, self.used)
            return True

    def try_acquire(self, n: int) -> bool:
        """acquire without waiting."""
        with self.cv:
            if self.used + n > self.cap or self.busy >= self.slots:
                return False
            self.used += n
            self.busy += 1
            self.peak_used = max(self.peak_used, self.used)
            return True

    def release(self, n: int) -> None:
        with self.cv:
            self.used -= n
            self.busy -= 1
            self.cv.notify_all()


# ---------------------------------------------------------------- tick planning

@dataclass
class Active:
    """An admitted request's remaining work, in units of the batched kernel:
    pages for a digest, 64 KiB items for a comparison."""
    req: Request
    total: int
    unit_bytes: int
    next: int = 0

    @property
    def remaining(self) -> int:
        return self.total - self.next


def plan_tick(active: list, tick_bytes: int, quantum_bytes: int) -> list:
    """Pieces of one tick: (Active, first unit, unit count), shortest
    remaining work first, each piece at most `quantum_bytes`, until the
    tick holds `tick_bytes` (at least one piece).  Pure host logic."""
    out = []
    room = tick_bytes
    for a in sorted(active, key=lambda a: (a.remaining * a.unit_bytes, a.req.rid)):
        if a.remaining <= 0:
            continue
        if out and room <= 0:
            break
        cap_units = max(1, min(quantum_bytes, max(room, a.unit_bytes)) // a.unit_bytes)
        cnt = int(min(a.remaining, cap_units))
        out.append((a, a.next, cnt))
        room -= cnt * a.unit_bytes
    return out


# ---------------------------------------------------------------- the two arms

class _Outputs:
    """Outputs of one request.  mapped (batched arm): the kernel writes page
    digests straight into pinned host memory and the job's last warp copies
    the comparison record there, so nothing is read back; otherwise
    (sequential arm) device outputs and an explicit read-back."""

    def __init__(self, req: Request, g: Goldens, device, mapped: bool):
        n = g.sizes[req.gid]
        self.pages = (n + g.page - 1) // g.page
        self.hash = self.zero = self.h_hash = self.h_zero = self.cmp = self.h_cmp = None
        if req.kind == DIGEST:
            self.h_hash = torch.empty(self.pages, dtype=torch.int64, pin_memory=True)
            self.h_zero = torch.empty(self.pages, dtype=torch.uint8, pin_memory=True)
            if mapped:
                self.hash, self.zero = self.h_hash, self.h_zero
            else:
                self.hash = torch.empty(self.pages, dtype=torch.int64, device=device)
                self.zero = torch.empty(self.pages, dtype=torch.uint8, device=device)
        else:
            self.cmp = torch.empty(64, dtype=torch.uint8, device=device)
            self.h_cmp = torch.empty(64, dtype=torch.uint8, pin_memory=True)

    def read_back(self, stream):
        with torch.cuda.stream(stream):
            if self.hash is not None:
                self.h_hash.copy_(self.hash, non_blocking=True)
                self.h_zero.copy_(self.zero, non_blocking=True)
            else:
                self.h_cmp.copy_(self.cmp, non_blocking=True)

    def host(self):
        if self.h_hash is not None:
            return self.h_hash.numpy(), self.h_zero.numpy(), None
        return None, None, self.h_cmp.numpy()


@dataclass
class ServeStats:
    mode: str
    n: int
    latencies_ms: list
    makespan_s: float
    algorithmic_bytes: int
    ticks: int = 0
    max_batch: int = 0
    mean_batch: float = 0.0
    launches: int = 0
    budget_waits: int = 0
    peak_admitted_bytes: int = 0
    queue_ms: list = field(default_factory=list)    # submission -> last piece enqueued
    device_ms: list = field(default_factory=list)   # last piece enqueued -> result on the host

    def summary(self) -> dict:
        lat = np.asarray(self.latencies_ms)
        parts = {}
        if self.queue_ms:
            parts = dict(queue_p50_ms=float(np.percentile(self.queue_ms, 50)),
                         queue_p99_ms=float(np.percentile(self.queue_ms, 99)),
                         run_p50_ms=float(np.percentile(self.device_ms, 50)),
                         run_p99_ms=float(np.percentile(self.device_ms, 99)))
        return dict(mode=self.mode, requests=self.n, p50_ms=float(np.percentile(lat, 50)),
                    p99_ms=float(np.percentile(lat, 99)), mean_ms=float(lat.mean()), max_ms=float(lat.max()),
                    makespan_s=self.makespan_s, GBps=self.algorithmic_bytes / self.makespan_s / 1e9,
                    ticks=self.ticks, max_requests_per_tick=self.max_batch,
                    mean_requests_per_tick=self.mean_batch, gpu_launches=self.launches,
                    admission_waits=self.budget_waits, peak_admitted_bytes=self.peak_admitted_bytes, **parts)


class Server:
    """Serves a list of requests against resident goldens, in one of two
    modes: "batched" (continuous batching over kc_batch_run) or
    "sequential" (FIFO, one kc_digest / kc_compare call per request).

    A request's latency is the time from its submission (its candidate
    exists) to its result on the host, plus the time it waited for
    admission; producing the candidate is the submitting agent's work and
    is not counted."""

    def __init__(self, ctx: kc.Context, goldens: Goldens, mode: str = "batched",
                 budget_bytes: int = 120 * 10**9, slots: int = 256, tick_bytes: int = 512 * W.MiB,
                 quantum_bytes: int = 128 * W.MiB, solo_quantum_bytes: int = 1024 * W.MiB,
                 max_inflight: int = 2, realtime: bool = True, preload: bool = False):
        assert mode in ("batched", "sequential")
        self.ctx, self.g, self.mode = ctx, goldens, mode
        self.budget = Budget(budget_bytes - goldens.resident_bytes, slots)
        self.slots = slots
        self.tick_bytes, self.quantum, self.solo_quantum = tick_bytes, quantum_bytes, solo_quantum_bytes
        self.max_inflight = max_inflight
        self.realtime = realtime and not preload
        self.preload = preload      # every candidate made before serving starts (closed-loop saturation)
        self.device = goldens.data.device

    # client side: admission, then the candidate, then the queue
    def _client(self, reqs, q, t0, stop, errors):
        try:
            gen = torch.cuda.Stream(device=self.device)
            for r in reqs:
                if self.realtime:
                    d = t0 + r.t_arrival - time.perf_counter()
                    if d > 0:
                        time.sleep(d)
                t_start = time.perf_counter()
                if self.preload:
                    # nothing is served yet, so nothing would free the budget
                    if not self.budget.try_acquire(request_bytes(r, self.g)):
                        raise RuntimeError("preload: the requests do not fit in the admission budget and slots")
                elif not self.budget.acquire(request_bytes(r, self.g), stop):
                    return
                r.admit_wait = time.perf_counter() - t_start
                r.t_start = t_start - t0
                cand = make_candidate(r, self.g, gen)
                gen.synchronize()
                r.t_ready = time.perf_counter() - t0
                q.put((r, cand))
        except BaseException as e:  # surfaced by serve()
            errors.append(e)
            stop.set()

    def serve(self, reqs: list) -> ServeStats:
        q = queue.Queue()
        stop = threading.Event()
        errors = []
        if self.mode == "batched":
            self._slot_buffers()
        if self.preload:
            self._client(reqs, q, time.perf_counter(), stop, errors)
            if errors:
                raise errors[0]
        torch.cuda.synchronize()
        l0 = kc.launch_count()
        t0 = time.perf_counter()
        if self.preload:
            for r in reqs:              # all submitted at the start
                r.t_start = r.t_ready = 0.0
                r.admit_wait = 0.0
        th = threading.Thread(target=self._client, args=([] if self.preload else reqs, q, t0, stop, errors),
                              daemon=True)
        th.start()
        try:
            if self.mode == "batched":
                ticks, sizes = self._loop_batched(len(reqs), q, t0, stop, errors)
            else:
                ticks, sizes = self._loop_sequential(len(reqs), q, t0, stop, errors)
        finally:
            stop.set()
            th.join()
        if errors:
            raise errors[0]
        lat = [1000.0 * (r.t_done - r.t_ready + r.admit_wait) for r in reqs]
        span = max(r.t_done for r in reqs) - min(r.t_start for r in reqs)
        st = ServeStats(self.mode, len(reqs), lat, span, sum(algorithmic_bytes(r, self.g) for r in reqs),
                        ticks=ticks, launches=kc.launch_count() - l0, budget_waits=self.budget.waits,
                        peak_admitted_bytes=self.budget.peak_used)
        if sizes:
            st.max_batch, st.mean_batch = max(sizes), float(np.mean(sizes))
        st.queue_ms = [1000.0 * (r.t_launch - r.t_ready) for r in reqs]
        st.device_ms = [1000.0 * (r.t_done - r.t_launch) for r in reqs]
        return st

    def _done(self, r, outs, t0):
        r.t_done = time.perf_counter() - t0
        finish(r, self.g, *outs.host())
        self.budget.release(request_bytes(r, self.g))

    def _get(self, q, stop, errors, timeout=None):
        while True:
            if errors:
                raise errors[0]
            try:
                if timeout == 0:
                    return q.get_nowait()
                return q.get(timeout=0.05 if timeout is None else timeout)
            except queue.Empty:
                if timeout is not None:
                    return None

    def _loop_sequential(self, n, q, t0, stop, errors):
        st = torch.cuda.Stream(device=self.device)
        g = self.g
        for _ in range(n):
            r, cand = self._get(q, stop, errors)
            outs = _Outputs(r, g, self.device, mapped=False)
            dt = g.dtypes[r.gid]
            cb = kc.bufs([(cand.data_ptr(), cand.numel(), dt, 0)])
            r.t_launch = time.perf_counter() - t0
            if r.kind == DIGEST:
                self.ctx.digest(cb, g.page, outs.hash, outs.zero, None, st)
            else:
                gb = kc.bufs([(g.view(r.gid).data_ptr(), g.sizes[r.gid], dt, 0)])
                self.ctx.compare(cb, gb, 0.0, 0.0, outs.cmp, st)
            outs.read_back(st)
            st.synchronize()
            self._done(r, outs, t0)
            del cand
        return n, []

    def _slot_buffers(self):
        """Per-slot outputs of the batched arm, allocated once per server:
        page digests and record copies in pinned host memory (written by
        the kernel), records on the device, the flags, the job arrays."""
        if getattr(self, "_slots_made", None) is None:
            g, S_ = self.g, self.slots
            max_pages = max((b + g.page - 1) // g.page for b in g.sizes)
            self._slots_made = dict(
                max_pages=max_pages,
                h_hash=torch.empty((S_, max_pages), dtype=torch.int64, pin_memory=True),
                h_zero=torch.empty((S_, max_pages), dtype=torch.uint8, pin_memory=True),
                h_cmp=torch.empty((S_, 64), dtype=torch.uint8, pin_memory=True),
                d_cmp=torch.empty((S_, 64), dtype=torch.uint8, device=self.device),
                flags=kc.FlagPoller(S_), jobs=(kc.KcJob * S_)(), work=(kc.KcWork * S_)(),
                events=[torch.cuda.Event() for _ in range(self.max_inflight + 1)])
        return self._slots_made

    def _loop_batched(self, n, q, t0, stop, errors):
        st = torch.cuda.Stream(device=self.device)
        g = self.g
        S_ = self.slots
        B = self._slot_buffers()
        max_pages, h_hash, h_zero, h_cmp, d_cmp = B["max_pages"], B["h_hash"], B["h_zero"], B["h_cmp"], B["d_cmp"]
        hb, zb, cb, dcb = h_hash.data_ptr(), h_zero.data_ptr(), h_cmp.data_ptr(), d_cmp.data_ptr()
        hv, zv, cv = h_hash.numpy(), h_zero.numpy(), h_cmp.numpy()
        flags, jobs, work, events = B["flags"], B["jobs"], B["work"], B["events"]
        for i in range(S_):
            flags.clear(i)
        ev_next = 0
        free = list(range(S_ - 1, -1, -1))
        active = []                                 # Active entries with work left to launch
        held = {}                                   # rid -> (candidate, slot)
        waiting = {}                                # slot -> request whose last piece is launched
        inflight = collections.deque()              # tick events
        finished = 0
        ticks, sizes = 0, []
        while finished < n:
            progressed = False
            # admit everything that is ready
            block = not active and not inflight and not waiting
            item = self._get(q, stop, errors, timeout=None if block else 0)
            while item is not None:
                r, cand = item
                slot = free.pop()
                flags.clear(slot)
                held[r.rid] = (cand, slot)
                if r.kind == DIGEST:
                    active.append(Active(r, (g.sizes[r.gid] + g.page - 1) // g.page, g.page))
                else:
                    active.append(Active(r, (g.sizes[r.gid] + kc.BATCH_ITEM_BYTES - 1) // kc.BATCH_ITEM_BYTES,
                                         kc.BATCH_ITEM_BYTES))
                item = self._get(q, stop, errors, timeout=0)
                progressed = True
            # results: a request is done when its flag is set
            for slot in flags.poll() if waiting else ():
                r = waiting.pop(slot)
                held.pop(r.rid)
                r.t_done = time.perf_counter() - t0
                if r.kind == DIGEST:
                    P = (g.sizes[r.gid] + g.page - 1) // g.page
                    finish(r, g, hv[slot, :P], zv[slot, :P], None)
                else:
                    finish(r, g, None, None, cv[slot])
                self.budget.release(request_bytes(r, g))
                flags.clear(slot)
                free.append(slot)
                finished += 1
                progressed = True
            while inflight and inflight[0].query():
                inflight.popleft()
            # launch a tick when there is work and room in the stream
            if active and len(inflight) < self.max_inflight:
                quantum = self.solo_quantum if len(active) == 1 else self.quantum
                pieces = plan_tick(active, self.tick_bytes if len(active) > 1 else quantum, quantum)
                now = time.perf_counter() - t0
                for k, (a, first, cnt) in enumerate(pieces):
                    r = a.req
                    cand, slot = held[r.rid]
                    last = a.next + cnt == a.total
                    J = jobs[k]
                    J.got_va = cand.data_ptr()
                    J.want_va = g.view(r.gid).data_ptr()
                    J.bytes = g.sizes[r.gid]
                    J.dtype = g.dtypes[r.gid]
                    dig = r.kind == DIGEST
                    J.flags = (kc.JOB_DIGEST if dig else kc.JOB_COMPARE) | (kc.JOB_INIT if a.next == 0 else 0)
                    J.d_hash = hb + slot * max_pages * 8 if dig else 0
                    J.d_zero = zb + slot * max_pages if dig else 0
                    J.d_cmp = 0 if dig else dcb + 64 * slot
                    J.d_done = flags.address(slot) if last else 0
                    J.d_cmp_copy = cb + 64 * slot if (last and not dig) else 0
                    w = work[k]
                    w.job, w.kind, w.first, w.count = k, (kc.WORK_DIGEST if dig else kc.WORK_COMPARE), first, cnt
                    a.next += cnt
                    if last:
                        waiting[slot] = r
                        r.t_launch = now
                self.ctx.batch_run(jobs, g.page, 0.0, 0.0, work_array=work, stream=st,
                                   njobs=len(pieces), nwork=len(pieces))
                ev = events[ev_next]
                ev_next = (ev_next + 1) % len(events)
                ev.record(st)
                inflight.append(ev)
                active = [a for a in active if a.remaining > 0]
                ticks += 1
                sizes.append(len(pieces))
                progressed = True
            if not progressed:
                time.sleep(0)                       # let the client thread run
        st.synchronize()
        return ticks, sizes
