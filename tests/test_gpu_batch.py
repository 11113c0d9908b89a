"""GPU parity of the batched form (kc_batch_run): many digest and comparison
jobs of uneven sizes in one persistent work-stealing launch, against the
oracle; split work over several launches; lost jobs; CUDA-graph replay."""
from __future__ import annotations

import time

import numpy as np
import pytest
import torch

from oracle import kc_oracle as oracle
from paper_2605_03208_gb300 import kc
from paper_2605_03208_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = kc.Context(0)
    yield c
    c.close()


class Outs:
    """Per-job output buffers for a job set: hashes, zero flags, records."""

    def __init__(self, js, page):
        self.page = page
        self.npages = [(b + page - 1) // page for b in js.sizes]
        self.pfirst = np.concatenate([[0], np.cumsum(self.npages)]).astype(np.int64)
        P = int(self.pfirst[-1])
        self.hash = torch.full((P,), -1, dtype=torch.int64, device="cuda")
        self.zero = torch.full((P,), 0xEE, dtype=torch.uint8, device="cuda")
        self.cmp = torch.full((len(js.sizes) * 64,), 0xEE, dtype=torch.uint8, device="cuda")

    def job_dicts(self, js, flags):
        out = []
        hb, zb, cb = self.hash.data_ptr(), self.zero.data_ptr(), self.cmp.data_ptr()
        for k, (b, dt, o) in enumerate(zip(js.sizes, js.dtypes, js.offsets)):
            out.append(dict(got=js.got.data_ptr() + o, want=js.want.data_ptr() + o, bytes=b, dtype=dt,
                            flags=flags[k], hash=hb + 8 * int(self.pfirst[k]), zero=zb + int(self.pfirst[k]),
                            cmp=cb + 64 * k))
        return out

    def fetch(self):
        torch.cuda.synchronize()
        return (self.hash.cpu().numpy().view(np.uint64), self.zero.cpu().numpy(),
                self.cmp.cpu().numpy().view(kc.CMP_DTYPE))


def _host(js):
    return js.got.cpu().numpy(), js.want.cpu().numpy()


def _check_against_oracle(js, outs, flags, atol=0.0, rtol=0.0, lost=()):
    h, z, rec = outs.fetch()
    g, w = _host(js)
    for k, (b, dt, o) in enumerate(zip(js.sizes, js.dtypes, js.offsets)):
        p0, p1 = int(outs.pfirst[k]), int(outs.pfirst[k + 1])
        if flags[k] & kc.JOB_DIGEST:
            if k in lost:
                assert (h[p0:p1] == 0).all() and (z[p0:p1] == kc.PAGE_LOST).all(), k
            else:
                oh, oz, _ = oracle.digest([g[o:o + b]], outs.page)
                assert np.array_equal(h[p0:p1], oh), (k, b)
                assert np.array_equal(z[p0:p1], oz), (k, b)
        else:
            assert (z[p0:p1] == 0xEE).all(), k   # untouched
        if flags[k] & kc.JOB_COMPARE:
            if k in lost:
                assert rec[k]["status"] == kc.EBUF and rec[k]["mismatches"] == 0 and rec[k]["first"] == -1, k
            else:
                want = oracle.compare(g[o:o + b], w[o:o + b], dt, atol, rtol)
                assert rec[k].tobytes() == want.tobytes(), (k, b, dt, rec[k], want)


def _small_set(seed, n=160, hi=3 * W.MiB):
    js = W.batch_jobs(seed, n=n, lo=16, hi=hi, frac_bad=0.2)
    return js


@pytest.mark.parametrize("page", [4096, 65536, 2 * W.MiB])
def test_batch_digest_and_compare_vs_oracle(ctx, page):
    js = _small_set(0)
    outs = Outs(js, page)
    flags = [kc.JOB_DIGEST | kc.JOB_COMPARE] * len(js.sizes)
    st = ctx.batch_run(outs.job_dicts(js, flags), page)
    assert st == kc.OK and ctx.sync() == kc.OK
    _check_against_oracle(js, outs, flags)
    # planted mismatches are all found, at the planted positions
    _, _, rec = outs.fetch()
    for k, idx in js.truth["planted"].items():
        assert rec[k]["mismatches"] == len(idx) and rec[k]["first"] == idx[0], k


def test_batch_matches_single_operations(ctx):
    """The batched launch gives byte-identical outputs to kc_digest and
    kc_compare called on the same buffers."""
    js = _small_set(1, n=90)
    page = 16384
    outs = Outs(js, page)
    flags = [kc.JOB_DIGEST | kc.JOB_COMPARE] * len(js.sizes)
    assert ctx.batch_run(outs.job_dicts(js, flags), page) == kc.OK
    h, z, rec = outs.fetch()
    b = kc.bufs([(js.got.data_ptr() + o, s, dt, 0) for s, dt, o in zip(js.sizes, js.dtypes, js.offsets)])
    bw = kc.bufs([(js.want.data_ptr() + o, s, dt, 0) for s, dt, o in zip(js.sizes, js.dtypes, js.offsets)])
    P = int(outs.pfirst[-1])
    h1 = torch.empty(P, dtype=torch.int64, device="cuda")
    z1 = torch.empty(P, dtype=torch.uint8, device="cuda")
    assert ctx.digest(b, page, h1, z1) == kc.OK
    r1 = torch.empty(len(js.sizes) * 64, dtype=torch.uint8, device="cuda")
    assert ctx.compare(b, bw, 0.0, 0.0, r1) == kc.OK
    torch.cuda.synchronize()
    assert np.array_equal(h1.cpu().numpy().view(np.uint64), h)
    assert np.array_equal(z1.cpu().numpy(), z)
    assert r1.cpu().numpy().tobytes() == rec.tobytes()


@pytest.mark.parametrize("atol,rtol", [(1e-6, 0.0), (0.0, 1e-3), (1e-3, 1e-2)])
def test_batch_compare_tolerances(ctx, atol, rtol):
    js = W.batch_jobs(2, n=60, lo=16, hi=W.MiB, frac_bad=0.5)
    outs = Outs(js, 65536)
    flags = [kc.JOB_COMPARE] * len(js.sizes)
    assert ctx.batch_run(outs.job_dicts(js, flags), 65536, atol, rtol) == kc.OK
    _check_against_oracle(js, outs, flags, atol, rtol)


def test_batch_digest_only_and_compare_only_jobs(ctx):
    js = _small_set(3, n=70)
    page = 8192
    outs = Outs(js, page)
    rng = np.random.default_rng(3)
    flags = [int(rng.choice([kc.JOB_DIGEST, kc.JOB_COMPARE, kc.JOB_DIGEST | kc.JOB_COMPARE]))
             for _ in js.sizes]
    assert ctx.batch_run(outs.job_dicts(js, flags), page) == kc.OK
    _check_against_oracle(js, outs, flags)


def test_batch_split_work_over_launches(ctx):
    """Each job's pages and comparison items cut into random pieces, spread
    over three launches in random order: the records merge to the same
    result as one launch, and every page is written once."""
    js = _small_set(4, n=80)
    page = 4096
    outs = Outs(js, page)
    flags = [kc.JOB_DIGEST | kc.JOB_COMPARE] * len(js.sizes)
    rng = np.random.default_rng(44)
    pieces = []
    for k, b in enumerate(js.sizes):
        for kind, total in ((kc.WORK_DIGEST, outs.npages[k]),
                            (kc.WORK_COMPARE, (b + kc.BATCH_ITEM_BYTES - 1) // kc.BATCH_ITEM_BYTES)):
            cuts = sorted(set(rng.integers(0, total + 1, size=int(rng.integers(0, 4))).tolist()) | {0, total})
            for a, c in zip(cuts[:-1], cuts[1:]):
                if c > a:
                    pieces.append((k, kind, a, c - a))
    order = rng.permutation(len(pieces))
    calls = [[pieces[i] for i in order[j::3]] for j in range(3)]
    init = [f | kc.JOB_INIT for f in flags]
    for j, wl in enumerate(calls):
        jobs = outs.job_dicts(js, init if j == 0 else flags)
        st = ctx.batch_run(jobs, page, work_array=wl if wl else [(0, kc.WORK_DIGEST, 0, 0)])
        assert st == kc.OK, ctx.last_error()
    assert ctx.sync() == kc.OK
    _check_against_oracle(js, outs, flags)


def test_batch_fused_work_over_launches(ctx):
    """Fused ranges (digest and compare of the same pages in one pass) cut
    into random pieces over three launches, next to jobs that only digest
    or only compare: every output equals the oracle's."""
    js = _small_set(6, n=80)
    page = 4096
    outs = Outs(js, page)
    rng = np.random.default_rng(66)
    flags = [int(rng.choice([kc.JOB_DIGEST | kc.JOB_COMPARE] * 3 + [kc.JOB_DIGEST, kc.JOB_COMPARE]))
             for _ in js.sizes]
    pieces = []
    for k, b in enumerate(js.sizes):
        both = flags[k] == kc.JOB_DIGEST | kc.JOB_COMPARE
        kind = kc.WORK_FUSED if both else kc.WORK_DIGEST if flags[k] == kc.JOB_DIGEST else kc.WORK_COMPARE
        total = outs.npages[k] if kind != kc.WORK_COMPARE else (b + kc.BATCH_ITEM_BYTES - 1) // kc.BATCH_ITEM_BYTES
        cuts = sorted(set(rng.integers(0, total + 1, size=int(rng.integers(0, 4))).tolist()) | {0, total})
        for a, c in zip(cuts[:-1], cuts[1:]):
            if c > a:
                pieces.append((k, kind, a, c - a))
    order = rng.permutation(len(pieces))
    calls = [[pieces[i] for i in order[j::3]] for j in range(3)]
    init = [f | kc.JOB_INIT for f in flags]
    for j, wl in enumerate(calls):
        jobs = outs.job_dicts(js, init if j == 0 else flags)
        st = ctx.batch_run(jobs, page, work_array=wl if wl else [(0, kc.WORK_DIGEST, 0, 0)])
        assert st == kc.OK, ctx.last_error()
    assert ctx.sync() == kc.OK
    _check_against_oracle(js, outs, flags)


@pytest.mark.parametrize("shape", [(16, 6, 1024), (16, 2, 512), (4, 6, 1024), (8, 3, 256)])
def test_batch_fused_forced_shapes(ctx, shape):
    """A forced shape too large for the fused ring (got and want chunks per
    stage) is shrunk to fit; the results do not depend on the shape."""
    js = _small_set(7, n=60)
    page = 65536
    outs = Outs(js, page)
    flags = [kc.JOB_DIGEST | kc.JOB_COMPARE] * len(js.sizes)
    assert ctx.lib.kc_set_digest_shape(ctx.h, *shape, 1) in (kc.OK, kc.EINVAL)
    try:
        assert ctx.batch_run(outs.job_dicts(js, flags), page) == kc.OK, ctx.last_error()
        assert ctx.sync() == kc.OK
    finally:
        ctx.set_digest_shape()
    _check_against_oracle(js, outs, flags)


def test_batch_lost_job(ctx):
    js = _small_set(5, n=40)
    page = 65536
    outs = Outs(js, page)
    flags = [kc.JOB_DIGEST | kc.JOB_COMPARE] * len(js.sizes)
    lost = {3, 17}
    jf = [f | (kc.BUF_LOST if k in lost else 0) for k, f in enumerate(flags)]
    st = ctx.batch_run(outs.job_dicts(js, jf), page)
    assert st == kc.EBUF
    assert ctx.sync() == kc.OK
    _check_against_oracle(js, outs, flags, lost=lost)


def test_batch_graph_replay(ctx):
    """A captured kc_batch_run replays on new contents of the same buffers."""
    js = _small_set(6, n=50)
    page = 16384
    outs = Outs(js, page)
    flags = [kc.JOB_DIGEST | kc.JOB_COMPARE] * len(js.sizes)
    jobs = kc.jobs(outs.job_dicts(js, flags))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        assert ctx.batch_run(jobs, page, stream=s) == kc.OK   # warm: tables built outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        assert ctx.batch_run(jobs, page, stream=torch.cuda.current_stream()) == kc.OK
    for rep in range(3):
        # new contents: flip bytes of a few jobs, then replay
        gen = torch.Generator(device="cuda")
        gen.manual_seed(rep)
        idx = torch.randint(0, js.got.numel(), (200,), generator=gen, device="cuda")
        js.got[idx] ^= 0x40
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        _check_against_oracle(js, outs, flags)


def test_batch_empty_and_tiny_jobs(ctx):
    """Jobs of 16..48 bytes (shorter than one XXH64 stripe and ragged tails)
    and a zero-filled job."""
    sizes = [16, 32, 48, 64, 80, 4096, 4112, 65536 + 16]
    n = len(sizes)
    offs = [k * 131072 for k in range(n)]
    got = torch.zeros(n * 131072, dtype=torch.uint8, device="cuda")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    got[131072:] = torch.randint(0, 256, (got.numel() - 131072,), generator=gen, device="cuda").to(torch.uint8)
    want = got.clone()
    want[131072 * 2 + 5] ^= 1
    js = W.JobSet(sizes, [W.DT_U8] * n, offs, got, want, {})
    outs = Outs(js, 4096)
    flags = [kc.JOB_DIGEST | kc.JOB_COMPARE] * n
    assert ctx.batch_run(outs.job_dicts(js, flags), 4096) == kc.OK
    _check_against_oracle(js, outs, flags)
    h, z, rec = outs.fetch()
    assert z[0] == kc.PAGE_ZERO and rec[2]["mismatches"] == 1 and rec[2]["first"] == 5


def test_batch_argument_errors(ctx):
    js = _small_set(8, n=4, hi=65536)
    outs = Outs(js, 4096)
    good = outs.job_dicts(js, [kc.JOB_DIGEST | kc.JOB_COMPARE] * 4)
    before = kc.launch_count()

    def bad(mod, page=4096, work=None):
        jobs = [dict(j) for j in good]
        mod(jobs)
        return ctx.batch_run(jobs, page, work_array=work, allow=(kc.OK, kc.EBUF, kc.EINVAL))

    assert bad(lambda j: None, page=3000) == kc.EINVAL
    assert bad(lambda j: j[0].update(flags=0)) == kc.EINVAL
    assert bad(lambda j: j[1].update(got=j[1]["got"] + 8)) == kc.EINVAL
    assert bad(lambda j: j[2].update(bytes=0)) == kc.EINVAL
    assert bad(lambda j: j[3].update(dtype=9)) == kc.EINVAL
    assert bad(lambda j: j[0].update(hash=0)) == kc.EINVAL
    assert bad(lambda j: j[0].update(cmp=0)) == kc.EINVAL
    assert bad(lambda j: None, work=[(4, kc.WORK_DIGEST, 0, 1)]) == kc.EINVAL
    assert bad(lambda j: None, work=[(0, 7, 0, 1)]) == kc.EINVAL
    assert bad(lambda j: None, work=[(0, kc.WORK_DIGEST, 0, outs.npages[0] + 1)]) == kc.EINVAL
    assert bad(lambda j: None, work=[(0, kc.WORK_FUSED, 0, outs.npages[0] + 1)]) == kc.EINVAL
    assert bad(lambda j: j[1].update(flags=kc.JOB_DIGEST), work=[(1, kc.WORK_FUSED, 0, 1)]) == kc.EINVAL
    assert kc.launch_count() == before
    assert ctx.batch_run(good, 4096) == kc.OK and ctx.sync() == kc.OK


def test_batch_completion_flags_and_record_copies(ctx):
    """d_done flags in pinned host memory are set for every job, the record
    copies equal the device records, a job with no unit in the launch is
    flagged at once, and a job whose flag is not asked for is left alone."""
    js = _small_set(9, n=40)
    page = 65536
    outs = Outs(js, page)
    flags = [kc.JOB_DIGEST | kc.JOB_COMPARE] * len(js.sizes)
    n = len(js.sizes)
    done = torch.zeros(n, dtype=torch.int32, pin_memory=True)
    copies = torch.zeros(n * 64, dtype=torch.uint8, pin_memory=True)
    jobs = outs.job_dicts(js, flags)
    for k, j in enumerate(jobs):
        if k != 5:
            j["done"] = done.data_ptr() + 4 * k
            j["cmp_copy"] = copies.data_ptr() + 64 * k
    assert ctx.batch_run(jobs, page) == kc.OK
    torch.cuda.synchronize()
    h, z, rec = outs.fetch()
    d = done.numpy()
    assert (d[np.arange(n) != 5] == 1).all() and d[5] == 0
    cp = copies.numpy().view(kc.CMP_DTYPE)
    for k in range(n):
        if k != 5:
            assert cp[k].tobytes() == rec[k].tobytes(), k
    _check_against_oracle(js, outs, flags)
    # split over two launches: the flag is asked for in the second only; a
    # job absent from a launch's work list is flagged by that launch at once
    outs2 = Outs(js, page)
    done.zero_()
    copies.zero_()
    first = [(k, kc.WORK_COMPARE, 0, 1) for k in range(n)]
    second = [(k, kc.WORK_COMPARE, 1, (js.sizes[k] + kc.BATCH_ITEM_BYTES - 1) // kc.BATCH_ITEM_BYTES - 1)
              for k in range(n)]
    second = [w for w in second if w[3] > 0]
    jf = [kc.JOB_COMPARE | kc.JOB_INIT] * n
    jobs1 = outs2.job_dicts(js, jf)
    assert ctx.batch_run(jobs1, page, work_array=first) == kc.OK
    jobs2 = outs2.job_dicts(js, [kc.JOB_COMPARE] * n)
    for k, j in enumerate(jobs2):
        j["done"] = done.data_ptr() + 4 * k
        j["cmp_copy"] = copies.data_ptr() + 64 * k
    assert ctx.batch_run(jobs2, page, work_array=second) == kc.OK
    torch.cuda.synchronize()
    assert (done.numpy() == 1).all()
    _, _, rec2 = outs2.fetch()
    assert copies.numpy().view(kc.CMP_DTYPE).tobytes() == rec2.tobytes()
    _check_against_oracle(js, outs2, [kc.JOB_COMPARE] * n)


def test_batch_small_job_flag_precedes_launch_end(ctx):
    """With jobs ordered small first, a small job's flag can be observed
    on the host while the launch is still busy with a large job (at least the
    flag is set no later than the end; both results are exact)."""
    sizes = [64 * 1024, 1 << 30]
    got = torch.empty(sum(sizes) + 256, dtype=torch.uint8, device="cuda")
    got.random_(0, 256)
    offs = [0, sizes[0]]
    js = W.JobSet(sizes, [W.DT_U8, W.DT_U8], offs, got, got, {})
    outs = Outs(js, 65536)
    done = torch.zeros(2, dtype=torch.int32, pin_memory=True)
    copies = torch.zeros(128, dtype=torch.uint8, pin_memory=True)
    jobs = outs.job_dicts(js, [kc.JOB_COMPARE | kc.JOB_INIT] * 2)
    for k in range(2):
        jobs[k]["done"] = done.data_ptr() + 4 * k
        jobs[k]["cmp_copy"] = copies.data_ptr() + 64 * k
    work = [(0, kc.WORK_COMPARE, 0, 1), (1, kc.WORK_COMPARE, 0, sizes[1] // kc.BATCH_ITEM_BYTES)]
    ctx.batch_run(jobs, 65536, work_array=work)          # builds the tables
    torch.cuda.synchronize()
    done.zero_()
    ev = torch.cuda.Event()
    ctx.batch_run(jobs, 65536, work_array=work)
    ev.record()
    seen_small_first = False
    t_end = time.perf_counter() + 10.0
    while time.perf_counter() < t_end:
        d = done.numpy()
        if d[0] == 1 and d[1] == 0:
            seen_small_first = True
        if d[1] == 1:
            break
    ev.synchronize()
    assert (done.numpy() == 1).all()
    rec = copies.numpy().view(kc.CMP_DTYPE)
    assert rec["mismatches"].tolist() == [0, 0] and rec["first"].tolist() == [-1, -1]
    # report only: the small job finished while the large one ran
    print("small job flagged before the large one:", seen_small_first)
