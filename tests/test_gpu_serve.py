"""GPU tests of the served form: continuous batching gives every request the
same result as handling it alone, as the sequential arm, and as the oracle;
admission under a tight budget; requests overlap on the device."""
from __future__ import annotations

import dataclasses
import hashlib

import numpy as np
import pytest
import torch

from oracle import kc_oracle as oracle
from paper_2605_03208_gb300 import kc
from paper_2605_03208_gb300 import serve as S
from paper_2605_03208_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    ctx = kc.Context(0)
    data, sizes, dtypes, offs = W.golden_set(3, n=8, lo=W.MiB, hi=48 * W.MiB)
    g = S.Goldens(ctx, data, sizes, dtypes, offs, page=65536)
    yield ctx, g
    ctx.close()


def _fresh(reqs):
    return [dataclasses.replace(r, result={}, planted=None, t_start=0.0, admit_wait=0.0, t_ready=0.0,
                                t_launch=0.0, t_done=0.0) for r in reqs]


def test_goldens_digest_matches_oracle(setup):
    ctx, g = setup
    for gid in range(len(g.sizes)):
        oh, oz, _ = oracle.digest([g.view(gid).cpu().numpy()], g.page)
        assert np.array_equal(g.hash[gid], oh) and np.array_equal(g.zero[gid], oz)


def test_mix_equals_sequential_solo_and_oracle(setup):
    ctx, g = setup
    base = S.request_stream(1, 80, rate=2000.0, n_goldens=len(g.sizes), frac_bad=0.5)
    budget = g.resident_bytes + 160 * W.MiB           # a few requests at a time: admission waits
    rb, rs = _fresh(base), _fresh(base)
    st_b = S.Server(ctx, g, "batched", budget_bytes=budget, tick_bytes=32 * W.MiB,
                    quantum_bytes=8 * W.MiB).serve(rb)
    st_s = S.Server(ctx, g, "sequential", budget_bytes=budget).serve(rs)
    assert st_b.ticks >= 1
    # everything queued at once: requests share ticks, results unchanged
    rp = _fresh(base)
    st_p = S.Server(ctx, g, "batched", tick_bytes=32 * W.MiB, quantum_bytes=8 * W.MiB, preload=True).serve(rp)
    assert st_p.max_batch > 1
    for a, b in zip(rp, rs):
        assert a.result == b.result, a.rid
    for a, b in zip(rb, rs):
        assert a.result == b.result, a.rid
        assert S.expected_ok(a, g), (a.rid, a.kind, a.result, a.planted)
    # alone: the same result
    for r in _fresh(base[:12]):
        S.Server(ctx, g, "batched", budget_bytes=budget).serve([r])
        assert r.result == rb[r.rid].result, r.rid
    # the oracle on the candidates (regenerated from their seeds)
    gen = torch.cuda.Stream()
    for r in _fresh(base[:24]):
        cand = S.make_candidate(r, g, gen)
        gen.synchronize()
        c = cand.cpu().numpy()
        if r.kind == S.DIGEST:
            oh, oz, _ = oracle.digest([c], g.page)
            assert hashlib.sha1(oh.tobytes() + oz.tobytes()).hexdigest() == rb[r.rid].result["digest_sha1"]
        else:
            o = oracle.compare(c, g.view(r.gid).cpu().numpy(), g.dtypes[r.gid])
            assert o.tobytes().hex() == rb[r.rid].result["record"], r.rid


def test_big_request_does_not_block_small_ones(setup):
    """A large comparison admitted first is cut into quanta: small requests
    that arrive after it finish before it does."""
    ctx, g = setup
    big = int(np.argmax(g.sizes))
    small = int(np.argmin(g.sizes))
    reqs = [S.Request(0, S.COMPARE, big, 0.0, 0, 1)] + \
           [S.Request(i, S.DIGEST, small, 0.0, 0, 1 + i) for i in range(1, 6)]
    S.Server(ctx, g, "batched", tick_bytes=2 * W.MiB, quantum_bytes=W.MiB, solo_quantum_bytes=W.MiB,
             realtime=False).serve(reqs)
    assert all(r.t_done < reqs[0].t_done for r in reqs[1:])
    assert reqs[0].result["mismatches"] == 0 and all(r.result["pages_differ"] == [] for r in reqs[1:])
