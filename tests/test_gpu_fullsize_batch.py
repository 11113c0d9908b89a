"""Batched form at full size: 4096 validation jobs (log-uniform 256 B -
64 MiB, ~44 GB of got + want), in the launch configuration the benchmark
times (graph-captured kc_batch_run at a tuned page size and shape).
Checks: byte equality with the plain one-call-per-buffer form on every job,
the planted mismatches found exactly, clean jobs clean, and a sample of
jobs against the oracle."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from oracle import kc_oracle as oracle
from paper_2605_03208_gb300 import batch as B
from paper_2605_03208_gb300 import kc
from paper_2605_03208_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def jobset():
    js = W.batch_jobs(0, n=4096, lo=256, hi=64 * W.MiB, frac_bad=0.05)
    yield js
    del js
    torch.cuda.empty_cache()


def test_batched_4096_jobs_equal_plain_and_oracle(jobset, tmp_path):
    js = jobset
    assert len(js.truth["planted"]) > 150
    ctx_b, ctx_p = kc.Context(0), kc.Context(0)
    try:
        # a short tuning pass over three page sizes (the cache is private to the test)
        tune = B.autotune(ctx_b, js, pages=[16384, 65536, 262144], cache_path=str(tmp_path / "tune.json"),
                          reps=1, budget_s=30.0)
        S = tune["page_bytes"]
        pb, pp = B.make_plan(js, S), B.make_plan(js, S)
        s = torch.cuda.current_stream()
        assert B.run_batched(ctx_b, pb, stream=s) == kc.OK
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        pb.hash.fill_(-1)
        pb.cmp.fill_(0xEE)
        cs = torch.cuda.Stream()
        cs.wait_stream(s)
        with torch.cuda.graph(g, stream=cs):
            assert B.run_batched(ctx_b, pb, stream=cs) == kc.OK
        g.replay()
        assert B.run_plain(ctx_p, pp, stream=s) == kc.OK
        torch.cuda.synchronize()
        assert ctx_b.sync() == kc.OK and ctx_p.sync() == kc.OK
        assert B.same_results(pb, pp)
        h, z, rec = B.results(pb)
        planted = js.truth["planted"]
        for k in range(len(js.sizes)):
            if k in planted:
                assert rec[k]["mismatches"] == len(planted[k]) and rec[k]["first"] == planted[k][0], k
            else:
                assert rec[k]["mismatches"] == 0 and rec[k]["first"] == -1, k
            assert rec[k]["status"] == kc.OK
        # oracle on a sample: the 8 largest jobs, 16 planted ones, 16 random ones
        rng = np.random.default_rng(1)
        order = np.argsort(js.sizes)[::-1]
        sample = set(order[:8].tolist()) | set(list(planted)[:16]) | set(rng.choice(len(js.sizes), 16).tolist())
        for k in sorted(sample):
            o, b, dt = js.offsets[k], js.sizes[k], js.dtypes[k]
            gk = js.got[o:o + b].cpu().numpy()
            wk = js.want[o:o + b].cpu().numpy()
            oh, oz, _ = oracle.digest([gk], S)
            p0, p1 = int(pb.pfirst[k]), int(pb.pfirst[k + 1])
            assert np.array_equal(h[p0:p1], oh) and np.array_equal(z[p0:p1], oz), k
            assert rec[k].tobytes() == oracle.compare(gk, wk, dt).tobytes(), k
    finally:
        ctx_b.close()
        ctx_p.close()
