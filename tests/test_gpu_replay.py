"""GPU test of multi-iteration replay: with the snapshot re-copied before
every iteration, a kernel that updates its inputs in place produces the
golden outputs every time; without it, later iterations drift."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_2605_03208_gb300 import kc
from paper_2605_03208_gb300 import replay as R

pytestmark = pytest.mark.gpu


def test_recopy_resets_state_and_no_recopy_drifts():
    ctx = kc.Context(0)
    try:
        g = torch.Generator(device="cuda")
        g.manual_seed(3)
        x = torch.randn(3 << 18, generator=g, device="cuda")             # 3 MiB, updated in place
        zeros = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")   # zero pages: not stored
        ctr = torch.zeros(1024, dtype=torch.int32, device="cuda")        # a counter the kernel bumps
        regions = [x, zeros, ctr]
        bufs = kc.bufs([(t.data_ptr(), t.numel() * t.element_size(), kc.RAW, 0) for t in regions])
        snap = R.capture(ctx, bufs, 65536)
        assert snap.n_blobs == 48   # the pages of x; zero pages (the zero region, the counter) are not stored
        captured = [t.clone() for t in regions]
        out = torch.empty_like(x)
        cnt = torch.empty_like(ctr)

        def kernel():
            x.add_(1.0)
            ctr.add_(1)
            torch.mul(x, 2.0, out=out)
            cnt.copy_(ctr)

        golden = [(captured[0] + 1.0) * 2.0, captured[2] + 1]
        outputs = [(out, kc.F32), (cnt, kc.I32)]
        rep = R.run(ctx, snap, kernel, outputs, golden, iterations=4, do_recopy=True)
        assert rep.all_match and len(rep.records) == 4
        assert all(t >= 0 for t in rep.recopy_ms)
        assert torch.equal(x, captured[0] + 1.0) and torch.equal(zeros, captured[1])
        rep2 = R.run(ctx, snap, kernel, outputs, golden, iterations=3, do_recopy=False)
        mism = [[int(r["mismatches"]) for r in rec] for rec in rep2.records]
        assert mism[0] == [0, 0]                                # starts from the captured state
        assert mism[1][1] == ctr.numel() and mism[1][0] > 0     # then drifts
        assert torch.equal(ctr, captured[2] + 3)
    finally:
        ctx.close()
