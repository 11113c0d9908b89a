"""Region validation reports over kc_compare.

The paper's variant validator reports, per output region, how many bytes
differ and what share of the region that is ("Replay Validation", byte-exact
comparison), and its tolerance validator compares by dtype with NaNs
reported.  kc_compare with dtype KC_RAW (or KC_U8) and zero tolerance is the
byte-exact comparison: its mismatch count is the number of differing bytes
and its first index the first differing byte.  This module only assembles
the per-region report from the kernel's records.
"""
from __future__ import annotations

import numpy as np
import torch

from . import kc


def byte_diff(ctx: kc.Context, got, want, stream=None) -> list:
    """Per region k: differing bytes, their share of the region (percent) and
    the first differing byte offset (-1 if none).  got / want: lists of
    (device address or tensor, bytes)."""
    g = kc.bufs([(kc._ptr(a), int(n), kc.RAW, 0) for a, n in got])
    w = kc.bufs([(kc._ptr(a), int(n), kc.RAW, 0) for a, n in want])
    out = torch.empty(len(got) * 64, dtype=torch.uint8, device="cuda")
    ctx.compare(g, w, 0.0, 0.0, out, stream)
    ctx.sync(stream)
    rec = out.cpu().numpy().view(kc.CMP_DTYPE)
    report = []
    for (_, n), r in zip(got, rec):
        d = int(r["mismatches"])
        report.append(dict(bytes=int(n), differing=d, percent=100.0 * d / int(n) if n else 0.0,
                           first=int(r["first"]), status=int(r["status"])))
    return report
