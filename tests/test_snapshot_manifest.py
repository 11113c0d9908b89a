"""Snapshot manifest checks (host only): a consistent directory is accepted,
inconsistent ones are rejected with a reason."""
from __future__ import annotations

import json
import os

import pytest

SIO = pytest.importorskip("paper_2605_03208_gb300.snapshot_io")


def _write(d, **over):
    S, sizes = 4096, [10000, 4096, 1]
    pf = [0]
    for b in sizes:
        pf.append(pf[-1] + -(-b // S))
    P = pf[-1]
    m = dict(format=SIO.FORMAT, page_bytes=S, pages=P,
             regions=[dict(index=i, base_va=0x7000_0000 + i * 0x10000, bytes=b, dtype=5) for i, b in enumerate(sizes)],
             page_first=pf, n_blobs=3, census=dict(inside=0, outside=0, stored=0, window=[0, 0], truncated=False),
             lost_regions=[], files=dict(pages="pages.bin", digest="digest.bin", arena="arena.bin", census="census.bin"),
             sizes=dict(pages=P * 16, digest=P * 9, arena=3 * S, census=0))
    m.update(over)
    for key, name in m["files"].items():
        with open(os.path.join(d, name), "wb") as f:
            f.write(b"\0" * dict(pages=P * 16, digest=P * 9, arena=3 * S, census=0)[key])
    with open(os.path.join(d, "memory_regions.json"), "w") as f:
        json.dump(m, f)
    return m


def test_consistent_manifest_is_accepted(tmp_path):
    m = _write(tmp_path)
    assert SIO.read_manifest(str(tmp_path))["pages"] == m["pages"] == 5


@pytest.mark.parametrize("bad", [dict(format="other"), dict(page_bytes=3000), dict(page_first=[0, 3, 4, 6]),
                                 dict(n_blobs=4), dict(sizes=dict(pages=80, digest=45, arena=3 * 4096, census=24))])
def test_inconsistent_manifest_is_rejected(tmp_path, bad):
    _write(tmp_path, **bad)
    with pytest.raises(ValueError):
        SIO.read_manifest(str(tmp_path))
