"""GPU tests of snapshots on disk and of the byte-diff report: a saved
snapshot restores byte for byte (into fresh regions and VA-faithfully into
the original ones), its page table, digests and census equal the oracle's,
and the byte-diff report equals the oracle's byte-exact comparison (and
a direct count of the differing bytes)."""
from __future__ import annotations

import os

import numpy as np
import pytest
import torch

import _gpu as G
from oracle import kc_oracle as oracle
from paper_2605_03208_gb300 import kc
from paper_2605_03208_gb300 import snapshot_io as SIO
from paper_2605_03208_gb300 import validate as V
from paper_2605_03208_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = kc.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("chunk", [1 << 20, 64 << 20])
def test_save_load_roundtrip(ctx, tmp_path, chunk):
    layout = W.tiny_layout(7, n=16, total=16 * W.MiB)
    snap, dev = G.device_snapshot(layout, W.tiny_fill, 7)
    b = G.region_bufs(snap, dev)
    S = snap.page_bytes
    m = SIO.save(ctx, b, S, str(tmp_path), chunk_bytes=chunk)
    assert SIO.read_manifest(str(tmp_path))["n_blobs"] == m["n_blobs"]
    # page table, digests and census against the oracle
    oh, oz, opf = oracle.digest(snap.regions, S)
    P = len(oh)
    raw = np.fromfile(os.path.join(tmp_path, "digest.bin"), dtype=np.uint8)
    assert np.array_equal(raw[:8 * P].view(np.uint64), oh) and np.array_equal(raw[8 * P:], oz)
    od = oracle.dedup(snap.regions, S, oh, oz)
    tbl = np.fromfile(os.path.join(tmp_path, "pages.bin"), dtype=kc.PAGE_DTYPE)
    assert np.array_equal(tbl["blob"], od["blob"]) and m["n_blobs"] == od["n_blobs"]
    arena = np.fromfile(os.path.join(tmp_path, "arena.bin"), dtype=np.uint8)
    assert np.array_equal(arena, oracle.pack(snap.regions, S, od))
    hits, nin, nout, rc = oracle.census(snap.regions, snap.bases, *m["census"]["window"])
    got_hits = np.fromfile(os.path.join(tmp_path, "census.bin"), dtype=kc.HIT_DTYPE)
    assert (m["census"]["inside"], m["census"]["outside"]) == (nin, nout)
    assert G.hits_tuples(got_hits) == G.hits_tuples(hits)
    # restore into fresh regions (a relocation the caller asks for)
    fresh = [torch.full_like(t, 0xA5) for t in dev]
    t = SIO.load(ctx, str(tmp_path), targets=G.region_bufs(snap, fresh), chunk_bytes=chunk)
    assert t["arena_stream_s"] >= 0
    for f, r in zip(fresh, snap.regions):
        assert np.array_equal(G.to_np(f), r)
    # VA-faithful: the original regions, overwritten, restored at their VAs
    for d in dev:
        d.fill_(0x5C)
    SIO.load(ctx, str(tmp_path), chunk_bytes=chunk)
    for d, r in zip(dev, snap.regions):
        assert np.array_equal(G.to_np(d), r)


def test_load_rejects_mismatched_targets(ctx, tmp_path):
    layout = W.tiny_layout(8, n=4, total=2 * W.MiB)
    snap, dev = G.device_snapshot(layout, W.tiny_fill, 8)
    SIO.save(ctx, G.region_bufs(snap, dev), snap.page_bytes, str(tmp_path))
    wrong = [torch.empty(int(s) + 64, dtype=torch.uint8, device="cuda") for s in snap.sizes]
    with pytest.raises(ValueError):
        SIO.load(ctx, str(tmp_path), targets=kc.bufs([(x.data_ptr(), x.numel()) for x in wrong]))


def test_byte_diff_report(ctx):
    rng = np.random.default_rng(9)
    sizes = [1, 15, 16, 4097, 1 << 20]
    got, want, expect = [], [], []
    for n in sizes:
        a = rng.integers(0, 256, n, dtype=np.uint8)
        b = a.copy()
        k = int(rng.integers(0, min(n, 50) + 1))
        idx = np.unique(rng.integers(0, n, k)) if k else np.zeros(0, np.int64)
        b[idx] ^= 0x80
        ga, wb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
        got.append((ga, n))
        want.append((wb, n))
        d = int((a != b).sum())
        expect.append((d, 100.0 * d / n, int(np.nonzero(a != b)[0][0]) if d else -1))
    rep = V.byte_diff(ctx, got, want)
    for r, (d, pct, first), (ga, n), (wb, _) in zip(rep, expect, got, want):
        # the oracle's byte-exact comparison (KC_RAW, zero tolerance) of the same bytes
        o = oracle.compare(ga.cpu().numpy(), wb.cpu().numpy(), oracle.DT_RAW)
        assert (r["differing"], r["first"]) == (int(o["mismatches"]), int(o["first"])) == (d, first)
        assert r["percent"] == pytest.approx(100.0 * int(o["mismatches"]) / n) == pytest.approx(pct)
