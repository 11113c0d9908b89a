"""GPU parity at full workload sizes, in the launch configuration the
benchmark times (automatic kernel shapes, default page sizes).

- llama.cpp-shaped snapshot (400 regions, ~0.39 GiB, 64 KiB pages): every
  output compared with the oracle element by element.
- MoE pool (30 GiB in one region + 1536 expert pointers, 2 MiB pages): the
  oracle hashes sampled pages one by one; the census must recover exactly the
  1536 planted pointers and nothing else; dedup must map every planted copy
  to its source; restore into a fresh region must reproduce all 30 GiB
  (checked on the device by torch.equal); the bf16 [4096, 7168] comparison is
  checked against the oracle on the full pair.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_03208_gb300 import kc
from paper_2605_03208_gb300 import workloads as W
from tests import _gpu as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    kc.load()
    c = kc.Context(0)
    yield c
    c.close()


def test_llama_full_parity(ctx):
    snap, dev = G.device_snapshot(W.llama_layout(0), W.llama_fill, 0)
    S = snap.page_bytes
    win = W.default_window(snap.bases, snap.sizes)
    st, r = G.run_scan(ctx, snap, dev, win, cap=1 << 16)
    assert st == kc.OK and ctx.sync() == kc.OK
    oh, oz, opf = oracle.digest(snap.regions, S)
    assert np.array_equal(r["page_first"], opf)
    assert np.array_equal(r["hash"], oh) and np.array_equal(r["zero"], oz)
    ohits, nin, nout, rc = oracle.census(snap.regions, snap.bases, *win)
    assert (int(r["counts"][0]), int(r["counts"][1])) == (nin, nout)
    assert G.hits_tuples(r["hits"][: nin + nout]) == G.hits_tuples(ohits)
    assert set(snap.truth["pointers"]) <= set(G.hits_tuples(ohits))
    h_dev = torch.from_numpy(r["hash"].view(np.int64).copy()).cuda()
    z_dev = torch.from_numpy(r["zero"].copy()).cuda()
    st, t, arena, nb = G.run_dedup(ctx, snap, dev, h_dev, z_dev, S)
    assert st == kc.OK and ctx.sync() == kc.OK
    ot = oracle.dedup(snap.regions, S, oh, oz)
    assert nb == ot["n_blobs"] and np.array_equal(t["blob"], ot["blob"])
    assert np.array_equal(G.to_np(arena)[: nb * S], oracle.pack(snap.regions, S, ot))
    targets = [torch.full_like(x, 0x5A) for x in dev]
    tbl = torch.from_numpy(t.view(np.uint8).copy()).cuda()
    assert ctx.restore(G.region_bufs(snap, targets), S, tbl, len(t), arena, nb * S) == kc.OK
    assert ctx.sync() == kc.OK
    for a, b in zip(targets, dev):
        assert torch.equal(a, b)
    pairs = W.llama_pairs(0)
    g = [torch.from_numpy(p.got.view(np.uint8)).cuda() for p in pairs]
    w = [torch.from_numpy(p.want.view(np.uint8)).cuda() for p in pairs]
    out = torch.empty(len(pairs) * 64, dtype=torch.uint8, device="cuda")
    ctx.compare(kc.bufs([(x.data_ptr(), x.numel(), kc.F32, 0) for x in g]),
                kc.bufs([(x.data_ptr(), x.numel(), kc.F32, 0) for x in w]), 0.0, 0.0, out)
    assert ctx.sync() == kc.OK
    recs = G.to_np(out).view(kc.CMP_DTYPE)
    for rec, p in zip(recs, pairs):
        assert rec.tobytes() == oracle.compare(p.got, p.want, p.dtype).tobytes()
        assert rec["mismatches"] == len(p.truth["perturbed"])


@pytest.fixture(scope="module")
def moe():
    free, total = torch.cuda.mem_get_info()
    if free < 100 * W.GiB:
        pytest.skip(f"needs ~100 GiB free device memory, have {free / W.GiB:.0f} GiB")
    snap, dev = W.moe_snapshot(0)
    yield snap, dev
    del dev
    torch.cuda.empty_cache()


def _page_bytes(pool, p, S):
    return pool[p * S:(p + 1) * S].cpu().numpy()


def test_moe_scan_dedup_restore(ctx, moe):
    snap, dev = moe
    S = snap.page_bytes
    pool, ptrs = dev
    b = kc.bufs([(pool.data_ptr(), pool.numel(), kc.BF16, 0), (ptrs.data_ptr(), ptrs.numel() * 8, kc.RAW, 0)])
    P = kc.page_count(b, S)
    assert P == 15361
    win = W.default_window(snap.bases, snap.sizes)
    h = torch.empty(P, dtype=torch.int64, device="cuda")
    z = torch.empty(P, dtype=torch.uint8, device="cuda")
    pf = torch.empty(3, dtype=torch.int64, device="cuda")
    cap = 1 << 16
    hits = torch.empty(cap * 24, dtype=torch.uint8, device="cuda")
    counts = torch.zeros(2, dtype=torch.int64, device="cuda")
    assert ctx.scan(b, S, h, z, pf, win[0], win[1], hits, cap, counts) == kc.OK
    assert ctx.sync() == kc.OK
    hh = G.to_np(h).view(np.uint64)
    zz = G.to_np(z)
    # census: exactly the 1536 planted pointers, in order, all into the pool
    c = G.to_np(counts).view(np.uint64)
    assert (int(c[0]), int(c[1])) == (1536, 0)
    got_hits = G.hits_tuples(G.to_np(hits).view(kc.HIT_DTYPE)[:1536])
    assert got_hits == snap.truth["pointers"]
    ptr_host = G.to_np(ptrs).view(np.uint8)
    # the pool as a target range only (its pages are sampled below), the
    # pointer array scanned whole
    ohits, nin, nout, _ = oracle.census([np.zeros(0, np.uint8), ptr_host], snap.bases, *win,
                                        sizes=snap.sizes)
    assert G.hits_tuples(ohits) == [(1, o, v, t) for (_, o, v, t) in snap.truth["pointers"]]
    # digest: sampled pages, every planted copy and its source, the last page
    rng = np.random.default_rng(7)
    sample = set(rng.choice(P - 1, 48, replace=False).tolist())
    sample |= set(snap.truth["dup_dst"][:16].tolist()) | set(snap.truth["dup_src"][:16].tolist())
    for p in sorted(sample):
        page = _page_bytes(pool, p, S)
        assert int(hh[p]) == oracle.xxh64(page), p
        # the sampled page, scanned against the full captured ranges: no hits
        pg_hits, a, bb, _ = oracle.census([page, np.zeros(0, np.uint8)],
                                          [snap.bases[0] + p * S, snap.bases[1]], *win,
                                          sizes=[S, snap.sizes[1]])
        assert a + bb == 0                           # bf16 words are never VAs
    assert int(hh[P - 1]) == oracle.xxh64(ptr_host)
    assert (zz == 0).all()
    for d, s_ in zip(snap.truth["dup_dst"], snap.truth["dup_src"]):
        assert hh[d] == hh[s_]
    # dedup: planted copies share their source's blob
    table = torch.empty(P * 16, dtype=torch.uint8, device="cuda")
    ndup = len(snap.truth["dup_dst"])
    arena = torch.empty((P - ndup) * S, dtype=torch.uint8, device="cuda")
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert ctx.dedup(b, S, h, z, table, arena, arena.numel(), nb) == kc.OK
    assert ctx.sync() == kc.OK
    n_blobs = int(G.to_np(nb).view(np.uint64)[0])
    assert n_blobs == P - ndup
    t = G.to_np(table).view(kc.PAGE_DTYPE)
    blob = t["blob"].astype(np.int64)
    assert np.array_equal(blob[snap.truth["dup_dst"]], blob[snap.truth["dup_src"]])
    assert len(np.unique(blob)) == n_blobs
    # canonical page of a planted class = its smallest page id; blob ids
    # follow the canonical pages in page order
    canon_of = np.arange(P)
    members = {}
    for d, s_ in zip(snap.truth["dup_dst"], snap.truth["dup_src"]):
        members.setdefault(int(s_), [int(s_)]).append(int(d))
    for m in members.values():
        canon_of[m] = min(m)
    is_canon = canon_of == np.arange(P)
    assert int(is_canon.sum()) == n_blobs
    expect_blob = np.cumsum(is_canon) - 1
    assert np.array_equal(blob, expect_blob[canon_of])
    for p in sorted(sample)[:12]:
        slot = arena[int(blob[p]) * S:(int(blob[p]) + 1) * S]
        assert torch.equal(slot, pool[p * S:(p + 1) * S])
    # restore into a fresh 30 GiB region at the same offsets
    target = torch.empty_like(pool)
    tptr = torch.empty_like(ptrs)
    tb = kc.bufs([(target.data_ptr(), target.numel(), kc.BF16, 0), (tptr.data_ptr(), tptr.numel() * 8, kc.RAW, 0)])
    assert ctx.restore(tb, S, table, P, arena, arena.numel()) == kc.OK
    assert ctx.sync() == kc.OK
    assert torch.equal(target, pool) and torch.equal(tptr, ptrs)
    del target, tptr, arena


def test_moe_compare_bf16(ctx):
    pairs = W.moe_pairs(0)
    out = torch.empty(len(pairs) * 64, dtype=torch.uint8, device="cuda")
    gb = kc.bufs([(g.data_ptr(), g.numel() * 2, kc.BF16, 0) for g, _, _ in pairs])
    wb = kc.bufs([(w.data_ptr(), w.numel() * 2, kc.BF16, 0) for _, w, _ in pairs])
    assert ctx.compare(gb, wb, 0.0, 0.0, out) == kc.OK
    assert ctx.sync() == kc.OK
    recs = G.to_np(out).view(kc.CMP_DTYPE)
    for rec, (g, w, truth) in zip(recs, pairs):
        o = oracle.compare(g.view(torch.int16).cpu().numpy(), w.view(torch.int16).cpu().numpy(), W.DT_BF16)
        assert rec.tobytes() == o.tobytes()
        assert rec["mismatches"] == len(truth["perturbed"])
        assert rec["first"] == (int(truth["perturbed"][0]) if len(truth["perturbed"]) else -1)
