"""GPU parity: every output of the CUDA path, through the C ABI, against the
CPU oracle on the same seeded inputs.  Integers, hashes, tables, arenas and
hit lists must be bit-exact; the FP64 error maxima too (they are single IEEE
operations and order-independent maxima, so the tolerance is zero).

Sizes: the tiny mixed snapshot (16 regions, ~16 MiB, ragged tails) spans
hundreds of 8-page digest tasks and compare tiles; page sizes 4 KiB..2 MiB
and forced kernel shapes cover one-stage to deep rings.
"""
import os

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


@pytest.fixture(scope="module")
def tiny():
    snap, dev = G.device_snapshot(W.tiny_layout(0), W.tiny_fill, 0)
    return snap, dev


def _oracle_digest(snap, S):
    return oracle.digest(snap.regions, S)


# ---------------------------------------------------------------- digest

@pytest.mark.parametrize("S", [4096, 65536, 2 * 1024 * 1024])
def test_digest_tiny_bit_exact(ctx, tiny, S):
    snap, dev = tiny
    st, h, z, pf = G.run_digest(ctx, snap, dev, S)
    assert st == kc.OK
    oh, oz, opf = _oracle_digest(snap, S)
    assert np.array_equal(pf, opf)
    assert np.array_equal(z, oz)
    assert np.array_equal(h, oh)
    assert ctx.sync() == kc.OK


@pytest.mark.parametrize("shape", [(1, 2, 256, 1), (2, 3, 512, 1), (4, 4, 1024, 1), (4, 2, 2048, 1),
                                   (3, 5, 384, 1), (16, 2, 256, 1), (8, 3, 1024, 1), (6, 3, 640, 1),
                                   (1, 3, 8192, 1), (2, 2, 4096, 0), (5, 8, 512, 1)])
def test_digest_forced_shapes(ctx, tiny, shape):
    """Hash warps per CTA (plus the producer warp), ring stages and chunk
    bytes change speed only: one stage in flight to deep rings, chunks that
    are and are not a compile-time size, one to sixteen hash warps."""
    snap, dev = tiny
    with pytest.raises(kc.KcError):
        ctx.set_digest_shape(2, 4, 1024, 2)    # two lanes per thread: no longer offered
    ctx.set_digest_shape(*shape)
    try:
        st, h, z, pf = G.run_digest(ctx, snap, dev, 65536)
    finally:
        ctx.set_digest_shape(0, 0, 0, 0)
    oh, oz, _ = _oracle_digest(snap, 65536)
    assert st == kc.OK and np.array_equal(h, oh) and np.array_equal(z, oz)


def test_digest_edge_lengths(ctx):
    sizes = [1, 7, 8, 15, 16, 31, 32, 33, 63, 64, 100, 4095, 4096, 4097, 8191, 12288 + 40, 70000]
    rng = np.random.default_rng(11)
    regions = [rng.integers(0, 256, s, dtype=np.uint8) for s in sizes]
    regions[5][:] = 0                      # an all-zero short page
    regions[13][4096:8191] = 0             # a zero second page
    dev = [torch.from_numpy(r).cuda() for r in regions]
    snap = W.Snapshot("edge", 4096, sizes, [t.data_ptr() for t in dev], regions, [kc.RAW] * len(sizes))
    for S in (4096, 8192):
        st, h, z, pf = G.run_digest(ctx, snap, dev, S)
        oh, oz, opf = _oracle_digest(snap, S)
        assert st == kc.OK
        assert np.array_equal(h, oh) and np.array_equal(z, oz) and np.array_equal(pf, opf)


def _golden_xxh64():
    path = os.path.join(os.path.dirname(__file__), "golden", "xxh64_edges.txt")
    rows = []
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                n, seed, h = line.split()
                rows.append((int(n), int(seed, 16), int(h, 16)))
    return rows


def test_digest_golden_xxh64_edges(ctx):
    """kc_digest against the stored XXH64 values (seed 0) of every tail path:
    one region per length, a page size above every length, so each region is
    one page whose hash is XXH64 of the whole region."""
    rows = [(n, h) for n, seed, h in _golden_xxh64() if seed == 0 and n > 0]
    regions = [((np.arange(n, dtype=np.int64) * 131 + 7) % 251).astype(np.uint8) for n, _ in rows]
    dev = [torch.from_numpy(r).cuda() for r in regions]
    sizes = [n for n, _ in rows]
    snap = W.Snapshot("golden-edges", 131072, sizes, [t.data_ptr() for t in dev], regions, [kc.RAW] * len(sizes))
    st, h, z, pf = G.run_digest(ctx, snap, dev, 131072)
    assert st == kc.OK and ctx.sync() == kc.OK
    assert np.array_equal(pf, np.arange(len(rows) + 1))
    assert [int(x) for x in h.view(np.uint64)] == [hv for _, hv in rows]
    assert not z.any()


# ---------------------------------------------------------------- census

def test_scan_fused_matches_digest_and_census(ctx, tiny):
    snap, dev = tiny
    win = W.default_window(snap.bases, snap.sizes)
    st, r = G.run_scan(ctx, snap, dev, win)
    assert st == kc.OK and ctx.sync() == kc.OK
    oh, oz, opf = _oracle_digest(snap, snap.page_bytes)
    assert np.array_equal(r["hash"], oh) and np.array_equal(r["zero"], oz)
    hits, nin, nout, rc = oracle.census(snap.regions, snap.bases, *win)
    assert rc == 0
    assert (int(r["counts"][0]), int(r["counts"][1])) == (nin, nout)
    n = nin + nout
    assert G.hits_tuples(r["hits"][:n]) == G.hits_tuples(hits)
    assert set(snap.truth["pointers"]) <= set(G.hits_tuples(r["hits"][:n]))


@pytest.mark.parametrize("page", [4096, 65536])
def test_scan_dense_pointers_many_chunks(ctx, page):
    """The fused scan's census tail over many chunks of pages, most of them
    holding hits (look-back across chunks), with truncation and count-only."""
    layout = W.tiny_layout(3, n=12, total=6 * W.MiB)
    snap, dev = G.device_snapshot(layout, W.tiny_fill, 3, p_ptr=0.6, p_zero=0.1)
    win = W.default_window(snap.bases, snap.sizes)
    ohits, nin, nout, rc = oracle.census(snap.regions, snap.bases, *win)
    assert nin + nout > 100000
    st, r = G.run_scan(ctx, snap, dev, win, page_bytes=page)
    assert ctx.sync() == kc.OK
    assert (int(r["counts"][0]), int(r["counts"][1])) == (nin, nout)
    assert G.hits_tuples(r["hits"][: nin + nout]) == G.hits_tuples(ohits)
    oh, oz, _ = _oracle_digest(snap, page)
    assert np.array_equal(r["hash"], oh) and np.array_equal(r["zero"], oz)
    cap = 777
    st, r = G.run_scan(ctx, snap, dev, win, cap=cap, page_bytes=page)
    assert ctx.sync() == kc.ETRUNC
    assert (int(r["counts"][0]), int(r["counts"][1])) == (nin, nout)
    assert G.hits_tuples(r["hits"][:cap]) == G.hits_tuples(ohits[:cap])
    st, r = G.run_scan(ctx, snap, dev, win, cap=0, page_bytes=page)
    assert ctx.sync() == kc.OK and (int(r["counts"][0]), int(r["counts"][1])) == (nin, nout)


def _sparse_pointer_fill(snap, bases, seed=0, n_ptr=1000):
    """Random bytes with n_ptr pointer words planted at random 8-byte
    offsets, plus an inside pointer in every word of each region's end past
    its last full 32-byte stripe."""
    rng = np.random.default_rng(seed + 5)
    snap.bases = [int(b) for b in bases]
    regions = [rng.integers(0, 256, s, dtype=np.uint8) for s in snap.sizes]
    weight = np.array(snap.sizes, dtype=np.float64) / sum(snap.sizes)
    for _ in range(n_ptr):
        i = int(rng.choice(len(snap.sizes), p=weight))
        w = int(rng.integers(0, snap.sizes[i] // 8))
        if rng.random() < 0.1:
            v = W._outside_value(rng, snap.bases, snap.sizes)
        else:
            v, _ = W._inside_value(rng, snap.bases, snap.sizes)
        regions[i][8 * w:8 * w + 8] = np.array([v], np.uint64).view(np.uint8)
    for i, s in enumerate(snap.sizes):
        for o in range(s & ~31, s - 7, 8):
            v, _ = W._inside_value(rng, snap.bases, snap.sizes)
            regions[i][o:o + 8] = np.array([v], np.uint64).view(np.uint8)
    snap.regions = regions
    snap.truth = {}
    return snap


@pytest.mark.parametrize("page", [4096, 2 * W.MiB])
@pytest.mark.parametrize("n_ptr", [300, 3000, 6000])
def test_scan_sparse_pointers(ctx, page, n_ptr):
    """Sparse pointers (300 to 6000 among random bytes) at 4 KiB and 2 MiB
    pages: hits in the regions' last words (past the last full 32-byte
    stripe, hashed from global memory), truncation, counts only and a lost
    region, all as the oracle's."""
    MiB = W.MiB
    sizes = [MiB + 24, 3 * MiB + 8, 517 * 4096 + 16, 64 * 1024 + 8, 40]
    layout = W.Snapshot("census-log", page, sizes, dtypes=[kc.RAW] * len(sizes))
    snap, dev = G.device_snapshot(layout, _sparse_pointer_fill, 11, n_ptr=n_ptr)
    win = W.default_window(snap.bases, snap.sizes)
    ohits, nin, nout, rc = oracle.census(snap.regions, snap.bases, *win)
    assert rc == 0 and nin + nout >= n_ptr * 0.9
    oh, oz, _ = _oracle_digest(snap, page)
    st, r = G.run_scan(ctx, snap, dev, win, page_bytes=page)
    assert st == kc.OK and ctx.sync() == kc.OK
    assert (int(r["counts"][0]), int(r["counts"][1])) == (nin, nout)
    assert G.hits_tuples(r["hits"][: nin + nout]) == G.hits_tuples(ohits)
    assert np.array_equal(r["hash"], oh) and np.array_equal(r["zero"], oz)
    st, r = G.run_scan(ctx, snap, dev, win, cap=100, page_bytes=page)
    assert ctx.sync() == kc.ETRUNC
    assert (int(r["counts"][0]), int(r["counts"][1])) == (nin, nout)
    assert G.hits_tuples(r["hits"][:100]) == G.hits_tuples(ohits[:100])
    st, r = G.run_scan(ctx, snap, dev, win, cap=0, page_bytes=page)
    assert ctx.sync() == kc.OK and (int(r["counts"][0]), int(r["counts"][1])) == (nin, nout)
    # region 1 lost: not scanned, still a target
    flags = [0, kc.BUF_LOST, 0, 0, 0]
    st, r = G.run_scan(ctx, snap, dev, win, page_bytes=page, flags=flags)
    assert st == kc.EBUF and ctx.sync() == kc.OK
    keep = [x for x in G.hits_tuples(ohits) if x[0] != 1]
    assert G.hits_tuples(r["hits"][: len(keep)]) == keep
    assert int(r["counts"][0]) + int(r["counts"][1]) == len(keep)


def test_scan_list_mode_several_rounds(ctx):
    """Up to 65536 pages the census tail numbers the flagged pages itself and
    deals them out 1 to 32 per chunk; with more flagged pages than the grid
    takes in one round (12,289 pages, about 96% of them holding one of 40,000
    planted pointers) CTAs take further chunks by ticket.  Hits, counts and
    truncation as the oracle's."""
    MiB = W.MiB
    sizes = [20 * MiB + 8, 28 * MiB - 40]
    layout = W.Snapshot("list-rounds", 4096, sizes, dtypes=[kc.RAW] * len(sizes))
    snap, dev = G.device_snapshot(layout, _sparse_pointer_fill, 9, n_ptr=40000)
    npages = sum(-(-s // 4096) for s in sizes)
    assert 304 * 32 < npages <= 65536
    win = W.default_window(snap.bases, snap.sizes)
    ohits, nin, nout, rc = oracle.census(snap.regions, snap.bases, *win)
    assert rc == 0 and nin + nout > 36000
    hit_pages = {(h[0], h[1] // 4096) for h in G.hits_tuples(ohits)}
    assert len(hit_pages) > 304 * 32
    st, r = G.run_scan(ctx, snap, dev, win, cap=nin + nout)
    assert st == kc.OK and ctx.sync() == kc.OK
    assert (int(r["counts"][0]), int(r["counts"][1])) == (nin, nout)
    assert G.hits_tuples(r["hits"][: nin + nout]) == G.hits_tuples(ohits)
    cap = 4321
    st, r = G.run_scan(ctx, snap, dev, win, cap=cap)
    assert ctx.sync() == kc.ETRUNC
    assert (int(r["counts"][0]), int(r["counts"][1])) == (nin, nout)
    assert G.hits_tuples(r["hits"][:cap]) == G.hits_tuples(ohits[:cap])


def test_scan_page_mode_above_list_limit(ctx):
    """More than 65536 pages: the fused scan's census tail takes chunks of
    consecutive pages (page mode) instead of the list of flagged pages; hits,
    counts and digests as the oracle's, and truncation keeps the first hits."""
    MiB = W.MiB
    sizes = [96 * MiB + 8, 64 * MiB - 40, 80 * MiB + 1234, 60 * MiB]
    layout = W.Snapshot("page-mode", 4096, sizes, dtypes=[kc.RAW] * len(sizes))
    snap, dev = G.device_snapshot(layout, W.tiny_fill, 7, p_ptr=0.02, p_zero=0.1)
    assert sum(-(-s // 4096) for s in sizes) > 65536
    win = W.default_window(snap.bases, snap.sizes)
    ohits, nin, nout, rc = oracle.census(snap.regions, snap.bases, *win)
    assert rc == 0 and nin + nout > 100000
    st, r = G.run_scan(ctx, snap, dev, win, cap=nin + nout)
    assert st == kc.OK and ctx.sync() == kc.OK
    assert (int(r["counts"][0]), int(r["counts"][1])) == (nin, nout)
    assert G.hits_tuples(r["hits"][: nin + nout]) == G.hits_tuples(ohits)
    oh, oz, _ = _oracle_digest(snap, 4096)
    assert np.array_equal(r["hash"], oh) and np.array_equal(r["zero"], oz)
    cap = 12345
    st, r = G.run_scan(ctx, snap, dev, win, cap=cap)
    assert ctx.sync() == kc.ETRUNC
    assert (int(r["counts"][0]), int(r["counts"][1])) == (nin, nout)
    assert G.hits_tuples(r["hits"][:cap]) == G.hits_tuples(ohits[:cap])
    # the bounded look-back wait in page mode: chunk 0 never published
    ctx.debug_stall_census(2000)
    st, r = G.run_scan(ctx, snap, dev, win, cap=nin + nout)
    assert st == kc.OK and ctx.sync() == kc.ETIMEOUT
    assert np.array_equal(r["hash"], oh)


def test_scan_census_bounded_wait_times_out(ctx):
    """The census tail's look-back waits are bounded: with the test hook, the
    first chunk of flagged pages is never published and every wait is cut
    at 2000 polls; the chunks behind it give up, the kernel finishes and
    kc_sync reports KC_ETIMEOUT (the digest of that call is still exact).
    The context stays usable: the next scan is exact again."""
    layout = W.tiny_layout(3, n=12, total=6 * W.MiB)
    snap, dev = G.device_snapshot(layout, W.tiny_fill, 3, p_ptr=0.6, p_zero=0.1)
    win = W.default_window(snap.bases, snap.sizes)
    ohits, nin, nout, rc = oracle.census(snap.regions, snap.bases, *win)
    oh, oz, _ = _oracle_digest(snap, 4096)
    ctx.debug_stall_census(2000)
    st, r = G.run_scan(ctx, snap, dev, win, page_bytes=4096)
    assert st == kc.OK and ctx.sync() == kc.ETIMEOUT
    assert np.array_equal(r["hash"], oh) and np.array_equal(r["zero"], oz)
    st, r = G.run_scan(ctx, snap, dev, win, page_bytes=4096)
    assert ctx.sync() == kc.OK
    assert (int(r["counts"][0]), int(r["counts"][1])) == (nin, nout)
    assert G.hits_tuples(r["hits"][: nin + nout]) == G.hits_tuples(ohits)
    with pytest.raises(kc.KcError):
        ctx.debug_stall_census(0)


def test_census_standalone(ctx, tiny):
    snap, dev = tiny
    win = W.default_window(snap.bases, snap.sizes)
    st, hits, counts = G.run_census(ctx, snap, dev, win)
    assert st == kc.OK and ctx.sync() == kc.OK
    ohits, nin, nout, rc = oracle.census(snap.regions, snap.bases, *win)
    assert (int(counts[0]), int(counts[1])) == (nin, nout)
    assert G.hits_tuples(hits[: nin + nout]) == G.hits_tuples(ohits)


def _edge_fill(snap, bases, seed=0):
    """Random bytes, with words at and next to every region's first and last
    byte, at the quarter points of the gaps between regions, and at the
    boundaries of 2^16 equal buckets over the regions' hull (around each
    region's ends), planted as 8-byte words in the two largest regions."""
    rng = np.random.default_rng(seed + 3)
    snap.bases = [int(b) for b in bases]
    lo = min(snap.bases)
    hi = max(b + s for b, s in zip(snap.bases, snap.sizes))
    shift = 0
    while ((hi - lo - 1) >> shift) >= 1 << 16:
        shift += 1
    vals = []
    for b, s in zip(snap.bases, snap.sizes):
        vals += [b - 8, b - 1, b, b + 1, b + s - 8, b + s - 1, b + s, b + s + 1, b + s + 8]
        for e in (b, b + s):
            k = (e - lo) >> shift
            for kk in (k - 1, k, k + 1, k + 2):
                x = lo + (kk << shift)
                vals += [x - 1, x, x + 1]
    order = sorted(zip(snap.bases, snap.sizes))
    for (b0, s0), (b1, _) in zip(order, order[1:]):
        if b1 > b0 + s0:
            vals += [b0 + s0 + (b1 - b0 - s0) * q // 4 for q in (1, 2, 3)]
    vals += [lo - 1, hi, hi + 1, 0, 2 ** 64 - 1]
    vals = np.array([v % 2 ** 64 for v in vals], dtype=np.uint64)
    regions = [rng.integers(0, 256, s, dtype=np.uint8) for s in snap.sizes]
    big = sorted(range(len(snap.sizes)), key=lambda i: -snap.sizes[i])[:2]
    for i in big:
        at = rng.choice(snap.sizes[i] // 8, size=len(vals), replace=False) * 8
        for v, o in zip(vals.tolist(), at.tolist()):
            regions[i][o:o + 8] = np.array([v], np.uint64).view(np.uint8)
    snap.regions = regions
    snap.truth = {"values": len(vals)}
    return snap


@pytest.mark.parametrize("page", [4096, 65536])
def test_census_edges_and_gaps(ctx, page):
    """Every planted word classified as the oracle does -- inside, outside or
    no hit -- at region edges, in the gaps between regions and on the
    classifier's bucket boundaries: fused scan and standalone census."""
    MiB, KiB = W.MiB, 1024
    sizes = [4096, 2 * MiB + 8, 64 * KiB, 20 * MiB, 4096 + 8, 3 * MiB, 40]
    layout = W.Snapshot("edges", page, sizes, dtypes=[kc.RAW] * len(sizes))
    snap, dev = G.device_snapshot(layout, _edge_fill, 4)
    win = W.default_window(snap.bases, snap.sizes)
    ohits, nin, nout, rc = oracle.census(snap.regions, snap.bases, *win)
    assert rc == 0 and nin > 0 and nout > 0
    st, r = G.run_scan(ctx, snap, dev, win, page_bytes=page)
    assert st == kc.OK and ctx.sync() == kc.OK
    assert (int(r["counts"][0]), int(r["counts"][1])) == (nin, nout)
    assert G.hits_tuples(r["hits"][: nin + nout]) == G.hits_tuples(ohits)
    st, hits, counts = G.run_census(ctx, snap, dev, win)
    assert st == kc.OK and ctx.sync() == kc.OK
    assert (int(counts[0]), int(counts[1])) == (nin, nout)
    assert G.hits_tuples(hits[: nin + nout]) == G.hits_tuples(ohits)


def test_census_dense_pointers_and_truncation(ctx):
    layout = W.tiny_layout(3, n=12, total=6 * W.MiB)
    snap, dev = G.device_snapshot(layout, W.tiny_fill, 3, p_ptr=0.6, p_zero=0.1)
    win = W.default_window(snap.bases, snap.sizes)
    ohits, nin, nout, rc = oracle.census(snap.regions, snap.bases, *win)
    assert nin + nout > 100000
    st, hits, counts = G.run_census(ctx, snap, dev, win)
    assert ctx.sync() == kc.OK
    assert G.hits_tuples(hits[: nin + nout]) == G.hits_tuples(ohits)
    cap = 1000
    st, hits, counts = G.run_census(ctx, snap, dev, win, cap=cap)
    assert ctx.sync() == kc.ETRUNC
    assert (int(counts[0]), int(counts[1])) == (nin, nout)
    assert G.hits_tuples(hits[:cap]) == G.hits_tuples(ohits[:cap])
    # count-only mode
    st, _, counts = G.run_census(ctx, snap, dev, win, cap=0)
    assert ctx.sync() == kc.OK and (int(counts[0]), int(counts[1])) == (nin, nout)


# ---------------------------------------------------------------- dedup / restore

def _dedup_vs_oracle(ctx, snap, dev, S, hash_bits=64, low_bits=None, xform=None):
    oh, oz, _ = _oracle_digest(snap, S)
    if xform is not None:
        oh = xform(oh)
    if hash_bits < 64:
        oh = oh & np.uint64((1 << hash_bits) - 1)
    if low_bits is not None:
        # keep the high 32 bits, squeeze the low 32 bits to a few values:
        # different hashes that agree on their low half
        oh = (oh & np.uint64(0xFFFFFFFF00000000)) | (oh & np.uint64((1 << low_bits) - 1))
    # the oracle's digest is the input of both sides
    h_dev = torch.from_numpy(oh.view(np.int64).copy()).cuda()
    z_dev = torch.from_numpy(oz.copy()).cuda()
    st, t, arena, nb = G.run_dedup(ctx, snap, dev, h_dev, z_dev, S)
    assert st == kc.OK and ctx.sync() == kc.OK
    ot = oracle.dedup(snap.regions, S, oh, oz)
    assert nb == ot["n_blobs"]
    assert np.array_equal(t["va_offset"], ot["off"])
    assert np.array_equal(t["alloc_id"], ot["alloc"])
    assert np.array_equal(t["blob"], ot["blob"])
    oarena = oracle.pack(snap.regions, S, ot)
    assert np.array_equal(G.to_np(arena)[: nb * S], oarena)
    return t, arena, nb


@pytest.mark.parametrize("S", [4096, 65536])
def test_dedup_tiny(ctx, tiny, S):
    snap, dev = tiny
    _dedup_vs_oracle(ctx, snap, dev, S)


@pytest.mark.parametrize("bits", [0, 3, 8])
def test_dedup_forced_collisions(ctx, tiny, bits):
    snap, dev = tiny
    _dedup_vs_oracle(ctx, snap, dev, 65536, hash_bits=bits)


@pytest.mark.parametrize("low_bits", [0, 2])
def test_dedup_low_half_collisions(ctx, tiny, low_bits):
    """Distinct hashes sharing their low 32 bits interleave in the sorted
    order; the result must still be the byte-defined classes."""
    snap, dev = tiny
    _dedup_vs_oracle(ctx, snap, dev, 4096, low_bits=low_bits)


def test_dedup_no_shared_keys(ctx):
    """No copies: every data page is its own class, and the grouping kernel's
    own table (data pages numbered in page order) is the result."""
    snap, dev = G.device_snapshot(W.tiny_layout(3), W.tiny_fill, 3, p_copy=0.0)
    t, _, nb = _dedup_vs_oracle(ctx, snap, dev, 4096)
    data = t["blob"][t["blob"] < kc.BLOB_LOST]
    assert nb == len(data) and np.array_equal(data, np.arange(nb))


@pytest.mark.parametrize("every", [1, 3])
def test_dedup_empty_marker_key(ctx, tiny, every):
    """Hashes whose low 32 bits equal the table's empty-slot marker (all ones)
    are grouped outside the table; mixed with ordinary keys (every 3rd page)
    and alone (every page).  All such pages form one group that fails its
    byte comparison, so the exact slow path splits it (64 KiB pages keep that
    quadratic split small)."""
    snap, dev = tiny

    def xform(oh):
        oh = oh.copy()
        oh[::every] |= np.uint64(0xFFFFFFFF)
        return oh
    _dedup_vs_oracle(ctx, snap, dev, 65536, xform=xform)


def test_dedup_tiled_sort_path(ctx):
    # > 8192 non-zero pages: the multi-CTA radix sort passes
    layout = W.tiny_layout(5, n=40, total=64 * W.MiB, page_bytes=4096)
    snap, dev = G.device_snapshot(layout, W.tiny_fill, 5)
    assert sum(-(-s // 4096) for s in snap.sizes) > 9000
    _dedup_vs_oracle(ctx, snap, dev, 4096)
    _dedup_vs_oracle(ctx, snap, dev, 4096, hash_bits=12)
    _dedup_vs_oracle(ctx, snap, dev, 4096, low_bits=6)


def test_restore_roundtrip(ctx, tiny):
    snap, dev = tiny
    S = snap.page_bytes
    t, arena, nb = _dedup_vs_oracle(ctx, snap, dev, S)
    table = torch.from_numpy(t.view(np.uint8).copy()).cuda()
    targets = [torch.full_like(x, 0xA5) for x in dev]
    b = G.region_bufs(snap, targets)
    st = ctx.restore(b, S, table, len(t), arena, nb * S)
    assert st == kc.OK and ctx.sync() == kc.OK
    for tg, r in zip(targets, snap.regions):
        assert np.array_equal(G.to_np(tg), r)


def test_restore_rejects_bad_rows(ctx, tiny):
    snap, dev = tiny
    S = snap.page_bytes
    targets = [torch.full_like(x, 0xA5) for x in dev[:2]]
    rows = np.zeros(4, dtype=kc.PAGE_DTYPE)
    rows[0] = (0, 0, kc.BLOB_ZERO)                 # fine: zeros
    rows[1] = (0, 7, kc.BLOB_ZERO)                 # region 7 does not exist in this list
    rows[2] = (1 << 40, 0, kc.BLOB_ZERO)           # offset beyond the region
    rows[3] = (0, 1, 1000)                         # blob beyond the arena
    arena = torch.zeros(S, dtype=torch.uint8, device="cuda")
    b = G.region_bufs(W.Snapshot("x", S, snap.sizes[:2], dtypes=[kc.RAW] * 2), targets)
    ctx.restore(b, S, torch.from_numpy(rows.view(np.uint8).copy()).cuda(), 4, arena, S)
    assert ctx.sync() == kc.EINVAL
    t0 = G.to_np(targets[0])
    assert (t0[: min(S, t0.size)] == 0).all()
    assert (G.to_np(targets[1]) == 0xA5).all()


# ---------------------------------------------------------------- compare

def _cmp_gpu(ctx, pairs, atol=0.0, rtol=0.0):
    g = [torch.from_numpy(np.ascontiguousarray(p.got).view(np.uint8)).cuda() for p in pairs]
    w = [torch.from_numpy(np.ascontiguousarray(p.want).view(np.uint8)).cuda() for p in pairs]
    gb = kc.bufs([(x.data_ptr(), x.numel(), p.dtype, 0) for x, p in zip(g, pairs)])
    wb = kc.bufs([(x.data_ptr(), x.numel(), p.dtype, 0) for x, p in zip(w, pairs)])
    out = torch.empty(len(pairs) * 64, dtype=torch.uint8, device="cuda")
    st = ctx.compare(gb, wb, atol, rtol, out)
    assert st == kc.OK and ctx.sync() == kc.OK
    return G.to_np(out).view(kc.CMP_DTYPE)


def _assert_records_equal(got, want):
    assert got.tobytes() == want.tobytes(), (got, want)


def test_compare_tiny_pairs(ctx):
    pairs = W.tiny_pairs(0)
    recs = _cmp_gpu(ctx, pairs)
    for rec, p in zip(recs, pairs):
        _assert_records_equal(rec, oracle.compare(p.got, p.want, p.dtype))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_compare_mixed_dtypes_ragged(ctx, seed):
    pairs = W.mixed_pairs(seed, n_pairs=15, max_elems=300_000)
    recs = _cmp_gpu(ctx, pairs)
    for rec, p in zip(recs, pairs):
        _assert_records_equal(rec, oracle.compare(p.got, p.want, p.dtype))


@pytest.mark.parametrize("atol,rtol", [(1e-7, 0.0), (0.0, 1e-6), (1e-6, 1e-5)])
def test_compare_tolerances(ctx, atol, rtol):
    pairs = W.tiny_pairs(1, n=1 << 18)
    recs = _cmp_gpu(ctx, pairs, atol, rtol)
    for rec, p in zip(recs, pairs):
        _assert_records_equal(rec, oracle.compare(p.got, p.want, p.dtype, atol, rtol))


@pytest.mark.parametrize("tol", [1e30, 0.0])
def test_compare_special_values(ctx, tol):
    inf, nan = np.inf, np.nan
    g = np.array([0.0, -0.0, inf, inf, -inf, 1.0, nan, nan, 2.0, 3.0, 0.0, 1e-45, 5, 6, 7, 8, 9],
                 dtype=np.float32)
    w = np.array([-0.0, 0.0, inf, -inf, 5.0, inf, nan, 1.0, nan, 3.0, 1.0, 0.0, 5, 6, 7, 8, 9.5],
                 dtype=np.float32)
    h16 = np.array([0x7C00, 0xFC00, 0x7E00, 0x0001, 0x8000, 0x3C00, 0x7BFF, 0x0400], dtype=np.uint16)
    w16 = np.array([0x7C00, 0x7C00, 0x7E01, 0x0000, 0x0000, 0x3C01, 0x7BFE, 0x03FF], dtype=np.uint16)
    pairs = [W.Pair(g, w, W.DT_F32), W.Pair(h16, w16, W.DT_F16), W.Pair(h16, w16, W.DT_BF16),
             W.Pair(np.array([-2**31, 2**31 - 1, 0, 1], np.int32),
                    np.array([2**31 - 1, -2**31, 0, 1], np.int32), W.DT_I32)]
    recs = _cmp_gpu(ctx, pairs, tol, tol)
    for rec, p in zip(recs, pairs):
        _assert_records_equal(rec, oracle.compare(p.got, p.want, p.dtype, tol, tol))


def _near_tie_f32(rng, n, k):
    """k scattered elements of an f32 pair whose relative differences agree
    to about 2^-23 (fp32 cannot order them, FP64 can), plus their indices."""
    want = rng.standard_normal(n).astype(np.float32)
    got = want.copy()
    idx = np.sort(rng.choice(n, k, replace=False))
    b = (1.0 + rng.integers(0, 4096, k) * 2.0**-23).astype(np.float32)   # distinct values just above 1
    want[idx] = b
    got[idx] = (b.astype(np.float64) + 2.0**-10).astype(np.float32)      # exact: the same difference
    return got, want, idx


@pytest.mark.parametrize("seed", [0, 1])
def test_compare_zero_tolerance_maxima_over_many_warps(ctx, seed):
    """Zero tolerances: many scattered differences of every size, near-ties
    that only FP64 orders, NaN / inf / zero / subnormal cases -- the exact
    maxima must come out whichever warps see which elements first."""
    rng = np.random.default_rng(seed + 77)
    n = 1 << 22
    got, want, _ = _near_tie_f32(rng, n, 3000)
    idx = rng.choice(n, 200_000, replace=False)
    got[idx] = (want[idx] * (1 + rng.uniform(-1e-3, 1e-3, idx.size))).astype(np.float32)
    sp = rng.choice(n, 64, replace=False)
    got[sp[:8]] = np.nan
    want[sp[8:16]] = np.nan
    got[sp[16:24]], want[sp[16:24]] = np.nan, np.nan
    got[sp[24:32]], want[sp[24:32]] = 0.0, -0.0
    got[sp[32:40]] = np.inf
    got[sp[40:48]], want[sp[40:48]] = 1e-45, 0.0
    got[sp[48:56]], want[sp[48:56]] = 3e38, -3e38
    want[sp[56:64]] = 0.0
    f32 = W.Pair(got, want, W.DT_F32)
    w32 = rng.integers(-2**31, 2**31, n, dtype=np.int64).astype(np.int32)
    g32 = w32.copy()
    j = rng.choice(n, 50_000, replace=False)
    g32[j] = rng.integers(-2**31, 2**31, j.size, dtype=np.int64).astype(np.int32)
    g32[j[:10]], w32[j[:10]] = 2**31 - 1, -2**31
    g32[j[10:20]], w32[j[10:20]] = 5, 0
    i32 = W.Pair(g32, w32, W.DT_I32)
    w8 = rng.integers(0, 256, n, dtype=np.uint8)
    g8 = w8.copy()
    j = rng.choice(n, 100_000, replace=False)
    g8[j] = rng.integers(0, 256, j.size, dtype=np.uint8)
    u8 = W.Pair(g8, w8, W.DT_U8)
    fb = rng.standard_normal(n).astype(np.float32)
    wb16 = (fb.view(np.uint32) >> 16).astype(np.uint16)
    gb16 = wb16.copy()
    j = rng.choice(n, 29_360, replace=False)
    gb16[j] ^= np.uint16(1)
    bf = W.Pair(gb16, wb16, W.DT_BF16)
    pairs = [f32, i32, u8, bf]
    recs = _cmp_gpu(ctx, pairs)
    for rec, p in zip(recs, pairs):
        _assert_records_equal(rec, oracle.compare(p.got, p.want, p.dtype))


# ---------------------------------------------------------------- failures

def test_lost_region_does_not_disturb_others(ctx, tiny):
    snap, dev = tiny
    flags = [0] * len(dev)
    flags[3] = kc.BUF_LOST
    st, h, z, pf = G.run_digest(ctx, snap, dev, 65536, flags=flags)
    assert st == kc.EBUF
    assert ctx.buf_status(3) == kc.EBUF and ctx.buf_status(2) == kc.OK
    oh, oz, opf = _oracle_digest(snap, 65536)
    lost = np.zeros(len(h), bool)
    lost[int(opf[3]):int(opf[4])] = True
    assert (z[lost] == kc.PAGE_LOST).all() and (h[lost] == 0).all()
    assert np.array_equal(h[~lost], oh[~lost]) and np.array_equal(z[~lost], oz[~lost])
    # the census skips the lost source but keeps it as a target
    win = W.default_window(snap.bases, snap.sizes)
    st, hits, counts = G.run_census(ctx, snap, dev, win, flags=flags)
    assert st == kc.EBUF and ctx.sync() == kc.OK
    ohits, nin, nout, rc = oracle.census(snap.regions, snap.bases, *win)
    keep = [x for x in G.hits_tuples(ohits) if x[0] != 3]
    assert G.hits_tuples(hits[: len(keep)]) == keep


def test_argument_errors(ctx, tiny):
    snap, dev = tiny
    h = torch.empty(1024, dtype=torch.int64, device="cuda")
    z = torch.empty(1024, dtype=torch.uint8, device="cuda")
    bad = kc.bufs([(dev[0].data_ptr() + 8, 100, kc.RAW, 0)])
    assert ctx.digest(bad, 4096, h, z, allow=range(8)) == kc.EINVAL
    assert ctx.digest(G.region_bufs(snap, dev), 3000, h, z, allow=range(8)) == kc.EINVAL
    ov = kc.bufs([(dev[0].data_ptr(), 4096), (dev[0].data_ptr() + 1024, 4096)])
    counts = torch.zeros(2, dtype=torch.int64, device="cuda")
    assert ctx.census(ov, 0, 0, None, 0, counts, allow=range(8)) == kc.EOVERLAP
    assert "overlap" in ctx.last_error()


# ---------------------------------------------------------------- graphs

def test_graph_capture_replays_bit_exact(ctx, tiny):
    """After one uncaptured call of each shape, the calls capture into a CUDA
    graph (no table upload, no scratch growth) and the replay reproduces the
    oracle's results."""
    snap, dev = tiny
    S = snap.page_bytes
    b = G.region_bufs(snap, dev)
    P = kc.page_count(b, S)
    win = W.default_window(snap.bases, snap.sizes)
    cap = sum(int(s) // 8 for s in snap.sizes)
    h = torch.empty(P, dtype=torch.int64, device="cuda")
    z = torch.empty(P, dtype=torch.uint8, device="cuda")
    pf = torch.empty(len(dev) + 1, dtype=torch.int64, device="cuda")
    hits = torch.empty(cap * 24, dtype=torch.uint8, device="cuda")
    counts = torch.zeros(2, dtype=torch.int64, device="cuda")
    table = torch.empty(P * 16, dtype=torch.uint8, device="cuda")
    arena = torch.empty(P * S, dtype=torch.uint8, device="cuda")
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    targets = [torch.full_like(x, 0xA5) for x in dev]
    tb = G.region_bufs(snap, targets)

    def step():
        ctx.scan(b, S, h, z, pf, win[0], win[1], hits, cap, counts)
        ctx.dedup(b, S, h, z, table, arena, P * S, nb)
        ctx.restore(tb, S, table, P, arena, P * S)

    step()
    assert ctx.sync() == kc.OK
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    oh, oz, _ = oracle.digest(snap.regions, S)
    ot = oracle.dedup(snap.regions, S, oh, oz)
    ohits, nin, nout, _ = oracle.census(snap.regions, snap.bases, *win)
    for _ in range(3):   # each replay leaves the state the next one starts from
        for t in (h, z, table, arena, nb, counts):
            t.zero_()
        for t in targets:
            t.fill_(0xA5)
        g.replay()
        torch.cuda.synchronize()
        assert ctx.sync() == kc.OK
        assert np.array_equal(G.to_np(h).view(np.uint64), oh) and np.array_equal(G.to_np(z), oz)
        assert tuple(G.to_np(counts).view(np.uint64)) == (nin, nout)
        got = G.to_np(hits).view(kc.HIT_DTYPE)[: nin + nout]
        assert G.hits_tuples(got) == G.hits_tuples(ohits)
        assert int(G.to_np(nb).view(np.uint64)[0]) == ot["n_blobs"]
        assert np.array_equal(G.to_np(table).view(kc.PAGE_DTYPE)["blob"], ot["blob"])
        for tg, r in zip(targets, snap.regions):
            assert np.array_equal(G.to_np(tg), r)


def test_digest_and_scan_interleave_on_one_context(ctx, tiny):
    """kc_digest and kc_scan take tasks from one counter of the context,
    each leaving it at zero behind its kernels: any order of the two gives
    the oracle's digests, and the scan the oracle's census."""
    snap, dev = tiny
    win = W.default_window(snap.bases, snap.sizes)
    oh, oz, _ = oracle.digest(snap.regions, snap.page_bytes)
    ohits, nin, nout, _ = oracle.census(snap.regions, snap.bases, *win)
    for op in ["scan", "digest", "digest", "scan", "scan", "digest", "scan"]:
        if op == "scan":
            st, r = G.run_scan(ctx, snap, dev, win)
            h, z = r["hash"], r["zero"]
            assert (int(r["counts"][0]), int(r["counts"][1])) == (nin, nout)
            assert G.hits_tuples(r["hits"][: nin + nout]) == G.hits_tuples(ohits)
        else:
            st, h, z, _ = G.run_digest(ctx, snap, dev)
        assert st == kc.OK and ctx.sync() == kc.OK
        assert np.array_equal(h, oh) and np.array_equal(z, oz)
