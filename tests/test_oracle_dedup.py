"""Pins of the oracle's page dedup, pack and restore.

- Dedup against brute-force pairwise page comparison on tiny inputs (at most
  64 pages): canonical(p) = the smallest page id whose bytes (and length)
  equal p's, blob ids in increasing canonical page id.
- Hash collisions forced by handing the oracle truncated hashes: the classes
  must not change, because byte equality decides.
- Planted copies of the generator map to their source.
- restore(pack(dedup(snapshot))) rewrites every byte of sentinel-filled
  targets with the original bytes (round-trip identity).
"""
import numpy as np
import pytest

import oracle
from paper_2605_03208_gb300 import workloads as W


def brute_dedup(regions, S, zero):
    pages = []
    for r in regions:
        for off in range(0, r.size, S):
            pages.append(r[off:off + S].tobytes())
    P = len(pages)
    canon = list(range(P))
    for p in range(P):
        if zero[p]:
            continue
        for q in range(p):
            if not zero[q] and pages[q] == pages[p]:
                canon[p] = q
                break
    blob, nxt = {}, 0
    for p in range(P):
        if not zero[p] and canon[p] == p:
            blob[p] = nxt
            nxt += 1
    tbl_blob = [oracle.BLOB_ZERO if zero[p] else blob[canon[p]] for p in range(P)]
    return canon, tbl_blob, nxt, pages


def small_snapshot(seed, S=4096, npages=48):
    """A few regions of 4 KiB pages with planted copies, equal-prefix partial
    pages, zero pages and random pages."""
    rng = np.random.default_rng(seed)
    sizes = [S * 7 + 100, S * 12, S * 3 + 4000, 100, S * 20 + 8]
    regions = [rng.integers(0, 256, s, dtype=np.uint8) for s in sizes]
    pages = [(i, off) for i, s in enumerate(sizes) for off in range(0, s, S)]
    assert len(pages) <= 64
    for _ in range(15):              # planted full or prefix copies
        (di, do), (si, so) = [pages[k] for k in rng.choice(len(pages), 2, replace=False)]
        ln = min(S, sizes[di] - do, sizes[si] - so)
        regions[di][do:do + ln] = regions[si][so:so + ln]
    for k in rng.choice(len(pages), 6, replace=False):    # zero pages
        i, off = pages[k]
        regions[i][off:off + S] = 0
    # a partial page equal to the prefix of a full page: same bytes, other length
    regions[3][:] = regions[1][:100]
    return regions


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("hash_bits", [64, 2, 0])
def test_dedup_matches_bruteforce(seed, hash_bits):
    S = 4096
    regions = small_snapshot(seed, S)
    h, z, pf = oracle.digest(regions, S)
    if hash_bits < 64:      # force collisions: only `hash_bits` low bits survive
        h = h & np.uint64((1 << hash_bits) - 1)
    t = oracle.dedup(regions, S, h, z)
    canon, tbl_blob, nblobs, pages = brute_dedup(regions, S, z)
    assert t["n_blobs"] == nblobs
    assert [int(c) for c in t["canon"]] == canon
    assert [int(b) for b in t["blob"]] == tbl_blob
    # VA-faithful rows: region index and offset of every page
    k = 0
    for i, r in enumerate(regions):
        for off in range(0, r.size, S):
            assert t["alloc"][k] == i and t["off"][k] == off
            k += 1
    arena = oracle.pack(regions, S, t)
    for p in range(len(pages)):
        if not z[p] and canon[p] == p:
            b = tbl_blob[p]
            slot = arena[b * S:(b + 1) * S].tobytes()
            assert slot[:len(pages[p])] == pages[p]
            assert slot[len(pages[p]):] == bytes(S - len(pages[p]))


def test_dedup_partial_prefix_is_a_separate_class():
    S = 4096
    rng = np.random.default_rng(9)
    a = rng.integers(0, 256, S, dtype=np.uint8)
    b = a[:100].copy()
    h, z, _ = oracle.digest([a, b], S)
    t = oracle.dedup([a, b], S, h * np.uint64(0), z)      # all hashes equal
    assert list(t["canon"]) == [0, 1] and t["n_blobs"] == 2


def _tiny(seed=0):
    snap = W.tiny_layout(seed)
    return W.tiny_fill(snap, W.fake_bases(snap.sizes, seed), seed)


def test_planted_copies_map_to_source_and_roundtrip():
    snap = _tiny(0)
    S = snap.page_bytes
    h, z, pf = oracle.digest(snap.regions, S)
    t = oracle.dedup(snap.regions, S, h, z)
    for dst, src, ln in snap.truth["copies"]:
        if ln == S:
            assert t["canon"][dst] == t["canon"][src]
            assert t["blob"][dst] == t["blob"][src]
    # every zero page is flagged ZERO, nothing else is
    assert set(np.nonzero(t["blob"] == oracle.BLOB_ZERO)[0]) == set(snap.truth["zero_pages"])
    arena = oracle.pack(snap.regions, S, t)
    assert arena.size == t["n_blobs"] * S
    targets = [np.full(r.size, 0xA5, dtype=np.uint8) for r in snap.regions]
    oracle.restore(targets, S, t, arena)
    for a, b in zip(targets, snap.regions):
        assert np.array_equal(a, b)
