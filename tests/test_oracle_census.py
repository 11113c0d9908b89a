"""Pins of the oracle's pointer census.

- Against a brute-force linear scan over all ranges (no sort, no binary
  search), vectorised with numpy.
- Every pointer the generator planted is found, with its target region.
- Truncation keeps the true counts; overlapping ranges are rejected.
- A region whose image is only a prefix (or nothing) is still a whole
  target range: only the image is scanned, values anywhere in the region
  are inside hits.
"""
import numpy as np
import pytest

import oracle
from paper_2605_03208_gb300 import workloads as W


def brute_census(regions, bases, win_lo, win_hi):
    out = []
    starts = np.array(bases, dtype=np.uint64)
    ends = np.array([b + r.size for b, r in zip(bases, regions)], dtype=np.uint64)
    for i, r in enumerate(regions):
        nw = r.size // 8
        w = r[: nw * 8].view("<u8")
        target = np.full(nw, -2, dtype=np.int64)
        for k in range(len(regions)):          # linear scan over every range
            m = (w >= starts[k]) & (w < ends[k])
            target[m] = k
        outside = (target == -2) & (w >= np.uint64(win_lo)) & (w < np.uint64(win_hi))
        target[outside] = -1
        for o in np.nonzero(target != -2)[0]:
            out.append((i, int(o) * 8, int(w[o]), int(target[o])))
    return out


def _as_tuples(hits):
    return [(int(h["src_alloc"]), int(h["src_offset"]), int(h["value"]), int(h["target"]))
            for h in hits]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_census_matches_linear_scan(seed):
    snap = W.tiny_layout(seed, n=10, total=2 * W.MiB)
    snap = W.tiny_fill(snap, W.fake_bases(snap.sizes, seed), seed, p_ptr=0.3)
    lo, hi = W.default_window(snap.bases, snap.sizes)
    hits, nin, nout, rc = oracle.census(snap.regions, snap.bases, lo, hi)
    assert rc == 0
    brute = brute_census(snap.regions, snap.bases, lo, hi)
    assert _as_tuples(hits) == brute
    assert nin == sum(1 for b in brute if b[3] >= 0)
    assert nout == sum(1 for b in brute if b[3] == -1)


def test_census_finds_every_planted_pointer():
    snap = W.tiny_layout(0)
    snap = W.tiny_fill(snap, W.fake_bases(snap.sizes, 0), 0)
    lo, hi = W.default_window(snap.bases, snap.sizes)
    hits, nin, nout, rc = oracle.census(snap.regions, snap.bases, lo, hi)
    got = set(_as_tuples(hits))
    planted = set(snap.truth["pointers"])
    assert planted and planted <= got
    assert any(p[3] == -1 for p in planted)


def test_census_llama_pointer_table():
    snap = W.llama_layout(0, variant="152MB")
    snap = W.llama_fill(snap, W.fake_bases(snap.sizes, 0), 0)
    lo, hi = W.default_window(snap.bases, snap.sizes)
    hits, nin, nout, rc = oracle.census(snap.regions, snap.bases, lo, hi)
    assert rc == 0
    assert set(snap.truth["pointers"]) <= set(_as_tuples(hits))


def test_census_half_open_ranges_and_window():
    base = [0x10000, 0x20000]
    r0 = np.zeros(64, dtype=np.uint8)
    vals = np.array([0x10000, 0x10000 + 63, 0x10000 + 64, 0x1FFFF, 0x20000, 0x5, 0x30000, 0],
                    dtype=np.uint64)
    r0[:] = vals.view(np.uint8)
    r1 = np.zeros(20, dtype=np.uint8)           # 2 whole words, 4 trailing bytes skipped
    r1[:16] = np.array([0x20000 + 19, 0x20000 + 20], dtype=np.uint64).view(np.uint8)
    r1[16:] = 0xFF
    hits, nin, nout, rc = oracle.census([r0, r1], base, 0x8000, 0x28000)
    t = _as_tuples(hits)
    assert t == [(0, 0, 0x10000, 0), (0, 8, 0x1003F, 0), (0, 16, 0x10040, -1),
                 (0, 24, 0x1FFFF, -1), (0, 32, 0x20000, 1), (1, 0, 0x20013, 1),
                 (1, 8, 0x20014, -1)]
    assert (nin, nout) == (4, 3)


def test_census_window_edges():
    """The window is half-open too: win_lo itself is an outside hit, the
    last word below win_hi is, win_hi and the word below win_lo are not."""
    base = [0x100000]
    lo, hi = 0x8000, 0x28000
    vals = np.array([lo, lo - 8, hi - 8, hi, hi - 1, lo + 1], dtype=np.uint64)
    r0 = vals.view(np.uint8).copy()
    hits, nin, nout, rc = oracle.census([r0], base, lo, hi)
    assert _as_tuples(hits) == [(0, 0, lo, -1), (0, 16, hi - 8, -1), (0, 32, hi - 1, -1), (0, 40, lo + 1, -1)]
    assert (nin, nout, rc) == (0, 4, 0)


def test_census_truncation_keeps_true_counts_and_overlap_rejected():
    snap = W.tiny_layout(1, n=6, total=1 * W.MiB)
    snap = W.tiny_fill(snap, W.fake_bases(snap.sizes, 1), 1, p_ptr=0.5)
    lo, hi = W.default_window(snap.bases, snap.sizes)
    full, nin, nout, rc = oracle.census(snap.regions, snap.bases, lo, hi)
    assert rc == 0 and len(full) == nin + nout > 10
    part, nin2, nout2, rc2 = oracle.census(snap.regions, snap.bases, lo, hi, cap=10)
    assert rc2 == 4 and (nin2, nout2) == (nin, nout)
    assert _as_tuples(part) == _as_tuples(full[:10])
    bad = list(snap.bases)
    bad[1] = bad[0] + 8                 # region 1 now starts inside region 0
    _, _, _, rc3 = oracle.census(snap.regions, bad, lo, hi)
    assert rc3 == 2


def test_census_scan_prefix_and_target_only():
    """Regions given as a prefix of their bytes (the oracle's `scan` lengths):
    the region stays a whole half-open target range, only the prefix is read.
    Region 1 passes its first 1 KiB of 8 KiB (its rest holds pointers that
    must not be read), region 2 passes nothing (a target only); words of
    region 0 point past region 1's prefix and into region 2."""
    bases = [0x100000, 0x200000, 0x300000]
    sizes = [4096, 8192, 4096]
    full = [np.zeros(s, dtype=np.uint8) for s in sizes]
    w0 = full[0].view("<u8")
    w0[0] = 0x200000 + 5000          # inside region 1, past its scanned prefix
    w0[1] = 0x200000 + 8191          # last byte of region 1
    w0[2] = 0x200000 + 8192          # one past region 1: the window
    w0[3] = 0x300000                 # region 2, never scanned itself
    w0[4] = 0x300000 + 4095
    w0[5] = 0x300000 + 4096          # one past region 2: the window
    w0[6] = 0x100000 + 8             # region 0 itself
    w1 = full[1].view("<u8")
    w1[1] = 0x300000 + 16            # inside the prefix: found
    w1[200] = 0x100000               # past the prefix (offset 1600): not read
    w1[1000] = 0x300000 + 8          # past the prefix: not read
    full[2].view("<u8")[:] = 0x100000   # target only: none of these is read
    images = [full[0], full[1][:1024], full[2][:0]]
    lo, hi = 0x80000, 0x380000
    hits, nin, nout, rc = oracle.census(images, bases, lo, hi, sizes=sizes)
    assert rc == 0
    # brute force: a linear scan over every full range, words of the images only
    brute = []
    for i, img in enumerate(images):
        for o in range(0, img.size - img.size % 8, 8):
            v = int(img[o:o + 8].view("<u8")[0])
            tgt = [k for k in range(3) if bases[k] <= v < bases[k] + sizes[k]]
            if tgt:
                brute.append((i, o, v, tgt[0]))
            elif lo <= v < hi:
                brute.append((i, o, v, -1))
    assert _as_tuples(hits) == brute
    assert brute[:7] == [(0, 0, 0x200000 + 5000, 1), (0, 8, 0x200000 + 8191, 1), (0, 16, 0x200000 + 8192, -1),
                         (0, 24, 0x300000, 2), (0, 32, 0x300000 + 4095, 2), (0, 40, 0x300000 + 4096, -1),
                         (0, 48, 0x100000 + 8, 0)]
    assert (1, 8, 0x300000 + 16, 2) in brute and not any(b[0] == 1 and b[1] >= 1024 for b in brute)
    assert not any(b[0] == 2 for b in brute)
    assert (nin, nout) == (sum(1 for b in brute if b[3] >= 0), sum(1 for b in brute if b[3] == -1))
