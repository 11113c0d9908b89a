"""Pins of the oracle's XXH64 and page digest against things other than itself.

- XXH64 values against the system libxxhash (the xxHash project's own
  implementation of the public specification), over every tail path of the
  algorithm (lengths 0..70, stripe and page edges) and several seeds.
- Page splitting against the closed form ceil(bytes / S).
- Zero flags against the pages the generator planted as zero.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2605_03208_gb300 import workloads as W
from tests._xxh_ref import load as load_xxh

xxh_ref = load_xxh()
needs_xxh = pytest.mark.skipif(xxh_ref is None, reason="libxxhash not present on this host")

EDGE_LENGTHS = (list(range(0, 71)) + [95, 96, 97, 127, 128, 129, 255, 256, 257, 1000,
                                      4095, 4096, 4097, 65535, 65536, 65537])


@needs_xxh
@pytest.mark.parametrize("seed", [0, 1, 0x9E3779B97F4A7C15, 2**64 - 1])
def test_xxh64_matches_libxxhash(seed):
    rng = np.random.default_rng(seed & 0xFFFF)
    for n in EDGE_LENGTHS:
        data = rng.integers(0, 256, n, dtype=np.uint8).tobytes()
        assert oracle.xxh64(data, seed) == xxh_ref(data, seed), (n, seed)


@needs_xxh
def test_xxh64_structured_inputs():
    # all-zero, all-0xFF and repeating patterns exercise the same lanes with
    # equal words; a transposed lane or a wrong rotation breaks them.
    for n in (1, 4, 8, 31, 32, 33, 64, 4096):
        for fill in (0x00, 0xFF, 0x5A):
            data = bytes([fill]) * n
            assert oracle.xxh64(data) == xxh_ref(data), (n, fill)
        data = bytes(range(256)) * (n // 256 + 1)
        data = data[:n]
        assert oracle.xxh64(data) == xxh_ref(data), n


def test_page_first_closed_form():
    rng = np.random.default_rng(3)
    for S in (4096, 65536, 2 * 1024 * 1024):
        sizes = rng.integers(1, 5 * S, 37)
        pf = oracle.page_first(sizes, S)
        expect = np.concatenate([[0], np.cumsum([-(-int(s) // S) for s in sizes])])
        assert np.array_equal(pf, expect.astype(np.uint64))


def _tiny(seed=0):
    snap = W.tiny_layout(seed)
    return W.tiny_fill(snap, W.fake_bases(snap.sizes, seed), seed)


@needs_xxh
def test_digest_pages_match_libxxhash_and_planted_zero_pages():
    snap = _tiny(0)
    S = snap.page_bytes
    h, z, pf = oracle.digest(snap.regions, S)
    assert pf[-1] == len(h)
    pid = 0
    for r in snap.regions:
        for off in range(0, r.size, S):
            page = r[off:off + S].tobytes()
            assert int(h[pid]) == xxh_ref(page, 0), pid
            pid += 1
    planted = set(snap.truth["zero_pages"])
    assert set(np.nonzero(z)[0].tolist()) == planted
    assert len(planted) > 0


def test_digest_partial_pages_are_not_padded():
    # A last page of 5 bytes must hash as 5 bytes, not as 5 bytes plus zeros.
    r = np.zeros(4096 + 5, dtype=np.uint8)
    r[4096:] = [1, 2, 3, 4, 5]
    h, z, _ = oracle.digest([r], 4096)
    assert h[1] == oracle.xxh64(bytes([1, 2, 3, 4, 5]))
    assert h[1] != oracle.xxh64(bytes([1, 2, 3, 4, 5]) + bytes(4096 - 5))
    assert list(z) == [1, 0]
    # an all-zero page is still hashed: XXH64 of that many zero bytes
    assert h[0] == oracle.xxh64(bytes(4096))


def _golden_rows():
    path = os.path.join(os.path.dirname(__file__), "golden", "xxh64_edges.txt")
    with open(path) as f:
        return [tuple(int(x, 0) for x in line.split()) for line in f if line.strip() and not line.startswith("#")]


def _pattern(n):
    return bytes((i * 131 + 7) % 251 for i in range(n))


def test_golden_xxh64_edges_reproduced_by_oracle():
    """The stored values are the oracle's (regression guard for the file)."""
    rows = _golden_rows()
    assert len(rows) == 4 * 87
    for n, seed, h in rows:
        assert oracle.xxh64(_pattern(n), seed) == h


@needs_xxh
def test_golden_xxh64_edges_match_libxxhash():
    """The stored values agree with the xxHash project's implementation, so the
    GPU tests that compare kc_digest with the file are pinned where libxxhash
    is not installed."""
    for n, seed, h in _golden_rows():
        assert xxh_ref(_pattern(n), seed) == h


def test_zero_flag_is_every_byte_of_the_page():
    """The zero flag by construction: a page with exactly one non-zero byte
    (first, second, middle or last byte of a full page; last byte of a
    partial page) is not zero, an all-zero partial page is."""
    S = 4096
    positions = [0, 1, S // 2, S - 1]
    regions = []
    for pos in positions:
        r = np.zeros(S, dtype=np.uint8)
        r[pos] = 1
        regions.append(r)
    tail = np.zeros(S + 100, dtype=np.uint8)
    tail[S + 99] = 0x80
    regions.append(tail)                       # pages: zero, then partial with its last byte set
    regions.append(np.zeros(S + 7, dtype=np.uint8))   # pages: zero, partial zero
    _, z, _ = oracle.digest(regions, S)
    assert z.tolist() == [0, 0, 0, 0, 1, 0, 1, 1]
