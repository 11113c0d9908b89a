"""ctypes wrapper of the plain C oracle (``kc_oracle.c``).

TEST INFRASTRUCTURE ONLY.  This module and the library it builds are used by
the tests, by ``__graft_entry__.smoke()`` and by the benchmark's CPU-baseline
leg; the product path never imports it.

Every function takes host numpy arrays.  A snapshot is a list of regions, each
a ``uint8`` numpy array (the region's bytes) plus the device VA it lives at;
the VA matters only to the census (values are compared with VAs) and is
otherwise just carried along.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kc_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libkc_oracle.so")
_lock = threading.Lock()
_lib = None

BLOB_ZERO = 0xFFFFFFFF
DT_U8, DT_I32, DT_F16, DT_BF16, DT_F32, DT_RAW = 0, 1, 2, 3, 4, 5

HIT_DTYPE = np.dtype([("src_offset", "<u8"), ("value", "<u8"), ("src_alloc", "<u4"),
                      ("target", "<i4")])
CMP_DTYPE = np.dtype([("mismatches", "<u8"), ("first", "<i8"), ("max_abs", "<f8"),
                      ("max_rel", "<f8"), ("nan_got", "<u8"), ("nan_want", "<u8"),
                      ("nan_mismatch", "<u8"), ("status", "<i4"), ("reserved", "<u4")])


def build(force: bool = False) -> str:
    """Compile ``kc_oracle.c`` with gcc (no FMA contraction) and return the path."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load(path: str):
    """Open an oracle library at `path` and declare its functions."""
    L = ctypes.CDLL(path)
    u64, u32, i32, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_void_p
    L.kco_xxh64.restype = u64
    L.kco_xxh64.argtypes = [vp, u64, u64]
    L.kco_page_first.restype = u64
    L.kco_page_first.argtypes = [i32, vp, u32, vp]
    L.kco_digest.restype = None
    L.kco_digest.argtypes = [i32, vp, vp, u32, vp, vp, vp]
    L.kco_dedup.restype = i32
    L.kco_dedup.argtypes = [i32, vp, vp, u32, vp, vp, vp, vp, vp, vp, vp]
    L.kco_pack.restype = None
    L.kco_pack.argtypes = [i32, vp, vp, u32, vp, vp, vp, vp, vp]
    L.kco_restore.restype = None
    L.kco_restore.argtypes = [i32, vp, vp, u32, u64, vp, vp, vp, vp]
    L.kco_census.restype = i32
    L.kco_census.argtypes = [i32, vp, vp, vp, vp, u64, u64, vp, u64, vp, vp]
    L.kco_compare.restype = None
    L.kco_compare.argtypes = [vp, vp, i32, u64, ctypes.c_double, ctypes.c_double, vp]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _load(build())
        return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _region_table(regions):
    """Return (pointer array, bytes array, keep-alive list) for uint8 regions."""
    keep = [np.ascontiguousarray(r, dtype=np.uint8).reshape(-1) for r in regions]
    keep = [r if r.size else np.zeros(1, np.uint8)[:0] for r in keep]
    ptrs = np.array([_ptr(r) if r.size else 0 for r in keep], dtype=np.uint64)
    nbytes = np.array([r.size for r in keep], dtype=np.uint64)
    return ptrs, nbytes, keep


def xxh64(data, seed: int = 0) -> int:
    """XXH64 of a bytes-like object (public xxHash specification)."""
    buf = np.frombuffer(bytes(data), dtype=np.uint8) if not isinstance(data, np.ndarray) \
        else np.ascontiguousarray(data).view(np.uint8).reshape(-1)
    if buf.size == 0:
        buf = np.zeros(1, dtype=np.uint8)
        return int(lib().kco_xxh64(_ptr(buf), 0, seed))
    return int(lib().kco_xxh64(_ptr(buf), buf.size, seed))


def page_first(sizes, page_bytes: int) -> np.ndarray:
    nb = np.asarray(sizes, dtype=np.uint64)
    out = np.zeros(len(nb) + 1, dtype=np.uint64)
    lib().kco_page_first(len(nb), _ptr(nb), page_bytes, _ptr(out))
    return out


def digest(regions, page_bytes: int):
    """Per-page XXH64 (seed 0) and zero flags; returns (hash u64[P], zero u8[P], page_first u64[n+1])."""
    ptrs, nbytes, keep = _region_table(regions)
    pf = page_first(nbytes, page_bytes)
    P = int(pf[-1])
    h = np.zeros(max(P, 1), dtype=np.uint64)
    z = np.zeros(max(P, 1), dtype=np.uint8)
    lib().kco_digest(len(keep), _ptr(ptrs), _ptr(nbytes), page_bytes, _ptr(h), _ptr(z), _ptr(pf))
    return h[:P], z[:P], pf


def dedup(regions, page_bytes: int, hashes, zero):
    """Byte-verified page dedup.  Returns dict(off, alloc, blob, canon, n_blobs)."""
    ptrs, nbytes, keep = _region_table(regions)
    P = int(page_first(nbytes, page_bytes)[-1])
    hashes = np.ascontiguousarray(hashes, dtype=np.uint64)
    zero = np.ascontiguousarray(zero, dtype=np.uint8)
    assert hashes.size == P and zero.size == P
    off = np.zeros(max(P, 1), dtype=np.uint64)
    alloc = np.zeros(max(P, 1), dtype=np.uint32)
    blob = np.zeros(max(P, 1), dtype=np.uint32)
    canon = np.zeros(max(P, 1), dtype=np.uint64)
    nb = np.zeros(1, dtype=np.uint64)
    rc = lib().kco_dedup(len(keep), _ptr(ptrs), _ptr(nbytes), page_bytes,
                         _ptr(hashes if P else np.zeros(1, np.uint64)),
                         _ptr(zero if P else np.zeros(1, np.uint8)),
                         _ptr(off), _ptr(alloc), _ptr(blob), _ptr(canon), _ptr(nb))
    if rc != 0:
        raise MemoryError("oracle dedup out of memory")
    return dict(off=off[:P], alloc=alloc[:P], blob=blob[:P], canon=canon[:P], n_blobs=int(nb[0]))


def pack(regions, page_bytes: int, table) -> np.ndarray:
    """Arena of n_blobs * page_bytes bytes: canonical pages in blob order, zero-filled slots."""
    ptrs, nbytes, keep = _region_table(regions)
    arena = np.zeros(max(table["n_blobs"] * page_bytes, 1), dtype=np.uint8)
    lib().kco_pack(len(keep), _ptr(ptrs), _ptr(nbytes), page_bytes,
                   _ptr(table["off"]), _ptr(table["alloc"]), _ptr(table["blob"]),
                   _ptr(table["canon"]), _ptr(arena))
    return arena[: table["n_blobs"] * page_bytes]


def restore(targets, page_bytes: int, table, arena) -> None:
    """Write every page of ``table`` into the uint8 arrays ``targets`` (in place)."""
    for t in targets:
        assert t.dtype == np.uint8 and t.flags.c_contiguous
    ptrs = np.array([_ptr(t) for t in targets], dtype=np.uint64)
    nbytes = np.array([t.size for t in targets], dtype=np.uint64)
    P = table["off"].size
    arena = np.ascontiguousarray(arena, dtype=np.uint8)
    a = arena if arena.size else np.zeros(1, np.uint8)
    lib().kco_restore(len(targets), _ptr(ptrs), _ptr(nbytes), page_bytes, P,
                      _ptr(np.ascontiguousarray(table["off"], dtype=np.uint64)),
                      _ptr(np.ascontiguousarray(table["alloc"], dtype=np.uint32)),
                      _ptr(np.ascontiguousarray(table["blob"], dtype=np.uint32)), _ptr(a))


def census(regions, bases, win_lo: int, win_hi: int, cap: int | None = None, sizes=None):
    """Embedded-pointer census.  Returns (hits structured array, n_inside, n_outside, rc).

    ``sizes`` (optional) gives each region's full size as a target range when
    the image passed in ``regions`` is only its first bytes (possibly none):
    only the image is scanned.
    """
    ptrs, scan, keep = _region_table(regions)
    bases = np.ascontiguousarray(bases, dtype=np.uint64)
    nbytes = scan if sizes is None else np.ascontiguousarray(sizes, dtype=np.uint64)
    assert np.all(scan <= nbytes)
    if cap is None:
        cap = int(sum(int(b) // 8 for b in scan))
    hits = np.zeros(max(cap, 1), dtype=HIT_DTYPE)
    nin = np.zeros(1, dtype=np.uint64)
    nout = np.zeros(1, dtype=np.uint64)
    rc = lib().kco_census(len(keep), _ptr(ptrs), _ptr(bases), _ptr(nbytes), _ptr(scan), win_lo,
                          win_hi, _ptr(hits), cap, _ptr(nin), _ptr(nout))
    if rc == -1:
        raise MemoryError("oracle census out of memory")
    total = int(nin[0] + nout[0])
    return hits[: min(total, cap)], int(nin[0]), int(nout[0]), rc


def compare(got: np.ndarray, want: np.ndarray, dtype_code: int, atol: float = 0.0,
            rtol: float = 0.0) -> np.ndarray:
    """Per-dtype FP64 comparison; returns one CMP_DTYPE record."""
    g = np.ascontiguousarray(got).view(np.uint8).reshape(-1)
    w = np.ascontiguousarray(want).view(np.uint8).reshape(-1)
    assert g.size == w.size
    esize = {DT_U8: 1, DT_RAW: 1, DT_I32: 4, DT_F16: 2, DT_BF16: 2, DT_F32: 4}[dtype_code]
    assert g.size % esize == 0
    out = np.zeros(1, dtype=CMP_DTYPE)
    gg = g if g.size else np.zeros(1, np.uint8)
    ww = w if w.size else np.zeros(1, np.uint8)
    lib().kco_compare(_ptr(gg), _ptr(ww), dtype_code, g.size // esize, atol, rtol, _ptr(out))
    return out[0]
