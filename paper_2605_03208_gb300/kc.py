"""Python binding of the C ABI in ``include/kc.h`` (argument marshalling only).

Every operation runs in the CUDA kernels of ``libkc.so``; this module only
turns torch tensors / integers into the pointers and sizes the C functions
take.  There is no CPU fallback: if the library is missing, loading fails.
"""
from __future__ import annotations

import ctypes
import operator
import os

import numpy as np

from . import build as _build

OK, EINVAL, EOVERLAP, ENOMEM, ETRUNC, ECUDA, ETIMEOUT, EBUF = range(8)
U8, I32, F16, BF16, F32, RAW = range(6)
BUF_LOST = 0x1
PAGE_DATA, PAGE_ZERO, PAGE_LOST = 0, 1, 2
BLOB_ZERO = 0xFFFFFFFF
BLOB_LOST = 0xFFFFFFFE

PAGE_DTYPE = np.dtype([("va_offset", "<u8"), ("alloc_id", "<u4"), ("blob", "<u4")])
HIT_DTYPE = np.dtype([("src_offset", "<u8"), ("value", "<u8"), ("src_alloc", "<u4"),
                      ("target", "<i4")])
CMP_DTYPE = np.dtype([("mismatches", "<u8"), ("first", "<i8"), ("max_abs", "<f8"),
                      ("max_rel", "<f8"), ("nan_got", "<u8"), ("nan_want", "<u8"),
                      ("nan_mismatch", "<u8"), ("status", "<i4"), ("reserved", "<u4")])
ESIZE = {U8: 1, RAW: 1, I32: 4, F16: 2, BF16: 2, F32: 4}

# Names declared in include/kc.h (the ABI surface).
EXPORTS = ["kc_version", "kc_launch_count", "kc_status_name", "kc_last_error", "kc_create", "kc_destroy", "kc_sync",
           "kc_buf_status", "kc_set_digest_shape", "kc_debug_stall_census", "kc_set_trace_events", "kc_get_digest_shape", "kc_page_count",
           "kc_digest", "kc_census", "kc_scan", "kc_dedup", "kc_restore", "kc_compare",
           "kc_census_static", "kc_batch_run", "kc_poll_flags", "kc_va_reserve", "kc_va_lease_bytes",
           "kc_va_release"]


class KcBuf(ctypes.Structure):
    _fields_ = [("base_va", ctypes.c_uint64), ("bytes", ctypes.c_uint64),
                ("dtype", ctypes.c_int32), ("flags", ctypes.c_int32)]


JOB_DIGEST, JOB_COMPARE, JOB_INIT = 0x10, 0x20, 0x40
WORK_DIGEST, WORK_COMPARE, WORK_FUSED = 0, 1, 2
BATCH_ITEM_BYTES = 65536


class KcJob(ctypes.Structure):
    _fields_ = [("got_va", ctypes.c_uint64), ("want_va", ctypes.c_uint64), ("bytes", ctypes.c_uint64),
                ("dtype", ctypes.c_int32), ("flags", ctypes.c_int32), ("d_hash", ctypes.c_uint64),
                ("d_zero", ctypes.c_uint64), ("d_cmp", ctypes.c_uint64), ("d_done", ctypes.c_uint64),
                ("d_cmp_copy", ctypes.c_uint64)]


class KcWork(ctypes.Structure):
    _fields_ = [("job", ctypes.c_uint32), ("kind", ctypes.c_uint32), ("first", ctypes.c_uint64),
                ("count", ctypes.c_uint64)]


class KcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status_name(status)}: {msg}")
        self.status = status


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libkc.so (optionally building it first).  Raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library {path} is not built; run __graft_entry__.build()")
        _build.build()
    L = ctypes.CDLL(path)
    vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    st = ctypes.c_int
    L.kc_version.restype = i32
    L.kc_launch_count.restype = u64
    L.kc_status_name.restype = ctypes.c_char_p
    L.kc_status_name.argtypes = [i32]
    L.kc_last_error.restype = ctypes.c_char_p
    L.kc_last_error.argtypes = [vp]
    L.kc_create.restype = st
    L.kc_create.argtypes = [ctypes.POINTER(vp), i32]
    L.kc_destroy.restype = None
    L.kc_destroy.argtypes = [vp]
    L.kc_sync.restype = st
    L.kc_sync.argtypes = [vp, vp]
    L.kc_buf_status.restype = i32
    L.kc_buf_status.argtypes = [vp, i32]
    L.kc_set_digest_shape.restype = st
    L.kc_set_digest_shape.argtypes = [vp, i32, i32, i32, i32]
    L.kc_debug_stall_census.restype = st
    L.kc_debug_stall_census.argtypes = [vp, u32]
    L.kc_set_trace_events.restype = st
    L.kc_set_trace_events.argtypes = [vp, vp, vp]
    L.kc_get_digest_shape.restype = st
    L.kc_get_digest_shape.argtypes = [vp, u32, u64] + [ctypes.POINTER(i32)] * 5
    L.kc_page_count.restype = u64
    L.kc_page_count.argtypes = [ctypes.POINTER(KcBuf), i32, u32]
    B = ctypes.POINTER(KcBuf)
    L.kc_digest.restype = st
    L.kc_digest.argtypes = [vp, B, i32, u32, vp, vp, vp, vp]
    L.kc_census.restype = st
    L.kc_census.argtypes = [vp, B, i32, u64, u64, vp, u64, vp, vp]
    L.kc_batch_run.restype = st
    L.kc_batch_run.argtypes = [vp, ctypes.POINTER(KcJob), i32, u32, ctypes.c_double, ctypes.c_double,
                               ctypes.POINTER(KcWork), i32, vp]
    L.kc_poll_flags.restype = i32
    L.kc_poll_flags.argtypes = [vp, i32, vp]
    L.kc_census_static.restype = st
    L.kc_census_static.argtypes = [B, i32, u64, u64, vp, u64, vp, vp]
    L.kc_va_reserve.restype = st
    L.kc_va_reserve.argtypes = [i32, B, i32, ctypes.POINTER(vp)]
    L.kc_va_lease_bytes.restype = u64
    L.kc_va_lease_bytes.argtypes = [vp]
    L.kc_va_release.restype = None
    L.kc_va_release.argtypes = [vp]
    L.kc_scan.restype = st
    L.kc_scan.argtypes = [vp, B, i32, u32, vp, vp, vp, u64, u64, vp, u64, vp, vp]
    L.kc_dedup.restype = st
    L.kc_dedup.argtypes = [vp, B, i32, u32, vp, vp, vp, vp, u64, vp, vp]
    L.kc_restore.restype = st
    L.kc_restore.argtypes = [vp, B, i32, u32, vp, u64, vp, u64, vp]
    L.kc_compare.restype = st
    L.kc_compare.argtypes = [vp, B, B, i32, ctypes.c_double, ctypes.c_double, vp, vp]
    _lib = L
    return L


def status_name(s: int) -> str:
    try:
        return load().kc_status_name(s).decode()
    except Exception:
        return f"status {s}"


def bufs(items) -> ctypes.Array:
    """Array of kc_buf from (base_va, bytes[, dtype[, flags]]) tuples or torch tensors."""
    arr = (KcBuf * len(items))()
    for i, it in enumerate(items):
        if hasattr(it, "data_ptr"):
            arr[i] = KcBuf(it.data_ptr(), it.numel() * it.element_size(), RAW, 0)
        else:
            t = tuple(it) + (RAW, 0)[len(it) - 2:]
            arr[i] = KcBuf(int(t[0]), int(t[1]), int(t[2]), int(t[3]))
    return arr


def _ptr(x) -> int:
    """Address of a tensor (data_ptr), or an integer address (Python or numpy
    integer) as given; None is 0."""
    if x is None:
        return 0
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return operator.index(x)


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


class Context:
    """One kc_ctx on one device; serves one stream at a time."""

    def __init__(self, device: int = 0):
        self.lib = load()
        h = ctypes.c_void_p()
        s = self.lib.kc_create(ctypes.byref(h), device)
        if s != OK:
            raise KcError(s, f"kc_create(device={device}) failed")
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            self.lib.kc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, s, allow=(OK, EBUF)):
        if s not in allow:
            raise KcError(s, self.lib.kc_last_error(self.h).decode())
        return s

    def last_error(self) -> str:
        return self.lib.kc_last_error(self.h).decode()

    def sync(self, stream=None) -> int:
        """kc_sync: wait, then return the device-side status (raises on none)."""
        return self.lib.kc_sync(self.h, _stream(stream))

    def buf_status(self, i: int) -> int:
        return self.lib.kc_buf_status(self.h, i)

    def set_digest_shape(self, warps=0, stages=0, chunk=0, lanes=0):
        return self._check(self.lib.kc_set_digest_shape(self.h, warps, stages, chunk, lanes), (OK,))

    def debug_stall_census(self, spin_limit: int):
        """kc_debug_stall_census: the next scan's census leaves its first
        chunk unpublished and bounds each look-back wait at spin_limit polls
        (a test of the bounded wait; kc_sync then reports KC_ETIMEOUT)."""
        return self._check(self.lib.kc_debug_stall_census(self.h, spin_limit), (OK,))

    def set_trace_events(self, start=None, stop=None):
        """Record torch.cuda.Event objects around the main kernel of later calls.

        torch creates the underlying cudaEvent_t on first record; a never
        recorded event is recorded once here so that it exists."""
        for e in (start, stop):
            if e is not None and not e.cuda_event:
                e.record()
        a = start.cuda_event if start is not None else None
        b = stop.cuda_event if stop is not None else None
        return self._check(self.lib.kc_set_trace_events(self.h, a, b), (OK,))

    def digest_shape(self, page_bytes: int, npages: int):
        v = [ctypes.c_int() for _ in range(5)]
        self._check(self.lib.kc_get_digest_shape(self.h, page_bytes, npages,
                                                 *[ctypes.byref(x) for x in v]), (OK,))
        return dict(warps=v[0].value, stages=v[1].value, chunk=v[2].value, ctas=v[3].value,
                    lanes=v[4].value)

    def digest(self, regions, page_bytes, hash_out, zero_out, page_first_out=None, stream=None,
               allow=(OK, EBUF)):
        b = regions if isinstance(regions, ctypes.Array) else bufs(regions)
        return self._check(self.lib.kc_digest(self.h, b, len(b), page_bytes, _ptr(hash_out),
                                              _ptr(zero_out), _ptr(page_first_out),
                                              _stream(stream)), allow)

    def scan(self, regions, page_bytes, hash_out, zero_out, page_first_out, win_lo, win_hi,
             hits_out, cap, counts_out, stream=None, allow=(OK, EBUF)):
        b = regions if isinstance(regions, ctypes.Array) else bufs(regions)
        return self._check(self.lib.kc_scan(self.h, b, len(b), page_bytes, _ptr(hash_out),
                                            _ptr(zero_out), _ptr(page_first_out), win_lo, win_hi,
                                            _ptr(hits_out), cap, _ptr(counts_out),
                                            _stream(stream)), allow)

    def census(self, regions, win_lo, win_hi, hits_out, cap, counts_out, stream=None,
               allow=(OK, EBUF)):
        b = regions if isinstance(regions, ctypes.Array) else bufs(regions)
        return self._check(self.lib.kc_census(self.h, b, len(b), win_lo, win_hi, _ptr(hits_out),
                                              cap, _ptr(counts_out), _stream(stream)), allow)

    def dedup(self, regions, page_bytes, hash_in, zero_in, table_out, arena_out, arena_cap,
              n_blobs_out, stream=None, allow=(OK, EBUF)):
        b = regions if isinstance(regions, ctypes.Array) else bufs(regions)
        return self._check(self.lib.kc_dedup(self.h, b, len(b), page_bytes, _ptr(hash_in),
                                             _ptr(zero_in), _ptr(table_out), _ptr(arena_out),
                                             arena_cap, _ptr(n_blobs_out), _stream(stream)), allow)

    def restore(self, regions, page_bytes, table, n_pages, arena, arena_bytes, stream=None,
                allow=(OK, EBUF)):
        b = regions if isinstance(regions, ctypes.Array) else bufs(regions)
        return self._check(self.lib.kc_restore(self.h, b, len(b), page_bytes, _ptr(table),
                                               n_pages, _ptr(arena), arena_bytes,
                                               _stream(stream)), allow)

    def batch_run(self, job_array, page_bytes, atol=0.0, rtol=0.0, work_array=None, stream=None,
                  allow=(OK, EBUF), njobs=None, nwork=None):
        """kc_batch_run.  job_array / work_array: ctypes arrays (or lists of
        dicts / tuples, converted); njobs / nwork use a prefix of a larger
        preallocated array."""
        j = job_array if isinstance(job_array, ctypes.Array) else jobs(job_array)
        w = work_array
        if w is not None and not isinstance(w, ctypes.Array):
            w = work(w)
        nj = len(j) if njobs is None else njobs
        nw = (0 if w is None else len(w)) if nwork is None else nwork
        return self._check(self.lib.kc_batch_run(self.h, j, nj, page_bytes, float(atol), float(rtol), w, nw,
                                                 _stream(stream)), allow)

    def compare(self, got, want, atol, rtol, out, stream=None, allow=(OK, EBUF)):
        g = got if isinstance(got, ctypes.Array) else bufs(got)
        w = want if isinstance(want, ctypes.Array) else bufs(want)
        assert len(g) == len(w)
        return self._check(self.lib.kc_compare(self.h, g, w, len(g), float(atol), float(rtol),
                                               _ptr(out), _stream(stream)), allow)


def jobs(items) -> ctypes.Array:
    """Array of kc_job from dicts with keys got, want, bytes, dtype, flags,
    hash, zero, cmp, done, cmp_copy (tensors or integer addresses; absent = 0)."""
    arr = (KcJob * len(items))()
    for i, it in enumerate(items):
        arr[i] = KcJob(_ptr(it.get("got")), _ptr(it.get("want")), int(it["bytes"]), int(it.get("dtype", RAW)),
                       int(it["flags"]), _ptr(it.get("hash")), _ptr(it.get("zero")), _ptr(it.get("cmp")),
                       _ptr(it.get("done")), _ptr(it.get("cmp_copy")))
    return arr


def work(items) -> ctypes.Array:
    """Array of kc_work from (job, kind, first, count) tuples."""
    arr = (KcWork * len(items))()
    for i, (j, k, f, c) in enumerate(items):
        arr[i] = KcWork(int(j), int(k), int(f), int(c))
    return arr


class FlagPoller:
    """Completion flags in pinned host memory for kc_job.d_done, read with
    acquire ordering through kc_poll_flags."""

    def __init__(self, n: int):
        import torch
        self.flags = torch.zeros(n, dtype=torch.int32, pin_memory=True)
        self.view = self.flags.numpy()
        self.idx = (ctypes.c_int32 * n)()
        self.n = n
        self.lib = load()

    def address(self, i: int) -> int:
        return self.flags.data_ptr() + 4 * i

    def clear(self, i: int) -> None:
        self.view[i] = 0

    def poll(self) -> list:
        k = self.lib.kc_poll_flags(self.flags.data_ptr(), self.n, self.idx)
        return list(self.idx[:k])


def census_static(regions, win_lo, win_hi, hits_out, cap, counts_out, stream=None) -> int:
    """kc_census_static: the census without a context and without allocating
    (scratch in a static device array; see include/kc.h).  regions None: the
    one-time set-up of the current device only.  Returns the status."""
    if regions is None:
        return int(load().kc_census_static(None, 0, 0, 0, None, 0, None, _stream(stream)))
    b = regions if isinstance(regions, ctypes.Array) else bufs(regions)
    return int(load().kc_census_static(b, len(b), win_lo, win_hi, _ptr(hits_out), cap,
                                       _ptr(counts_out), _stream(stream)))


class VaLease:
    """Device memory mapped at a snapshot's captured VAs (kc_va_reserve);
    release() (or garbage collection) unmaps it."""

    def __init__(self, handle):
        self.h = handle
        self.lib = load()

    @property
    def bytes(self) -> int:
        return int(self.lib.kc_va_lease_bytes(self.h)) if self.h else 0

    def release(self):
        if getattr(self, "h", None):
            self.lib.kc_va_release(self.h)
            self.h = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


def va_reserve(device: int, regions) -> "VaLease":
    """kc_va_reserve: map device memory at exactly the regions' VAs (a list
    of (base_va, bytes) or a kc_buf array).  Raises KcError with the status
    (KC_EOVERLAP when a range is already in use in this process)."""
    b = regions if isinstance(regions, ctypes.Array) else bufs(regions)
    h = ctypes.c_void_p()
    s = int(load().kc_va_reserve(device, b, len(b), ctypes.byref(h)))
    if s != OK:
        raise KcError(s, "exact-VA reservation failed")
    return VaLease(h)


def launch_count() -> int:
    """Kernels launched by libkc.so in this process so far."""
    return int(load().kc_launch_count())


def page_count(regions, page_bytes: int) -> int:
    b = regions if isinstance(regions, ctypes.Array) else bufs(regions)
    return int(load().kc_page_count(b, len(b), page_bytes))
