"""The CUDA library builds for sm_103a, loads without a GPU and exports every
entry point declared in include/kc.h (no compute call is made here)."""
import os
import re
import subprocess

from paper_2605_03208_gb300 import build, kc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "kc.h")).read()
    return sorted(set(re.findall(r"KC_API\s+[\w\s\*]*?\b(kc_\w+)\s*\(", src)))


def test_header_declares_the_binding_surface():
    assert declared_symbols() == sorted(kc.EXPORTS)


def test_library_loads_and_exports_every_declared_symbol():
    path = build.build()
    lib = kc.load()
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert lib.kc_version() == 1
    assert kc.status_name(kc.ETRUNC) == "KC_ETRUNC"
    # nothing but the kc_* ABI is exported
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = sorted(l.split()[-1] for l in out.splitlines() if l.split()[-1].startswith("kc_"))
    assert exported == declared_symbols()


def test_page_count_is_host_only():
    b = kc.bufs([(0x1000, 4096 * 3 + 1), (0x100000, 5)])
    assert kc.page_count(b, 4096) == 5
    assert kc.page_count(b, 65536) == 2


def test_struct_layouts_match_the_header(tmp_path):
    """Sizes and field offsets of the C structs, compiled from include/kc.h
    by the host C compiler, equal the binding's ctypes layouts."""
    import ctypes
    import numpy as np
    src = tmp_path / "layout.c"
    src.write_text('''#include <stdio.h>
#include <stddef.h>
#include "kc.h"
#define F(T, m) printf(#T "." #m " %zu\\n", offsetof(T, m))
int main(void) {
    printf("kc_buf %zu\\nkc_page %zu\\nkc_hit %zu\\nkc_cmp_result %zu\\nkc_job %zu\\nkc_work %zu\\n",
           sizeof(kc_buf), sizeof(kc_page), sizeof(kc_hit), sizeof(kc_cmp_result), sizeof(kc_job),
           sizeof(kc_work));
    F(kc_job, got_va); F(kc_job, want_va); F(kc_job, bytes); F(kc_job, dtype); F(kc_job, flags);
    F(kc_job, d_hash); F(kc_job, d_zero); F(kc_job, d_cmp); F(kc_job, d_done); F(kc_job, d_cmp_copy);
    F(kc_work, job); F(kc_work, kind); F(kc_work, first); F(kc_work, count);
    return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    got = {k: int(v) for k, v in got.items()}
    assert got["kc_buf"] == ctypes.sizeof(kc.KcBuf)
    assert got["kc_page"] == kc.PAGE_DTYPE.itemsize
    assert got["kc_hit"] == kc.HIT_DTYPE.itemsize
    assert got["kc_cmp_result"] == kc.CMP_DTYPE.itemsize == 64
    assert got["kc_job"] == ctypes.sizeof(kc.KcJob) == 72
    assert got["kc_work"] == ctypes.sizeof(kc.KcWork)
    for cls, cname in ((kc.KcJob, "kc_job"), (kc.KcWork, "kc_work")):
        for name, _ in cls._fields_:
            assert got[f"{cname}.{name}"] == getattr(cls, name).offset, (cname, name)


def test_poll_flags_host_helper():
    import ctypes
    import numpy as np
    lib = kc.load()
    f = np.array([0, 1, 0, 7, 1], dtype=np.uint32)
    idx = (ctypes.c_int32 * 5)()
    assert lib.kc_poll_flags(f.ctypes.data, 5, idx) == 3 and list(idx[:3]) == [1, 3, 4]
    assert lib.kc_poll_flags(f.ctypes.data, 0, idx) == 0
    assert lib.kc_poll_flags(None, 5, idx) == -1 and lib.kc_poll_flags(f.ctypes.data, -1, idx) == -1


def test_plain_c_client_builds_links_and_gets_errors_not_crashes(tmp_path):
    """A C program that includes only include/kc.h and links libkc.so: the
    host-only calls work, a context on a device that does not exist is
    refused with an error (and no handle), and a call without a context is
    refused before any device work."""
    path = build.build()
    src = tmp_path / "client.c"
    src.write_text('''#include <stdio.h>
#include <string.h>
#include "kc.h"
int main(void) {
    kc_buf b[2] = {{0x1000, 4096 * 3 + 1, KC_RAW, 0}, {0x100000, 5, KC_RAW, 0}};
    if (kc_version() != 1) return 1;
    if (strcmp(kc_status_name(KC_ETRUNC), "KC_ETRUNC") != 0) return 2;
    if (kc_page_count(b, 2, 4096) != 5) return 3;
    kc_ctx *c = NULL;
    kc_status s = kc_create(&c, 9999);
    if (s == KC_OK || c != NULL) return 4;
    if (kc_digest(NULL, b, 2, 4096, NULL, NULL, NULL, NULL) != KC_EINVAL) return 5;
    if (kc_compare(NULL, b, b, 1, 0.0, 0.0, NULL, NULL) != KC_EINVAL) return 6;
    printf("ok %s\\n", kc_status_name(s));
    return 0;
}
''')
    exe = tmp_path / "client"
    libdir = os.path.dirname(path)
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    "-L", libdir, "-l:" + os.path.basename(path), "-Wl,-rpath," + libdir], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.startswith("ok KC_E")


def test_census_static_argument_checks_are_host_only():
    """kc_census_static validates on the host before touching a device: the
    region-count and chunk limits, empty or misaligned regions and
    overlapping ranges are refused without any CUDA call (these addresses
    are never dereferenced)."""
    lib = kc.load()
    counts = 0x7000_0000_0000     # never written: every call below is refused first
    cases = [
        ([(0x10000 + 4096 * i, 4096) for i in range(1025)], kc.EINVAL),           # 1025 regions
        ([(0x10_0000_0000, 4 * 2**30 + 65536)], kc.EINVAL),                        # 65537 chunks
        ([(0x10_0000_0000, 2**32), (0x20_0000_0000, 1)], kc.EINVAL),              # 65537 chunks over two
        ([(0x10000, 0)], kc.EINVAL),                                               # empty region
        ([(0x10008, 64)], kc.EINVAL),                                              # not 16-byte aligned
        ([(0x10000, 8192), (0x11000, 64)], kc.EOVERLAP),                          # overlapping ranges
    ]
    for regions, want in cases:
        b = kc.bufs(regions)
        assert lib.kc_census_static(b, len(b), 0, 0, None, 0, counts, 0) == want, regions
    b = kc.bufs([(0x10000, 64)])
    assert lib.kc_census_static(b, 1, 0, 0, None, 0, None, 0) == kc.EINVAL       # no counts output
    assert lib.kc_census_static(b, 1, 0, 0, None, 5, counts, 0) == kc.EINVAL     # cap without hits
    assert lib.kc_census_static(None, 1, 0, 0, None, 0, counts, 0) == kc.EINVAL  # no regions, n = 1


def test_va_reserve_argument_checks_are_host_only():
    """kc_va_reserve refuses bad arguments before touching a device."""
    import ctypes
    lib = kc.load()
    h = ctypes.c_void_p()
    b = kc.bufs([(0x7f0000000000, 4096)])
    assert lib.kc_va_reserve(0, b, 1, None) == kc.EINVAL                       # no lease output
    assert lib.kc_va_reserve(0, None, 1, ctypes.byref(h)) == kc.EINVAL         # no regions
    assert lib.kc_va_reserve(0, b, 0, ctypes.byref(h)) == kc.EINVAL            # n = 0
    assert lib.kc_va_reserve(0, kc.bufs([(0x7f0000000000, 0)]), 1, ctypes.byref(h)) == kc.EINVAL   # empty
    assert lib.kc_va_reserve(0, kc.bufs([(0, 4096)]), 1, ctypes.byref(h)) == kc.EINVAL             # null base
    assert lib.kc_va_reserve(0, kc.bufs([(2**64 - 4096, 8192)]), 1, ctypes.byref(h)) == kc.EINVAL  # wraps
    assert h.value is None
    assert lib.kc_va_lease_bytes(None) == 0
    lib.kc_va_release(None)                                                   # a no-op
