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
