"""Exact-VA restore into a fresh process (the paper's VA-faithful replay).

A child process captures a snapshot (its regions allocated by PyTorch with
expandable segments, the VMM-based allocator, and filled with data that
embeds pointers to their own VAs) and saves it; a second child -- a new
CUDA context that never saw the snapshot -- maps device memory at the
captured VAs with kc_va_reserve before allocating anything else, loads the
snapshot back at those VAs (snapshot_io.load + kc_restore) and reports what
it finds.  Checked here: every region's bytes are the captured ones at the
captured VA; the digest and the pointer census of the restored image
(kc_scan in the replaying process) equal the CPU oracle's on the captured
bytes at the captured bases, so every embedded pointer again points into
the closure; a second reservation of the same ranges is refused with
KC_EOVERLAP rather than relocated; and, in this process, a range already in
use is refused too.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle
from paper_2605_03208_gb300 import kc
from paper_2605_03208_gb300 import workloads as W
from tests import _gpu as G

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CAPTURE = r'''
import json, sys
import numpy as np
root, snapdir, out = sys.argv[1:4]
sys.path.insert(0, root)
import torch
from paper_2605_03208_gb300 import kc
from paper_2605_03208_gb300 import snapshot_io as SIO
from paper_2605_03208_gb300 import workloads as W
layout = W.tiny_layout(5, n=10, total=6 * W.MiB)
dev = [torch.empty(int(s), dtype=torch.uint8, device="cuda") for s in layout.sizes]
snap = W.tiny_fill(layout, [t.data_ptr() for t in dev], 5, p_ptr=0.3)
for t, r in zip(dev, snap.regions):
    t.copy_(torch.from_numpy(r))
torch.cuda.synchronize()
ctx = kc.Context(0)
SIO.save(ctx, kc.bufs([(t.data_ptr(), t.numel(), kc.RAW, 0) for t in dev]), snap.page_bytes, snapdir)
np.savez(out + ".npz", *snap.regions)
json.dump({"bases": snap.bases, "sizes": [int(x) for x in snap.sizes], "page_bytes": snap.page_bytes,
           "pointers": [list(p) for p in snap.truth["pointers"]]}, open(out + ".json", "w"))
ctx.close()
'''

REPLAY = r'''
import json, sys
import numpy as np
root, snapdir, out = sys.argv[1:4]
sys.path.insert(0, root)
from paper_2605_03208_gb300 import kc
from paper_2605_03208_gb300 import snapshot_io as SIO
from paper_2605_03208_gb300 import workloads as W
m = SIO.read_manifest(snapdir)
regs = [(int(r["base_va"]), int(r["bytes"])) for r in m["regions"]]
lease = kc.va_reserve(0, regs)             # first of all: nothing else may take these VAs
try:
    kc.va_reserve(0, regs)
    second = "granted"
except kc.KcError as e:
    second = e.status
import torch


class View:                                # a device VA range seen as a torch uint8 tensor
    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "|u1", "data": (ptr, False),
                                         "version": 3, "strides": None}


ctx = kc.Context(0)
SIO.load(ctx, snapdir)                     # restores every page at its captured VA
back = [torch.as_tensor(View(p, n), device="cuda").cpu().numpy() for p, n in regs]
np.savez(out + ".npz", *back)
b = kc.bufs([(p, n, int(r["dtype"]), 0) for (p, n), r in zip(regs, m["regions"])])
S = int(m["page_bytes"])
P = kc.page_count(b, S)
win = W.default_window([p for p, _ in regs], [n for _, n in regs])
cap = sum(n // 8 for _, n in regs)
h = torch.empty(P, dtype=torch.int64, device="cuda")
z = torch.empty(P, dtype=torch.uint8, device="cuda")
hits = torch.empty(cap * 24, dtype=torch.uint8, device="cuda")
counts = torch.zeros(2, dtype=torch.int64, device="cuda")
ctx.scan(b, S, h, z, None, win[0], win[1], hits, cap, counts)
st = ctx.sync()
c = counts.cpu().numpy().view(np.uint64)
n = int(c[0] + c[1])
hits.cpu().numpy()[: n * 24].tofile(out + ".hits")
h.cpu().numpy().tofile(out + ".hash")
z.cpu().numpy().tofile(out + ".zero")
json.dump({"second": second, "status": st, "lease_bytes": lease.bytes, "counts": [int(c[0]), int(c[1])]},
          open(out + ".json", "w"))
ctx.close()
lease.release()
'''


def test_restore_at_the_captured_vas_in_a_fresh_process(tmp_path):
    d = str(tmp_path / "snap")
    cap = str(tmp_path / "capture")
    out = str(tmp_path / "replay")
    env = dict(os.environ, PYTORCH_CUDA_ALLOC_CONF="expandable_segments:True")
    r = subprocess.run([sys.executable, "-c", CAPTURE, ROOT, d, cap], capture_output=True, text=True, timeout=600,
                       env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    meta = json.load(open(cap + ".json"))
    regions = [np.load(cap + ".npz")[f"arr_{i}"] for i in range(len(meta["sizes"]))]
    bases, S = meta["bases"], meta["page_bytes"]
    r = subprocess.run([sys.executable, "-c", REPLAY, ROOT, d, out], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.load(open(out + ".json"))
    assert res["second"] == kc.EOVERLAP
    assert res["status"] == kc.OK
    assert res["lease_bytes"] >= sum(meta["sizes"])
    back = np.load(out + ".npz")
    for i, reg in enumerate(regions):
        assert np.array_equal(back[f"arr_{i}"], reg), f"region {i} differs after the restore"
    oh, oz, _ = oracle.digest(regions, S)
    assert np.array_equal(np.fromfile(out + ".hash", dtype=np.uint64), oh)
    assert np.array_equal(np.fromfile(out + ".zero", dtype=np.uint8), oz)
    win = W.default_window(bases, meta["sizes"])
    ohits, nin, nout, rc = oracle.census(regions, bases, *win)
    assert rc == 0 and nin > 0
    assert res["counts"] == [nin, nout]
    got = np.fromfile(out + ".hits", dtype=kc.HIT_DTYPE)
    assert got.tobytes() == ohits.tobytes()
    assert {tuple(p) for p in meta["pointers"]} <= set(G.hits_tuples(got))


def test_reservation_refuses_a_range_in_use_here():
    """In this process the captured VAs are live torch allocations: the
    reservation must fail with KC_EOVERLAP and leave nothing behind."""
    kc.load()
    t = torch.empty(4 * W.MiB, dtype=torch.uint8, device="cuda")
    free0, _ = torch.cuda.mem_get_info()
    with pytest.raises(kc.KcError) as e:
        kc.va_reserve(0, [(t.data_ptr(), t.numel())])
    assert e.value.status == kc.EOVERLAP
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
