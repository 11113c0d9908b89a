"""Seeded synthetic snapshots and output-buffer pairs.

These generators stand in for the captured applications of the paper's
evaluation (llama.cpp, vLLM's fused MoE kernel, ...), whose processes,
weights and snapshots are not available: they reproduce the shapes, sizes,
value distributions and planted structure (zero pages, duplicate pages,
embedded device pointers, perturbed outputs) of those workloads.

This module holds none of the method's arithmetic: no hashing, no dedup, no
pointer classification and no error computation.  It only draws bytes and
records what it planted.  Both the CUDA path and the oracle consume its
output, so the two see identical inputs.

Host generators return numpy arrays.  Regions are described by their sizes
first (``*_layout``), so a caller can allocate device memory, learn the VAs,
and then fill the bytes (``*_fill``): pointer-holding pages must contain the
real VAs of the captured regions.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

KiB = 1024
MiB = 1024 * KiB
GiB = 1024 * MiB

DT_U8, DT_I32, DT_F16, DT_BF16, DT_F32, DT_RAW = 0, 1, 2, 3, 4, 5
DTYPE_NAMES = {DT_U8: "uint8", DT_I32: "int32", DT_F16: "fp16", DT_BF16: "bf16",
               DT_F32: "fp32", DT_RAW: "raw"}
ESIZE = {DT_U8: 1, DT_RAW: 1, DT_I32: 4, DT_F16: 2, DT_BF16: 2, DT_F32: 4}


@dataclass
class Snapshot:
    """A synthetic captured address space: regions at VAs, plus planted truth."""
    name: str
    page_bytes: int
    sizes: list
    bases: list = field(default_factory=list)
    regions: list = field(default_factory=list)   # uint8 numpy arrays
    dtypes: list = field(default_factory=list)
    truth: dict = field(default_factory=dict)

    @property
    def total_bytes(self) -> int:
        return int(sum(self.sizes))


# --------------------------------------------------------------------------
# VA helpers
# --------------------------------------------------------------------------

def fake_bases(sizes, seed: int = 0, start: int = 0x7F00_0000_0000, align: int = 2 * MiB):
    """Disjoint, ascending-by-construction (then shuffled) VAs for host-only use."""
    rng = np.random.default_rng(seed + 7919)
    order = rng.permutation(len(sizes))
    bases = [0] * len(sizes)
    cur = start
    for k in order:
        cur += int(rng.integers(0, 4)) * align          # random gap
        bases[k] = cur
        cur += (int(sizes[k]) + align - 1) // align * align
    return bases


def default_window(bases, sizes):
    """Census window: the captured span rounded out to 2 MiB, plus 1 GiB each side."""
    lo = min(int(b) for b in bases)
    hi = max(int(b) + int(s) for b, s in zip(bases, sizes))
    lo = (lo // (2 * MiB)) * (2 * MiB) - GiB
    hi = (hi + 2 * MiB - 1) // (2 * MiB) * (2 * MiB) + GiB
    return max(lo, 0), hi


def _outside_value(rng, bases, sizes):
    """A VA inside the default window's margins, hence outside every region."""
    lo = min(int(b) for b in bases)
    hi = max(int(b) + int(s) for b, s in zip(bases, sizes))
    wlo, whi = default_window(bases, sizes)
    if rng.random() < 0.5 and lo - wlo >= 16:
        v = int(rng.integers(wlo, lo))
    else:
        v = int(rng.integers(hi, whi))
    return v & ~7


def _inside_value(rng, bases, sizes):
    k = int(rng.integers(0, len(sizes)))
    off = int(rng.integers(0, max(int(sizes[k]) // 8, 1))) * 8
    return int(bases[k]) + off, k


# --------------------------------------------------------------------------
# Tiny mixed snapshot: 16 regions, ~16 MiB, 64 KiB pages
# --------------------------------------------------------------------------

def tiny_layout(seed: int = 0, n: int = 16, total: int = 16 * MiB, lo: int = 4 * KiB,
                hi: int = 4 * MiB, page_bytes: int = 64 * KiB) -> Snapshot:
    """16 regions, sizes log-uniform in [4 KiB, 4 MiB] rescaled to ~16 MiB total."""
    rng = np.random.default_rng(seed)
    raw = np.exp(rng.uniform(math.log(lo), math.log(hi), n))
    raw = raw * (total / raw.sum())
    sizes = [int(min(max(int(x) // 8 * 8, lo), hi)) for x in raw]
    # leave a ragged tail: make sizes non-multiples of the page where possible
    sizes = [s - 8 * int(rng.integers(0, 4)) if s > lo else s for s in sizes]
    return Snapshot("tiny-16x-log-uniform-4KiB-4MiB", page_bytes, sizes,
                    dtypes=[DT_RAW] * n)


def tiny_fill(snap: Snapshot, bases, seed: int = 0, p_zero=0.30, p_copy=0.20, p_ptr=0.10,
              p_outside=0.01) -> Snapshot:
    """Fill the tiny snapshot page by page (zero / copy / pointer / random)."""
    rng = np.random.default_rng(seed + 1)
    S = snap.page_bytes
    snap.bases = [int(b) for b in bases]
    regions = [np.empty(s, dtype=np.uint8) for s in snap.sizes]
    full_nonzero = []          # (region, offset) of earlier non-zero full pages
    truth_zero, truth_copy, truth_ptr = [], [], []
    pid = 0
    for i, s in enumerate(snap.sizes):
        for off in range(0, s, S):
            ln = min(S, s - off)
            u = rng.random()
            page = regions[i][off:off + ln]
            if u < p_zero:
                page[:] = 0
                truth_zero.append(pid)
            elif u < p_zero + p_copy and full_nonzero:
                si, so, spid = full_nonzero[int(rng.integers(0, len(full_nonzero)))]
                page[:] = regions[si][so:so + ln]
                truth_copy.append((pid, spid, ln))
                if ln == S:
                    full_nonzero.append((i, off, pid))
            elif u < p_zero + p_copy + p_ptr:
                nw = ln // 8
                words = np.empty(nw, dtype=np.uint64)
                for w in range(nw):
                    if rng.random() < p_outside:
                        words[w] = _outside_value(rng, snap.bases, snap.sizes)
                        truth_ptr.append((i, off + 8 * w, int(words[w]), -1))
                    else:
                        v, k = _inside_value(rng, snap.bases, snap.sizes)
                        words[w] = v
                        truth_ptr.append((i, off + 8 * w, v, k))
                page[: nw * 8] = words.view(np.uint8)
                page[nw * 8:] = rng.integers(1, 256, ln - nw * 8, dtype=np.uint8)
                if ln == S:
                    full_nonzero.append((i, off, pid))
            else:
                page[:] = rng.integers(0, 256, ln, dtype=np.uint8)
                page[0] |= 1              # never all-zero by chance
                if ln == S:
                    full_nonzero.append((i, off, pid))
            pid += 1
    snap.regions = regions
    snap.truth = dict(zero_pages=truth_zero, copies=truth_copy, pointers=truth_ptr)
    return snap


# --------------------------------------------------------------------------
# llama.cpp-shaped snapshot: 400 regions, 64 KiB pages
# --------------------------------------------------------------------------

def llama_layout(seed: int = 0, variant: str = "full", page_bytes: int = 64 * KiB) -> Snapshot:
    """334 Q4-block weight regions, 64 fp16 KV regions, int32 tokens, pointer table.

    ``variant="full"``: KV 32 layers x {K,V} x 512 tokens x 4096 fp16 (4 MiB
    each) and 128 MiB of weights; ``variant="152MB"``: 128 tokens and 80 MiB
    of weights, about 152 MB in total.
    """
    rng = np.random.default_rng(seed)
    tokens, wtotal = (512, 128 * MiB) if variant == "full" else (128, 80 * MiB)
    nw = 334
    raw = np.exp(rng.uniform(math.log(16 * KiB), math.log(2 * MiB), nw))
    raw = raw * (wtotal / raw.sum())
    wsizes = [max(int(x) // 144 * 144, 144) for x in raw]     # whole 18-byte Q4 blocks
    kv = [tokens * 4096 * 2] * 64
    sizes = wsizes + kv + [8 * 512 * 4] + [64 * 8]
    dtypes = [DT_U8] * nw + [DT_F16] * 64 + [DT_I32] + [DT_RAW]
    return Snapshot(f"llama-shaped-400-regions-{variant}", page_bytes, sizes, dtypes=dtypes)


def llama_fill(snap: Snapshot, bases, seed: int = 0) -> Snapshot:
    rng = np.random.default_rng(seed + 1)
    snap.bases = [int(b) for b in bases]
    regions = []
    nw = 334
    for i, s in enumerate(snap.sizes):
        if i < nw:
            nblk = s // 18
            blk = np.empty((nblk, 18), dtype=np.uint8)
            scale = (rng.standard_normal(nblk) * 0.02).astype(np.float16)
            blk[:, 0:2] = scale.view(np.uint8).reshape(nblk, 2)
            blk[:, 2:] = rng.integers(0, 256, (nblk, 16), dtype=np.uint8)
            r = np.zeros(s, dtype=np.uint8)
            r[: nblk * 18] = blk.reshape(-1)
            regions.append(r)
        elif i < nw + 64:
            kv = rng.standard_normal(s // 2, dtype=np.float32).astype(np.float16)
            regions.append(kv.view(np.uint8))
        elif i == nw + 64:
            regions.append(rng.integers(0, 32000, s // 4, dtype=np.int32).view(np.uint8))
        else:
            targets = rng.choice(nw, 64, replace=False)
            vals = []
            for t in targets:
                t = int(t)
                off = 0 if rng.random() < 0.5 else int(rng.integers(0, snap.sizes[t] // 8)) * 8
                vals.append(snap.bases[t] + off)
            regions.append(np.array(vals, dtype=np.uint64).view(np.uint8))
            snap.truth["pointers"] = [(i, 8 * w, v, int(t)) for w, (v, t) in
                                      enumerate(zip(vals, targets))]
    snap.regions = regions
    return snap


# --------------------------------------------------------------------------
# Output-buffer pairs for the comparison
# --------------------------------------------------------------------------

@dataclass
class Pair:
    got: np.ndarray
    want: np.ndarray
    dtype: int
    truth: dict = field(default_factory=dict)


def _nudge(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Where the perturbed value rounded back onto the original, step one ulp away."""
    same = (y == x) & np.isfinite(x)
    if same.any():
        y = y.copy()
        y[same] = np.nextafter(x[same], np.array(np.inf, dtype=x.dtype))
    return y


def _perturb_float(rng, want: np.ndarray, frac: float, rel: float):
    n = want.size
    k = max(1, int(round(n * frac)))
    idx = np.sort(rng.choice(n, k, replace=False))
    got = want.copy()
    sign = np.where(rng.random(k) < 0.5, -1.0, 1.0)
    y = (want[idx].astype(np.float64) * (1.0 + sign * rel)).astype(want.dtype)
    got[idx] = _nudge(want[idx], y)
    return got, idx


def tiny_pairs(seed: int = 0, n: int = 1 << 20):
    """Four fp32 pairs of 1M elements, want ~ N(0, 1).

    0: identical; 1: 1% of elements times (1 +- 1e-6); 2: NaN at 0.1% of the
    positions in both, plus 10 NaN-vs-number positions; 3: both perturbations.
    """
    rng = np.random.default_rng(seed + 101)
    pairs = []
    for kind in range(4):
        want = rng.standard_normal(n, dtype=np.float32)
        got = want.copy()
        mism = np.zeros(0, dtype=np.int64)
        nan_both = np.zeros(0, dtype=np.int64)
        nan_one = np.zeros(0, dtype=np.int64)
        if kind in (1, 3):
            got, mism = _perturb_float(rng, want, 0.01, 1e-6)
        if kind in (2, 3):
            nan_both = np.sort(rng.choice(n, n // 1000, replace=False))
            want[nan_both] = np.nan
            got[nan_both] = np.nan
            free = np.setdiff1d(np.arange(n), np.concatenate([nan_both, mism]))
            nan_one = np.sort(rng.choice(free, 10, replace=False))
            got[nan_one[:5]] = np.nan                 # NaN in got only
            want[nan_one[5:]] = np.nan                # NaN in want only
        pairs.append(Pair(got, want, DT_F32, dict(perturbed=mism, nan_both=nan_both,
                                                  nan_one=nan_one)))
    return pairs


def llama_pairs(seed: int = 0):
    """fp32 logits [8, 32000] ~ N(0, 3): one pair with 0.1% elements times
    (1 +- 1e-5), and one identical pair."""
    rng = np.random.default_rng(seed + 202)
    want = (rng.standard_normal(8 * 32000, dtype=np.float32) * np.float32(3.0))
    got, idx = _perturb_float(rng, want, 0.001, 1e-5)
    want2 = (rng.standard_normal(8 * 32000, dtype=np.float32) * np.float32(3.0))
    return [Pair(got, want, DT_F32, dict(perturbed=idx)),
            Pair(want2.copy(), want2, DT_F32, dict(perturbed=np.zeros(0, np.int64)))]


def mixed_pairs(seed: int = 0, n_pairs: int = 10, max_elems: int = 50_000):
    """Small pairs of every dtype with special values, for edge-case checks."""
    rng = np.random.default_rng(seed + 303)
    out = []
    for k in range(n_pairs):
        dt = [DT_F32, DT_F16, DT_BF16, DT_I32, DT_U8][k % 5]
        n = int(rng.integers(1, max_elems))
        if dt == DT_F32:
            want = rng.standard_normal(n, dtype=np.float32)
        elif dt == DT_F16:
            want = rng.standard_normal(n, dtype=np.float32).astype(np.float16)
        elif dt == DT_BF16:
            f = rng.standard_normal(n, dtype=np.float32)
            want = (f.view(np.uint32) >> 16).astype(np.uint16)   # truncated bf16 bits
        elif dt == DT_I32:
            want = rng.integers(-2**31, 2**31, n, dtype=np.int64).astype(np.int32)
        else:
            want = rng.integers(0, 256, n, dtype=np.uint8)
        got = want.copy()
        m = int(rng.integers(0, 8))
        idx = np.sort(rng.choice(n, min(m, n), replace=False))
        if dt in (DT_F32, DT_F16):
            got[idx] = _nudge(want[idx], (want[idx].astype(np.float64) * 1.01).astype(want.dtype))
        elif dt == DT_BF16:
            got[idx] = want[idx] ^ np.uint16(1)        # one-ulp flip of the bit pattern
        elif dt == DT_I32:
            got[idx] = want[idx] ^ np.int32(1)
        else:
            got[idx] = want[idx] ^ np.uint8(1)
        out.append(Pair(got, want, dt, dict(perturbed=idx)))
    return out


# --------------------------------------------------------------------------
# MoE weight pool: 64 experts x 24 layers x 20 MiB of bf16 in one region
# --------------------------------------------------------------------------

MOE_EXPERTS, MOE_LAYERS, MOE_EXPERT_BYTES = 64, 24, 20 * MiB


def moe_snapshot(seed: int = 0, experts: int = MOE_EXPERTS, layers: int = MOE_LAYERS,
                 expert_bytes: int = MOE_EXPERT_BYTES, dup_frac: float = 0.02,
                 page_bytes: int = 2 * MiB, device: str = "cuda"):
    """Generate the pool on the device with torch's seeded generator.

    Region 0: the pool, experts x layers x expert_bytes of bf16 ~ N(0, 0.02)
    with no exact zeros; dup_frac of its pages are then overwritten with
    exact copies of other (never overwritten) pages.  Region 1: the int64
    indirection array of every expert's base VA.  Returns (Snapshot without
    host regions, [pool, ptrs] device tensors, truth).
    """
    import torch
    n_exp = experts * layers
    pool_bytes = n_exp * expert_bytes
    pool = torch.empty(pool_bytes, dtype=torch.uint8, device=device)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    view = pool.view(torch.bfloat16)
    step = 256 * MiB // 2
    tiny = torch.tensor(2.0 ** -120, dtype=torch.bfloat16, device=device)
    for s in range(0, view.numel(), step):
        x = torch.randn(min(step, view.numel() - s), generator=g, device=device) * 0.02
        x = x.to(torch.bfloat16)
        x = torch.where(x == 0, tiny, x)
        view[s:s + x.numel()] = x
        del x
    npages = pool_bytes // page_bytes
    rng = np.random.default_rng(seed + 404)
    ndup = int(round(npages * dup_frac))
    perm = rng.permutation(npages)
    dst = np.sort(perm[:ndup])
    src = rng.choice(perm[ndup:], ndup, replace=True)
    pv = pool.view(npages, page_bytes)
    for d, s_ in zip(dst.tolist(), src.tolist()):
        pv[d].copy_(pv[s_])
    base = pool.data_ptr()
    vals = np.array([base + e * expert_bytes for e in range(n_exp)], dtype=np.uint64)
    ptrs = torch.from_numpy(vals.view(np.int64).copy()).to(device)
    torch.cuda.synchronize()
    snap = Snapshot(f"moe-pool-{experts}x{layers}x{expert_bytes // MiB}MiB", page_bytes,
                    [pool_bytes, ptrs.numel() * 8], [base, ptrs.data_ptr()], [],
                    [DT_BF16, DT_RAW])
    snap.truth = dict(dup_dst=dst, dup_src=src, pointers=[(1, 8 * e, int(v), 0)
                                                          for e, v in enumerate(vals)])
    return snap, [pool, ptrs]


def moe_host_sample(seed: int = 0, pages: int = 32, page_bytes: int = 2 * MiB, dup_frac: float = 0.02,
                    pair_rows: int = 256, cols: int = 7168) -> tuple:
    """A host-side sample of the MoE workload with the pool's recipe, for
    CPU-side timing where the whole 30 GiB pool is not wanted: `pages` pages
    of bf16 ~ N(0, 0.02) with no exact zeros (torch's CPU generator), dup_frac
    of them overwritten with copies of other pages of the sample, the int64
    array of the 1536 expert base VAs (experts of 20 MiB from a fake pool
    base), and the two bf16 comparison pairs cut to `pair_rows` rows (one
    identical, one with 0.1% of elements one ulp away in the bit pattern).
    Returns (Snapshot with host regions, [Pair, Pair])."""
    import torch
    g = torch.Generator()
    g.manual_seed(seed + 909)
    n = pages * page_bytes // 2
    x = (torch.randn(n, generator=g) * 0.02).to(torch.bfloat16)
    tiny = torch.tensor(2.0 ** -120, dtype=torch.bfloat16)
    x = torch.where(x == 0, tiny, x)
    pool = x.view(torch.uint8).numpy().copy()
    rng = np.random.default_rng(seed + 910)
    ndup = int(round(pages * dup_frac))
    if ndup:
        perm = rng.permutation(pages)
        pv = pool.reshape(pages, page_bytes)
        for d, s_ in zip(np.sort(perm[:ndup]).tolist(), rng.choice(perm[ndup:], ndup).tolist()):
            pv[d] = pv[s_]
    n_exp = MOE_EXPERTS * MOE_LAYERS
    bases = fake_bases([pages * page_bytes, n_exp * 8], seed)
    vals = np.array([bases[0] + (e * MOE_EXPERT_BYTES) % (pages * page_bytes) for e in range(n_exp)], dtype=np.uint64)
    ptrs = vals.view(np.uint8).copy()
    snap = Snapshot(f"moe-pool-sample-{pages}x{page_bytes // MiB}MiB", page_bytes, [pool.size, ptrs.size],
                    bases, [pool, ptrs], [DT_BF16, DT_RAW])
    m = pair_rows * cols
    want = (torch.randn(m, generator=g)).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16).copy()
    want2 = (torch.randn(m, generator=g)).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16).copy()
    idx = np.sort(rng.choice(m, m // 1000, replace=False))
    got = want.copy()
    got[idx] = want[idx] ^ np.uint16(1)          # one ulp of the bit pattern
    return snap, [Pair(want2.copy(), want2, DT_BF16), Pair(got, want, DT_BF16, dict(perturbed=idx))]


def moe_pairs(seed: int = 0, rows: int = 4096, cols: int = 7168, device: str = "cuda"):
    """bf16 [rows, cols] ~ N(0, 1): one identical pair and one pair with 0.1% of
    elements times (1 +- 1e-2) (a step of one ulp where that rounds away).
    Returns [(got, want, truth)] as device tensors."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed + 505)
    want = torch.randn(rows * cols, generator=g, device=device).to(torch.bfloat16)
    want2 = torch.randn(rows * cols, generator=g, device=device).to(torch.bfloat16)
    rng = np.random.default_rng(seed + 506)
    n = rows * cols
    idx = np.sort(rng.choice(n, n // 1000, replace=False))
    ti = torch.from_numpy(idx).to(device)
    sign = torch.from_numpy(np.where(rng.random(idx.size) < 0.5, -1.0, 1.0)).to(device)
    x = want[ti]
    y = (x.double() * (1.0 + sign * 1e-2)).to(torch.bfloat16)
    same = y == x
    if bool(same.any()):
        bits = x.view(torch.int16)
        y = torch.where(same, (bits + 1).view(torch.bfloat16), y)
    got = want.clone()
    got[ti] = y
    torch.cuda.synchronize()
    return [(want2.clone(), want2, dict(perturbed=np.zeros(0, np.int64))),
            (got, want, dict(perturbed=idx))]


# --------------------------------------------------------------------------
# Batched validation jobs: many (got, want) pairs of uneven sizes
# --------------------------------------------------------------------------

@dataclass
class JobSet:
    """Jobs laid out in two device buffers (got, want) at 256-byte offsets."""
    sizes: list
    dtypes: list
    offsets: list
    got: object = None       # torch uint8 tensor
    want: object = None
    truth: dict = field(default_factory=dict)

    @property
    def total_bytes(self) -> int:
        return int(sum(self.sizes))


def batch_jobs(seed: int = 0, n: int = 4096, lo: int = 256, hi: int = 64 * MiB,
               frac_bad: float = 0.05, device: str = "cuda") -> JobSet:
    """n jobs, sizes log-uniform in [lo, hi], dtypes uniform over fp32 / fp16 /
    bf16 / int32 / uint8; want holds finite values of the dtype, got is a copy
    with 1..64 planted mismatches in a `frac_bad` share of the jobs (one ulp
    step of the bit pattern for floats, +1 for integers)."""
    import torch
    rng = np.random.default_rng(seed + 606)
    dts = [DT_F32, DT_F16, DT_BF16, DT_I32, DT_U8]
    sizes, dtypes, offsets = [], [], []
    off = 0
    for _ in range(n):
        dt = dts[int(rng.integers(0, 5))]
        b = int(np.exp(rng.uniform(math.log(lo), math.log(hi))))
        b = max(16, b // 16 * 16)
        sizes.append(b)
        dtypes.append(dt)
        offsets.append(off)
        off += (b + 255) // 256 * 256
    total = off
    want = torch.empty(total, dtype=torch.uint8, device=device)
    g = torch.Generator(device=device)
    g.manual_seed(seed + 607)
    for b, dt, o in zip(sizes, dtypes, offsets):
        fill_typed(want[o:o + b], dt, g)
    got = want.clone()
    bad = {}
    for k in np.nonzero(rng.random(n) < frac_bad)[0].tolist():
        dt, b, o = dtypes[k], sizes[k], offsets[k]
        m = int(rng.integers(1, 65))
        bad[k] = plant(got[o:o + b], dt, m, rng)
    torch.cuda.synchronize()
    return JobSet(sizes, dtypes, offsets, got, want, dict(planted=bad))


def fill_typed(seg, dt: int, g) -> None:
    """Fill a device byte segment with finite values of dtype dt: N(0, 1)
    for the float types, uniform 32-bit integers, uniform bytes."""
    import torch
    b = seg.numel()
    dev = seg.device
    if dt == DT_F32:
        seg.view(torch.float32).copy_(torch.randn(b // 4, generator=g, device=dev))
    elif dt == DT_F16:
        seg.view(torch.float16).copy_(torch.randn(b // 2, generator=g, device=dev))
    elif dt == DT_BF16:
        seg.view(torch.bfloat16).copy_(torch.randn(b // 2, generator=g, device=dev))
    elif dt == DT_I32:
        seg.view(torch.int32).copy_(torch.randint(-2**31, 2**31 - 1, (b // 4,), generator=g, device=dev,
                                                  dtype=torch.int64).to(torch.int32))
    else:
        seg.copy_(torch.randint(0, 256, (b,), generator=g, device=dev, dtype=torch.int32).to(torch.uint8))


def plant(seg, dt: int, m: int, rng) -> np.ndarray:
    """Change up to m elements of a device byte segment in place (drawn
    with replacement, duplicates dropped): the lowest bit of a float's
    pattern flipped (one ulp), +1 for integers.  Returns the sorted element
    indices changed."""
    import torch
    ne = seg.numel() // ESIZE[dt]
    idx = np.unique(rng.integers(0, ne, int(min(m, ne))))
    ti = torch.from_numpy(idx).to(seg.device)
    if dt in (DT_F32, DT_I32):
        v = seg.view(torch.int32)
        v[ti] = v[ti] + 1 if dt == DT_I32 else v[ti] ^ 1
    elif dt in (DT_F16, DT_BF16):
        v = seg.view(torch.int16)
        v[ti] = v[ti] ^ 1
    else:
        seg[ti] = seg[ti] + 1
    return idx


def golden_set(seed: int = 0, n: int = 64, lo: int = MiB, hi: int = 2 * GiB, device: str = "cuda"):
    """n resident golden buffers, sizes log-uniform in [lo, hi] (multiples
    of 256 bytes), dtypes uniform over the five, in one device allocation.
    Returns (data u8 tensor, sizes, dtypes, offsets)."""
    import torch
    rng = np.random.default_rng(seed + 808)
    dts = [DT_F32, DT_F16, DT_BF16, DT_I32, DT_U8]
    sizes = [int(np.exp(rng.uniform(math.log(lo), math.log(hi)))) // 256 * 256 for _ in range(n)]
    dtypes = [dts[int(rng.integers(0, 5))] for _ in range(n)]
    offsets = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64).tolist()
    data = torch.empty(int(sum(sizes)), dtype=torch.uint8, device=device)
    g = torch.Generator(device=device)
    g.manual_seed(seed + 809)
    for b, dt, o in zip(sizes, dtypes, offsets):
        fill_typed(data[o:o + b], dt, g)
    torch.cuda.synchronize()
    return data, sizes, dtypes, offsets
