"""Pins of the oracle's per-dtype FP64 comparison.

- Which elements mismatch (count, first index) against numpy.isclose on the
  values widened by numpy/torch (a library routine; equal_nan=True gives the
  NaN == NaN rule, infinities are close only when equal).
- max_abs and max_rel against exact rational arithmetic (fractions): an IEEE
  subtraction or division is the exact result rounded once, so
  float(Fraction(a) - Fraction(b)) must equal the oracle's FP64 value bit for
  bit.
- fp16 / bf16 widening of every bit pattern against numpy / torch.
- Planted truth: identical buffers compare clean; planted perturbations and
  NaNs are counted exactly.
"""
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
from paper_2605_03208_gb300 import workloads as W


def widen(x: np.ndarray, dt: int) -> np.ndarray:
    """Widen to float64 with numpy / torch (independent of the oracle's bit code)."""
    if dt == W.DT_BF16:
        t = torch.from_numpy(x.view(np.int16).copy()).view(torch.bfloat16)
        return t.to(torch.float64).numpy()
    return x.astype(np.float64)


def expected(got, want, dt, atol=0.0, rtol=0.0):
    a, b = widen(got, dt), widen(want, dt)
    close = np.isclose(a, b, rtol=rtol, atol=atol, equal_nan=True)
    mism = np.nonzero(~close)[0]
    unequal = ~(np.isnan(a) | np.isnan(b)) & (a != b)
    max_abs, max_rel = 0.0, 0.0
    for i in np.nonzero(unequal)[0]:
        ai, bi = float(a[i]), float(b[i])
        if np.isinf(ai) or np.isinf(bi):
            d = float("inf")
        else:
            d = float(abs(Fraction(ai) - Fraction(bi)))
        if bi == 0.0 or np.isinf(d):
            r = float("inf")
        else:
            r = float(Fraction(d) / abs(Fraction(bi)))
        max_abs, max_rel = max(max_abs, d), max(max_rel, r)
    return dict(mismatches=len(mism), first=int(mism[0]) if len(mism) else -1,
                max_abs=max_abs, max_rel=max_rel,
                nan_got=int(np.isnan(a).sum()), nan_want=int(np.isnan(b).sum()),
                nan_mismatch=int((np.isnan(a) != np.isnan(b)).sum()))


def check(rec, exp):
    for k, v in exp.items():
        got = rec[k].item()
        if isinstance(v, float):
            assert np.float64(got).tobytes() == np.float64(v).tobytes(), (k, got, v)
        else:
            assert got == v, (k, got, v)


@pytest.mark.parametrize("seed", [0, 1])
def test_mixed_dtypes_against_isclose_and_exact_arithmetic(seed):
    for p in W.mixed_pairs(seed, n_pairs=10, max_elems=4000):
        rec = oracle.compare(p.got, p.want, p.dtype)
        check(rec, expected(p.got, p.want, p.dtype))
        assert rec["mismatches"] == len(p.truth["perturbed"])


@pytest.mark.parametrize("atol,rtol", [(0.0, 0.0), (1e-7, 0.0), (0.0, 1e-6), (1e-6, 1e-5),
                                       (0.5, 0.0)])
def test_tolerances_against_isclose(atol, rtol):
    rng = np.random.default_rng(5)
    want = rng.standard_normal(20000, dtype=np.float32)
    got = want.copy()
    idx = rng.choice(want.size, 400, replace=False)
    got[idx] = (want[idx] * (1 + rng.uniform(-1e-5, 1e-5, idx.size))).astype(np.float32)
    rec = oracle.compare(got, want, W.DT_F32, atol, rtol)
    check(rec, expected(got, want, W.DT_F32, atol, rtol))


def test_tolerance_scales_with_want_not_got():
    """rtol multiplies |want| (numpy.isclose's b): pairs whose verdict flips
    when it multiplies |got| instead, in fp32, fp16 and int32."""
    want = np.array([1.0, 1.0, 4.0, -2.0, 10.0, 0.5], dtype=np.float64)
    got = np.array([1.5, 0.7, 2.0, -1.0, 6.5, 0.75], dtype=np.float64)
    for dt, npdt in ((W.DT_F32, np.float32), (W.DT_F16, np.float16)):
        g, w = got.astype(npdt), want.astype(npdt)
        rec = oracle.compare(g, w, dt, 0.0, 0.4)
        check(rec, expected(g, w, dt, 0.0, 0.4))
        assert rec["mismatches"] == 4 and rec["first"] == 0      # elements 0, 2, 3, 5
    gi, wi = np.array([15, 7, 40, -10], dtype=np.int32), np.array([10, 10, 40, -20], dtype=np.int32)
    rec = oracle.compare(gi, wi, W.DT_I32, 0.0, 0.4)
    check(rec, expected(gi, wi, W.DT_I32, 0.0, 0.4))
    assert rec["mismatches"] == 2 and rec["first"] == 0          # elements 0, 3


def test_identical_buffers_compare_clean():
    rng = np.random.default_rng(0)
    for dt, arr in [(W.DT_F32, rng.standard_normal(5000, dtype=np.float32)),
                    (W.DT_I32, rng.integers(-9, 9, 5000).astype(np.int32)),
                    (W.DT_U8, rng.integers(0, 256, 5000).astype(np.uint8))]:
        rec = oracle.compare(arr, arr.copy(), dt)
        assert rec["mismatches"] == 0 and rec["first"] == -1
        assert rec["max_abs"] == 0.0 and rec["max_rel"] == 0.0


def test_special_values():
    inf, nan = np.float32(np.inf), np.float32(np.nan)
    got = np.array([0.0, -0.0, inf, inf, -inf, 1.0, nan, nan, 2.0, 3.0, 0.0, 1e-45],
                   dtype=np.float32)
    want = np.array([-0.0, 0.0, inf, -inf, 5.0, inf, nan, 1.0, nan, 3.0, 1.0, 0.0],
                    dtype=np.float32)
    rec = oracle.compare(got, want, W.DT_F32, atol=1e30, rtol=1e30)
    # +-0 equal, equal infinities equal, NaN==NaN; infinities never within
    # tolerance; NaN-vs-number always mismatches.
    assert rec["mismatches"] == 5 and rec["first"] == 3
    assert rec["nan_mismatch"] == 2 and rec["nan_got"] == 2 and rec["nan_want"] == 2
    assert rec["max_abs"] == np.inf and rec["max_rel"] == np.inf
    check(rec, expected(got, want, W.DT_F32, 1e30, 1e30))


def test_integer_extremes():
    g = np.array([-2**31, 2**31 - 1, 0, 7], dtype=np.int32)
    w = np.array([2**31 - 1, -2**31, 0, 7], dtype=np.int32)
    rec = oracle.compare(g, w, W.DT_I32)
    assert rec["mismatches"] == 2 and rec["first"] == 0
    assert rec["max_abs"] == 2.0**32 - 1
    g8 = np.array([0, 255, 9], dtype=np.uint8)
    w8 = np.array([255, 0, 9], dtype=np.uint8)
    rec = oracle.compare(g8, w8, W.DT_U8)
    assert rec["mismatches"] == 2 and rec["max_abs"] == 255.0 and rec["max_rel"] == np.inf


def test_half_widening_every_bit_pattern():
    bits = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    zero = np.zeros(1, dtype=np.uint16)
    f16 = bits.view(np.float16).astype(np.float64)
    bf16 = widen(bits.copy(), W.DT_BF16)
    for b in range(0, 65536, 1):
        if b % 7 and not (0x7C00 <= (b & 0x7FFF) <= 0x7C10) and (b & 0x7FFF) > 8:
            continue                         # every 7th pattern plus all edges
        g = bits[b:b + 1]
        r16 = oracle.compare(g, zero, W.DT_F16)
        rbf = oracle.compare(g, zero, W.DT_BF16)
        for rec, ref in ((r16, f16[b]), (rbf, bf16[b])):
            if np.isnan(ref):
                assert rec["nan_got"] == 1
            else:
                assert rec["max_abs"] == abs(ref), (b, rec["max_abs"], ref)


def test_planted_tiny_pairs():
    for p in W.tiny_pairs(0, n=1 << 16):
        rec = oracle.compare(p.got, p.want, W.DT_F32)
        t = p.truth
        assert rec["mismatches"] == len(t["perturbed"]) + len(t["nan_one"])
        assert rec["nan_mismatch"] == len(t["nan_one"])
        assert rec["nan_got"] == len(t["nan_both"]) + min(5, len(t["nan_one"]))
        firsts = np.concatenate([t["perturbed"], t["nan_one"]])
        assert rec["first"] == (int(firsts.min()) if firsts.size else -1)
        if len(t["perturbed"]):
            # |delta| of 1e-6 relative, rounded to fp32: the max relative error
            # lies within one fp32 ulp of 1e-6
            assert 1e-6 - 2**-23 <= rec["max_rel"] <= 1e-6 + 2**-23
