"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of oracle/kc_oracle.c -- a wrong
rotation or shift, a wrong sign or prime, a transposed operand, a dropped
term, an off-by-one bound, a wrong order, a dropped rule -- compiles it with
the oracle's own flags, swaps it in for the real library, and runs the pins
of the part it touches (the functions of tests/test_oracle_*.py).  At least
one pin must fail.  The mistakes are chosen so that the mutant never reads
or writes outside the buffers it is given and never loops forever; the
unmodified oracle passes the same pins in the other test modules.
"""
import os
import subprocess

import pytest

import oracle.kc_oracle as ko
from tests import test_oracle_census as TC
from tests import test_oracle_compare as TK
from tests import test_oracle_dedup as TD
from tests import test_oracle_digest as TG


def _digest_pins():
    TG.test_page_first_closed_form()
    TG.test_digest_partial_pages_are_not_padded()
    TG.test_zero_flag_is_every_byte_of_the_page()
    TG.test_golden_xxh64_edges_reproduced_by_oracle()
    if TG.xxh_ref is not None:
        TG.test_xxh64_structured_inputs()
        TG.test_digest_pages_match_libxxhash_and_planted_zero_pages()


def _dedup_pins():
    TD.test_dedup_partial_prefix_is_a_separate_class()
    TD.test_planted_copies_map_to_source_and_roundtrip()
    for seed in range(6):
        for bits in (64, 2, 0):
            TD.test_dedup_matches_bruteforce(seed, bits)


def _census_pins():
    TC.test_census_half_open_ranges_and_window()
    TC.test_census_window_edges()
    TC.test_census_finds_every_planted_pointer()
    TC.test_census_llama_pointer_table()
    TC.test_census_truncation_keeps_true_counts_and_overlap_rejected()
    TC.test_census_scan_prefix_and_target_only()
    for seed in (0, 1, 2):
        TC.test_census_matches_linear_scan(seed)


def _compare_pins():
    TK.test_identical_buffers_compare_clean()
    TK.test_special_values()
    TK.test_integer_extremes()
    TK.test_half_widening_every_bit_pattern()
    TK.test_planted_tiny_pairs()
    TK.test_tolerance_scales_with_want_not_got()
    for seed in (0, 1):
        TK.test_mixed_dtypes_against_isclose_and_exact_arithmetic(seed)
    for atol, rtol in ((0.0, 0.0), (1e-7, 0.0), (0.0, 1e-6), (1e-6, 1e-5)):
        TK.test_tolerances_against_isclose(atol, rtol)


# (name, text in kc_oracle.c -- must occur exactly once, replacement, pins)
MUTANTS = [
    # XXH64
    ("round rotation 31 -> 30", "    acc = rotl64(acc, 31);\n", "    acc = rotl64(acc, 30);\n", _digest_pins),
    ("lane read big-endian", "for (int i = 7; i >= 0; --i) v = (v << 8) | (uint64_t)p[i];",
     "for (int i = 0; i <= 7; ++i) v = (v << 8) | (uint64_t)p[i];", _digest_pins),
    ("fourth accumulator start sign", "uint64_t a4 = seed - XP1;", "uint64_t a4 = seed + XP1;", _digest_pins),
    ("convergence merges a3 twice", "acc = xmerge(acc, a4);", "acc = xmerge(acc, a3);", _digest_pins),
    ("length add uses the remainder", "acc = acc + len;", "acc = acc + remaining;", _digest_pins),
    ("4-byte tail prime", "acc = rotl64(acc, 23) * XP2 + XP3;", "acc = rotl64(acc, 23) * XP1 + XP3;", _digest_pins),
    ("1-byte tail rotation", "acc = rotl64(acc, 11) * XP1;", "acc = rotl64(acc, 13) * XP1;", _digest_pins),
    ("avalanche shift 29 -> 31", "acc = acc ^ (acc >> 29);", "acc = acc ^ (acc >> 31);", _digest_pins),
    # page digest
    ("sub-8-byte tail of a partial page dropped", "hash[pid] = kco_xxh64(pg, len, 0);",
     "hash[pid] = kco_xxh64(pg, len & ~7ULL, 0);", _digest_pins),
    ("zero flag skips the first byte", "for (uint64_t b = 0; b < len; ++b)\n                if (pg[b] != 0)",
     "for (uint64_t b = 1; b < len; ++b)\n                if (pg[b] != 0)", _digest_pins),
    # dedup
    ("group visited in decreasing page id", "if (x->page != y->page) return x->page < y->page ? -1 : 1;",
     "if (x->page != y->page) return x->page > y->page ? -1 : 1;", _dedup_pins),
    ("length not part of page equality", "if (lp != lq) return 0;", "if (lp > lq) return 0;", _dedup_pins),
    ("blob ids also count zero pages", "if (!zero[p] && canon[p] == p) blob_of[p] = next++;",
     "if (canon[p] == p) blob_of[p] = next++;", _dedup_pins),
    ("restore leaves zero pages unwritten", "if (tbl_blob[p] == KCO_BLOB_ZERO) memset(img[a] + off, 0, (size_t)len);",
     "if (tbl_blob[p] == KCO_BLOB_ZERO) (void)0;", _dedup_pins),
    ("equal hashes taken as equal pages", "if (pages_equal(n, img, bytes, pf, S, p, reps[r])) break;",
     "if (1) break;", _dedup_pins),
    # census
    ("range end inclusive", "if (lo > 0 && v < rg[lo - 1].end)", "if (lo > 0 && v <= rg[lo - 1].end)", _census_pins),
    ("window start exclusive", "else if (win_lo <= v && v < win_hi)", "else if (win_lo < v && v < win_hi)",
     _census_pins),
    ("last word of a region skipped", "for (uint64_t o = 0; o + 8 <= lim; o += 8)",
     "for (uint64_t o = 0; o + 16 <= lim; o += 8)", _census_pins),
    ("outside hits counted as inside", "{ target = -1; ++nout; }", "{ target = -1; ++nin; }", _census_pins),
    ("range end taken from the scanned prefix", "rg[k].end = base[k] + bytes[k];",
     "rg[k].end = base[k] + (scan ? scan[k] : bytes[k]);", _census_pins),
    ("target = sorted index, not list index", "{ target = rg[lo - 1].id; ++nin; }",
     "{ target = lo - 1; ++nin; }", _census_pins),
    # compare
    ("relative error divides by |got|", "d / fabs(b);", "d / fabs(a);", _compare_pins),
    ("tolerance scales with |got|", "mis = d > atol + rtol * fabs(b);", "mis = d > atol + rtol * fabs(a);",
     _compare_pins),
    ("NaN == NaN counted as a mismatch", "if (na && nb) continue;",
     "if (na && nb) { r.mismatches += 1; continue; }", _compare_pins),
    ("last mismatch index instead of first", "        if (mis) {\n            r.mismatches += 1;\n"
     "            if (r.first < 0) r.first = (int64_t)i;",
     "        if (mis) {\n            r.mismatches += 1;\n            r.first = (int64_t)i;", _compare_pins),
    ("NaN count of got reads want", "r.nan_got += (uint64_t)na;", "r.nan_got += (uint64_t)nb;", _compare_pins),
    ("fp16 subnormal scale", "if (ex == 0) v = ldexp((double)fr, -24);", "if (ex == 0) v = ldexp((double)fr, -25);",
     _compare_pins),
    ("bf16 widened from the wrong bit", "uint32_t u = (uint32_t)h << 16;", "uint32_t u = (uint32_t)h << 15;",
     _compare_pins),
]


@pytest.mark.parametrize("name,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_planted_mistake(tmp_path, monkeypatch, name, old, new, pins):
    with open(ko._SRC) as f:
        src = f.read()
    assert src.count(old) == 1, f"mutation site not unique: {old!r}"
    c = tmp_path / "mutant.c"
    c.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                    "-o", str(so), str(c), "-lm"], check=True)
    monkeypatch.setattr(ko, "_lib", ko._load(str(so)))
    with pytest.raises(Exception):   # a failed assert, or outputs a pin cannot even read
        pins()


def test_unmodified_oracle_passes_every_pin_set():
    for pins in (_digest_pins, _dedup_pins, _census_pins, _compare_pins):
        pins()
