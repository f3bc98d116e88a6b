"""The oracle's pins must catch plausible mistakes in the oracle itself.

Each case plants one mistake in a copy of oracle/xt_oracle.c (on the CPU, in a
temporary directory), loads the copy in place of the real oracle and checks
that at least one pin check fails.
"""
import ctypes
import os
import random
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import tests.test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "xt_oracle.c")

MUTANTS = {
    "local_restart": ("int64_t M = D > 0 ? D + score(sc, t[i], q[j]) : 0;",
                      "int64_t M = D + score(sc, t[i], q[j]);"),
    "gap_open_from_E_only": ("int64_t E = max2(0, max2(Hc[j] - alpha, Ec[j] - beta));",
                             "int64_t E = max2(0, max2(Hc[j] - beta, Ec[j] - beta));"),
    "F_wrong_extend": ("int64_t F = max2(0, max2(Hp[j + 1] - alpha, Fp[j + 1] - beta));",
                       "int64_t F = max2(0, max2(Hp[j + 1] - alpha, Fp[j + 1] - alpha));"),
    "diag_from_up": ("int64_t D = Hp[j];", "int64_t D = Hp[j + 1];"),
    "band_off_by_one": ("return iabs64(r - c) <= w;", "return iabs64(r - c) < w;"),
    "smallest_j_tie": ("if (H >= m) { m = H; mj = j; }", "if (H > m) { m = H; mj = j; }"),
    "gscore_latest_row": ("if (g > 0 && g > gscore)", "if (g > 0 && g >= gscore)"),
    "zdrop_no_gap_correction": ("int64_t drop = best - m - iabs64(d) * beta;",
                                "int64_t drop = best - m;"),
    "zdrop_ties_stop": ("      if (drop > sc->zdrop) break;\n    }\n    int64_t* tmp;",
                        "      if (drop >= sc->zdrop) break;\n    }\n    int64_t* tmp;"),
    "zdrop_signed_offset": ("int64_t drop = best - m - iabs64(d) * beta;",
                            "int64_t drop = best - m - d * beta;"),
    "boundary_row_missing_open": ("int64_t v = max2(0, h0 - alpha - beta * c);",
                                  "int64_t v = max2(0, h0 - beta - beta * c);"),
    "n_scored_as_mismatch": ("if (a >= 4 || b >= 4) return sc->n_score;",
                             "if (a >= 4 && b >= 4) return sc->n_score;"),
    "transposed_score": ("score(sc, t[i], q[j])", "score(sc, t[j < tlen ? j : 0], q[i < qlen ? i : 0])"),
    "max_off_signless": ("max_off = max2(max_off, iabs64(mj - i));",
                         "max_off = max2(max_off, mj - i);"),
    "cells_count_all_rows": ("for (int64_t i = 0; i <= last_live; ++i) n += band_width(i, qlen, w);",
                             "for (int64_t i = 0; i < tlen; ++i) n += band_width(i, qlen, w);"),
}


def build_mutant(name, tmp):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert old in src, name
    path = os.path.join(tmp, f"{name}.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    so = os.path.join(tmp, f"lib{name}.so")
    subprocess.run(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-pthread", path, "-o", so],
                   check=True)
    return so


def pins_fail():
    """Run the pin checks against whatever library oracle._LIB points at."""
    checks = [
        lambda: [pins.test_handworked_tables(n) for n in
                 ("handworked_identical_3x3.json", "handworked_anchoring_3x3.json",
                  "handworked_band_n_3x4.json")],
        pins.test_handworked_zdrop_tail,
        pins.test_single_deletion_closed_form,
        pins.test_band_zero_is_diagonal_only,
        pins.test_all_mismatch_single_cell_gscore,
        pins.test_boundary_runs_match_enumeration,
        pins.test_path_enumeration_fixes_every_cell,
        pins.test_path_enumeration_fixes_zdrop,
    ]
    for c in checks:
        try:
            c()
        except AssertionError:
            return True
    return False


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, monkeypatch):
    with tempfile.TemporaryDirectory() as tmp:
        so = build_mutant(name, tmp)
        saved = oracle._LIB
        try:
            oracle._LIB = None
            monkeypatch.setattr(oracle, "build", lambda force=False: so)
            assert pins_fail(), f"no pin detects mutant {name}"
        finally:
            oracle._LIB = saved


# ------------------------------------------- the BWA-MEM-compatible variant
import tests.test_oracle_bwa_pins as bwa_pins  # noqa: E402

BWA_MUTANTS = {
    "bwa_ins_open_from_H": ("max2(Mc[j] - oe_ins, Ec[j] - e_ins)", "max2(Hc[j] - oe_ins, Ec[j] - e_ins)"),
    "bwa_del_open_from_H": ("max2(Mp[j + 1] - oe_del, Fp[j + 1] - e_del)",
                            "max2(Hp[j + 1] - oe_del, Fp[j + 1] - e_del)"),
    "bwa_ins_uses_del_penalties": ("max2(Mc[j] - oe_ins, Ec[j] - e_ins)",
                                   "max2(Mc[j] - oe_del, Ec[j] - e_del)"),
    "bwa_zdrop_ins_extension_only": ("best - m - (di - dj) * e_del :", "best - m - (di - dj) * e_ins :"),
    "bwa_zdrop_del_extension_only": ("best - m - (dj - di) * e_ins;", "best - m - (dj - di) * e_del;"),
    "bwa_gscore_earliest_row": ("Hc[qlen] >= gscore", "Hc[qlen] > gscore"),
    "bwa_gscore_positive_only": ("end == qlen && Hc[qlen] >= gscore",
                                 "end == qlen && Hc[qlen] > 0 && Hc[qlen] >= gscore"),
    "bwa_trim_live_run_only": ("    int64_t a = beg, b = end - 1;\n    while (Hc[a + 1] == 0) ++a;  /* Hc[a+1] holds column a */\n    while (Hc[b + 1] == 0) --b;",
                               "    int64_t a = mj, b = mj;\n    while (a - 1 >= beg && Hc[a] > 0) --a;\n    while (b + 1 < end && Hc[b + 2] > 0) ++b;"),
    "bwa_trim_drops_run_start": ("else { next_beg = a; next_end = b + 2; }",
                                 "else { next_beg = a + 1; next_end = b + 2; }"),
    "bwa_trim_no_diagonal_step": ("else { next_beg = a; next_end = b + 2; }",
                                  "else { next_beg = a; next_end = b + 1; }"),
    "bwa_narrow_off_by_one": ("(gain - sc->o_del) / sc->e_del + 1;", "(gain - sc->o_del) / sc->e_del;"),
    "bwa_narrow_ignores_end_bonus": ("qlen * sc->match + sc->end_bonus;", "qlen * sc->match;"),
    "bwa_no_dead_row_stop": ("    if (m == 0) break;\n    n_cells", "    n_cells"),
    "bwa_range_ignores_band": ("int64_t beg = max2(next_beg, i - w);", "int64_t beg = next_beg;"),
    "bwa_diag_from_up": ("const int64_t D = Hp[j];", "const int64_t D = Hp[j + 1];"),
    "bwa_boundary_col_ins_penalty": ("max2(0, h0 - oe_del - e_del * i)", "max2(0, h0 - oe_ins - e_ins * i)"),
    "bwa_best_tie_latest": ("    if (m > best) {\n      best = m; bi = i; bj = mj;\n      max_off = max2(max_off, iabs64(mj - i));\n    } else if (sc->zdrop > 0) {\n      const int64_t di",
                            "    if (m >= best) {\n      best = m; bi = i; bj = mj;\n      max_off = max2(max_off, iabs64(mj - i));\n    } else if (sc->zdrop > 0) {\n      const int64_t di"),
}


def build_bwa_mutant(name, tmp):
    old, new = BWA_MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = os.path.join(tmp, f"{name}.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    so = os.path.join(tmp, f"lib{name}.so")
    subprocess.run(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-pthread", path, "-o", so],
                   check=True)
    return so


def bwa_pins_fail():
    checks = [
        bwa_pins.test_handworked_trimming_table,
        bwa_pins.test_handworked_trimming_keeps_interior_dead_cells,
        bwa_pins.test_handworked_zdrop_insertion_direction,
        bwa_pins.test_boundary_runs_by_enumeration,
        bwa_pins.test_insertion_then_deletion_is_not_a_path,
        lambda: [bwa_pins.test_zdrop_deletion_direction(z, c) for z, c in ((1, 2), (2, 6), (0, 6))],
        lambda: [bwa_pins.test_narrowing_threshold(k, e, f) for k, e, f in
                 ((11, 12, True), (12, 13, True), (12, 12, False), (6, 7, True), (7, 7, False))],
        lambda: [bwa_pins.test_path_enumeration(si) for si in range(len(bwa_pins.PATH_SCORINGS))],
        lambda: [bwa_pins.test_identical_sequences(L) for L in (1, 3, 17, 60)],
    ]
    for c in checks:
        try:
            c()
        except AssertionError:
            return True
    return False


@pytest.mark.parametrize("name", sorted(BWA_MUTANTS))
def test_bwa_pins_catch_mutant(name, monkeypatch):
    with tempfile.TemporaryDirectory() as tmp:
        so = build_bwa_mutant(name, tmp)
        saved = oracle._LIB
        try:
            oracle._LIB = None
            monkeypatch.setattr(oracle, "build", lambda force=False: so)
            assert bwa_pins_fail(), f"no pin detects mutant {name}"
        finally:
            oracle._LIB = saved
