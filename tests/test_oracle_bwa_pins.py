"""Pins for the BWA-MEM-compatible variant of the CPU oracle, each independent
of the oracle's own code.

* hand-worked tables (tests/golden/handworked_bwa_*.json): every H/M/E/F value,
  row range and row summary of small extensions, derived on paper;
* independent path enumeration: every alignment path from the seed is scored
  move by move under the variant's move rules (a gap opens only after a match
  step or the seed, so an insertion never touches a deletion), which fixes
  every cell of tiny extensions with trimming and narrowing switched off;
* closed forms: identical sequences; the band-narrowing threshold (a
  deletion of k bases is reachable exactly when k <= the narrowed band); the
  z-drop in the deletion direction; an insertion directly followed by a
  deletion, which the default definition allows and this variant does not;
* invariants: trimming and the move rules only remove paths, so cell values
  never rise; output ranges.
"""
import json
import os
import random

import numpy as np
import pytest

import oracle
from oracle import BWA_NO_NARROW, BWA_NO_TRIM, BwaScoring, Scoring

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CODES = {"A": 0, "C": 1, "G": 2, "T": 3, "N": 4}


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------- hand-worked
def test_handworked_trimming_table():
    g = load("handworked_bwa_trim_3x4.json")
    sc = BwaScoring(**g["scoring"])
    tr = oracle.extend_one_bwa(g["q"], g["t"], g["h0"], sc, trace=True)
    for k in ("H", "M", "E", "F"):
        assert getattr(tr, k).tolist() == g[k], k
    assert tr.row_beg.tolist() == g["row_beg"]
    assert tr.row_end.tolist() == g["row_end"]
    assert tr.row_m.tolist() == g["row_m"]
    assert tr.row_mj.tolist() == g["row_mj"]
    assert list(tr.result) == g["result"] and tr.cells == g["cells"]
    u = g["untrimmed"]
    tu = oracle.extend_one_bwa(g["q"], g["t"], g["h0"], sc, flags=BWA_NO_TRIM, trace=True)
    assert tu.row_end.tolist() == u["row_end"]
    assert tu.H[3, 4] == u["H_row2_col3"] and tu.E[3, 4] == u["E_row2_col3"]
    assert list(tu.result) == u["result"] and tu.cells == u["cells"]


def test_handworked_trimming_keeps_interior_dead_cells():
    """Row trimming drops only the dead cells at the two ends of a row: a row
    with two live cells and a dead one between them computes all three next
    row, and the far cell's descendants reach the last query column."""
    g = load("handworked_bwa_trim_ends_3x3.json")
    sc = BwaScoring(**g["scoring"])
    tr = oracle.extend_one_bwa(g["q"], g["t"], g["h0"], sc, trace=True)
    for k in ("H", "M", "E", "F"):
        assert getattr(tr, k).tolist() == g[k], k
    assert tr.row_beg.tolist() == g["row_beg"]
    assert tr.row_end.tolist() == g["row_end"]
    assert tr.row_m.tolist() == g["row_m"]
    assert tr.row_mj.tolist() == g["row_mj"]
    assert list(tr.result) == g["result"] and tr.cells == g["cells"]
    # the earlier live-run reading gives a different gscore on this pair
    assert g["live_run_rule"]["result"] != g["result"]


def test_handworked_zdrop_insertion_direction():
    g = load("handworked_bwa_zdrop_ins_3x4.json")
    for case in g["cases"]:
        sc = BwaScoring(**g["scoring"], zdrop=case["zdrop"])
        tr = oracle.extend_one_bwa(g["q"], g["t"], g["h0"], sc, trace=True)
        n = len(g["t"]) if case["stop_row"] is None else case["stop_row"] + 1
        assert list(tr.result) == case["result"], case
        assert tr.cells == case["cells"], case
        assert tr.row_m.tolist() == g["row_m"][:n] and tr.row_mj.tolist() == g["row_mj"][:n]
        for k in ("H", "M", "E", "F"):
            assert getattr(tr, k)[:n + 1].tolist() == g[k][:n + 1], (k, case)


# ------------------------------------------------------- path enumeration
def enumerate_cells(q, t, h0, sc: BwaScoring, w):
    """Best value per cell and last move, over every alive path from the seed.

    A path starts at (-1,-1) with value h0 and moves M (diagonal, + score),
    I (consumes a query base), D (consumes a target base).  A gap's first base
    costs o + e and each further base e; a gap may follow only an M move or
    the seed, so I and D are never adjacent.  A path stays alive while every
    value it reaches is > 0, and only in-band cells (|r - c| <= w) are used.
    Returns dicts {(r, c): value} for paths whose last move is M (the value
    may be <= 0 there: the move is made from a live cell), I, and D."""
    qa = [CODES[ch] for ch in q]
    ta = [CODES[ch] for ch in t]

    def s(r, c):
        if qa[c] >= 4 or ta[r] >= 4:
            return sc.n_score
        return sc.match if qa[c] == ta[r] else sc.mismatch

    best = {"M": {}, "I": {}, "D": {}}
    stack = [(-1, -1, "S", h0)]
    while stack:
        r, c, last, v = stack.pop()
        # M move
        if r + 1 < len(ta) and c + 1 < len(qa) and abs((r + 1) - (c + 1)) <= w:
            nv = v + s(r + 1, c + 1)
            key = (r + 1, c + 1)
            best["M"][key] = max(best["M"].get(key, nv), nv)
            if nv > 0:
                stack.append((r + 1, c + 1, "M", nv))
        # I move
        if last != "D" and c + 1 < len(qa) and abs(r - (c + 1)) <= w:
            nv = v - (sc.e_ins if last == "I" else sc.o_ins + sc.e_ins)
            if nv > 0:
                best["I"][(r, c + 1)] = max(best["I"].get((r, c + 1), 0), nv)
                stack.append((r, c + 1, "I", nv))
        # D move
        if last != "I" and r + 1 < len(ta) and abs((r + 1) - c) <= w:
            nv = v - (sc.e_del if last == "D" else sc.o_del + sc.e_del)
            if nv > 0:
                best["D"][(r + 1, c)] = max(best["D"].get((r + 1, c), 0), nv)
                stack.append((r + 1, c, "D", nv))
    return best


def expected_from_paths(q, t, h0, sc, w):
    """The variant's outputs with trimming and narrowing off and no z-drop,
    from the enumerated cell values: rows in order, row maxima over the band
    (largest column on ties), gscore on the latest row, stop at a dead row."""
    ql, tl = len(q), len(t)
    b = enumerate_cells(q, t, h0, sc, w)
    H = np.zeros((tl + 1, ql + 1), np.int64)
    M = np.zeros_like(H)
    E = np.zeros_like(H)
    F = np.zeros_like(H)
    for (r, c), v in b["M"].items():
        M[r + 1, c + 1] = v
    for (r, c), v in b["I"].items():
        E[r + 1, c + 1] = v
    for (r, c), v in b["D"].items():
        F[r + 1, c + 1] = v
    H[:] = np.maximum(np.maximum(M, E), np.maximum(F, 0))
    best, bi, bj, max_off = h0, -1, -1, 0
    gscore, gtle, cells, n_rows = -1, 0, 0, 0
    for i in range(tl):
        lo, hi = max(0, i - w), min(ql, i + w + 1)
        n_rows = i + 1
        if hi <= lo:
            break
        row = H[i + 1, lo + 1:hi + 1]
        m = int(row.max())
        mj = lo + int(np.nonzero(row == m)[0][-1])
        if hi == ql and H[i + 1, ql] >= gscore:
            gscore, gtle = int(H[i + 1, ql]), i + 1
        if m == 0:
            break
        cells += hi - lo
        if m > best:
            best, bi, bj = m, i, mj
            max_off = max(max_off, abs(mj - i))
    return (best, bj + 1, bi + 1, gscore, gtle, max_off, 0), cells, n_rows, (H, M, E, F)


def rand_seq(rng, n, alphabet):
    return "".join(rng.choice(alphabet) for _ in range(n))


PATH_SCORINGS = [
    BwaScoring(match=1, mismatch=-3, o_del=1, e_del=1, o_ins=2, e_ins=1, zdrop=0),
    BwaScoring(match=2, mismatch=-2, o_del=0, e_del=2, o_ins=3, e_ins=1, zdrop=0, n_score=-2),
    BwaScoring(match=1, mismatch=-6, o_del=2, e_del=1, o_ins=1, e_ins=1, zdrop=0),
    BwaScoring(match=3, mismatch=-1, o_del=4, e_del=2, o_ins=0, e_ins=3, zdrop=0),
]


@pytest.mark.parametrize("si", range(len(PATH_SCORINGS)))
def test_path_enumeration(si):
    sc = PATH_SCORINGS[si]
    rng = random.Random(100 + si)
    n_checked = 0
    for case in range(60):
        ql, tl = rng.randint(1, 5), rng.randint(1, 5)
        alphabet = "ACN" if case % 5 == 0 else "AC"
        q, t = rand_seq(rng, ql, alphabet), rand_seq(rng, tl, alphabet)
        h0 = rng.randint(1, 12)
        w = rng.choice([1, 2, 10])
        scw = BwaScoring(**{**sc.__dict__, "w": w})
        want, cells, n_rows, mats = expected_from_paths(q, t, h0, scw, w)
        tr = oracle.extend_one_bwa(q, t, h0, scw, flags=BWA_NO_TRIM | BWA_NO_NARROW, trace=True)
        what = (q, t, h0, w)
        assert tr.result == want, what
        assert tr.cells == cells, what
        assert len(tr.row_m) == n_rows, what
        for name, mat in zip("HMEF", mats):
            # rows after the stop row are not evaluated; column -1 is the
            # boundary run, checked through the row-0 and column-0 values
            got = getattr(tr, name)[1:n_rows + 1, 1:]
            assert got.tolist() == mat[1:n_rows + 1, 1:].tolist(), (name, what)
        n_checked += 1
    assert n_checked == 60


def test_boundary_runs_by_enumeration():
    # the boundary row and column values are the seed's gap runs
    sc = BwaScoring(match=1, mismatch=-4, o_del=2, e_del=1, o_ins=3, e_ins=2, w=10, zdrop=0)
    tr = oracle.extend_one_bwa("CCCCC", "GGGGG", 20, sc, flags=BWA_NO_NARROW, trace=True)
    assert tr.H[0, 1:].tolist() == [20 - 5 - 2 * c for c in range(5)]
    assert tr.H[1:, 0].tolist()[:len(tr.row_m)] == [20 - 3 - r for r in range(len(tr.row_m))]


# ----------------------------------------------------------------- closed forms
@pytest.mark.parametrize("L", [1, 3, 17, 60])
def test_identical_sequences(L):
    rng = random.Random(L)
    s = rand_seq(rng, L, "ACGT")
    for h0 in (1, 9, 40):
        res, cells = oracle.extend_one_bwa(s, s, h0, BwaScoring(zdrop=100))
        assert res == (h0 + L, L, L, h0 + L, L, 0, 0)


@pytest.mark.parametrize("k,end_bonus,found", [(11, 12, True), (12, 13, True), (12, 12, False),
                                               (6, 7, True), (7, 7, False)])
def test_narrowing_threshold(k, end_bonus, found):
    # q = ACTT, t = G^k ACTT: the best end-to-end path deletes the k G's from
    # the seed (cost 6 + k) and matches the four bases, h0 - 2 - k, ending in
    # the last row.  Every other path to the last query column has a mismatch
    # (-30) or a second gap: at most h0 - 39 in row 0, h0 - 10 - k in the
    # rows that end with an insertion.  With narrowing the band is
    # (4 + end_bonus - 6) // 1 + 1 = end_bonus - 1, and the path needs the
    # cell (k, 0), i.e. k <= band.
    h0 = 100
    q, t = "ACTT", "G" * k + "ACTT"
    sc = BwaScoring(match=1, mismatch=-30, o_del=6, e_del=1, o_ins=6, e_ins=1, w=100, zdrop=0,
                    end_bonus=end_bonus)
    band = end_bonus - 1
    assert oracle.bwa_band(sc, 4) == band
    res, _ = oracle.extend_one_bwa(q, t, h0, sc)
    assert res[0:3] == (h0, 0, 0)
    if found:
        assert res[3:5] == (h0 - 2 - k, k + 4)
    else:
        assert res[3] < h0 - 2 - k
        assert res[4] <= 3 + band + 1          # the last row that reaches column 3
    # without narrowing the path is always found
    res_wide, _ = oracle.extend_one_bwa(q, t, h0, sc, flags=BWA_NO_NARROW)
    assert res_wide[3:5] == (h0 - 2 - k, k + 4)


def test_narrowing_small_gain():
    # gain below the opening cost: the band collapses to 1
    sc = BwaScoring(o_ins=30, o_del=30, end_bonus=0, w=50)
    assert oracle.bwa_band(sc, 10) == 1
    assert oracle.bwa_band(BwaScoring(w=3, end_bonus=100), 10) == 3


@pytest.mark.parametrize("zdrop,cells", [(1, 2), (2, 6), (0, 6)])
def test_zdrop_deletion_direction(zdrop, cells):
    # q = A, t = A C^5: best 11 at (0,0); every later row peaks on the deletion
    # run in column 0 at 9 - i, so drop = 11 - (9 - i) - i*e_del = 2 with the
    # deletion extension e_del = 1 (the insertion extension 4 would never stop)
    sc = BwaScoring(match=1, mismatch=-4, o_del=2, e_del=1, o_ins=2, e_ins=4, w=10, zdrop=zdrop,
                    end_bonus=50)
    tr = oracle.extend_one_bwa("A", "ACCCCC", 10, sc, trace=True)
    assert tr.result == (11, 1, 1, 11, 1, 0, 0)
    assert tr.cells == cells
    assert tr.row_m.tolist() == [11, 8, 7, 6, 5, 4][:cells]


def test_insertion_then_deletion_is_not_a_path():
    # q = A G^n, t = C G^n, mismatch -20: the first bases must be mismatched
    # (-20) or gapped.  t's C can only be deleted straight from the seed (no
    # match step comes before it) and q's A only inserted straight from the
    # seed, so gapping both needs an insertion touching a deletion (-7 - 7):
    # the default definition takes it, this variant pays the mismatch.
    n, h0 = 30, 30
    q, t = "A" + "G" * n, "C" + "G" * n
    dflt, _ = oracle.extend_one(q, t, h0, Scoring(match=1, mismatch=-20, w=100, zdrop=0))
    bwa, _ = oracle.extend_one_bwa(q, t, h0, BwaScoring(match=1, mismatch=-20, w=100, zdrop=0))
    assert dflt[:5] == (h0 - 14 + n, n + 1, n + 1, h0 - 14 + n, n + 1)
    assert bwa[:5] == (h0 - 20 + n, n + 1, n + 1, h0 - 20 + n, n + 1)


def test_degenerate_inputs():
    sc = BwaScoring()
    assert oracle.extend_one_bwa("", "ACGT", 7, sc) == ((7, 0, 0, 7, 0, 0, 0), 0)
    assert oracle.extend_one_bwa("ACGT", "", 7, sc) == ((7, 0, 0, -1, 0, 0, 0), 0)


def test_scoring_checks():
    assert oracle.check_bwa_scoring(BwaScoring())
    for bad in (dict(e_del=0), dict(e_ins=0), dict(match=0), dict(mismatch=1), dict(o_del=-1),
                dict(w=-1), dict(end_bonus=-1), dict(n_score=3)):
        assert not oracle.check_bwa_scoring(BwaScoring(**bad)), bad


# ------------------------------------------------------------------ invariants
def test_trimming_and_move_rules_only_remove_paths():
    rng = random.Random(5)
    for case in range(150):
        ql, tl = rng.randint(1, 30), rng.randint(1, 40)
        q = rand_seq(rng, ql, "ACGT")
        t = q[:rng.randint(0, ql)] + rand_seq(rng, max(0, tl - ql), "ACGT")
        t = t[:tl] if t else rand_seq(rng, tl, "ACGT")
        h0 = rng.randint(1, 40)
        sc = BwaScoring(w=rng.choice([3, 10, 100]), zdrop=0, end_bonus=rng.choice([0, 5, 100]))
        trim = oracle.extend_one_bwa(q, t, h0, sc, trace=True)
        full = oracle.extend_one_bwa(q, t, h0, sc, flags=BWA_NO_TRIM, trace=True)
        n = len(trim.row_m)
        assert np.all(trim.H[:n + 1] <= full.H[:n + 1])
        assert trim.result[0] <= full.result[0]
        assert trim.cells <= full.cells
        w = oracle.bwa_band(sc, ql)
        for i in range(n):
            assert max(0, i - w) <= trim.row_beg[i] and trim.row_end[i] <= min(ql, i + w + 1)
        res = trim.result
        assert res[0] >= h0 and 0 <= res[1] <= ql and 0 <= res[2] <= tl
        if res[1] > 0:
            assert abs(res[1] - res[2]) <= w
        # the move rules: no more paths than the default definition with the
        # same penalties (both switches off, no z-drop, same band)
        d = oracle.extend_one(q, t, h0, Scoring(gap_open=6, gap_extend=1, w=w, zdrop=0),
                              trace=True)
        nb = oracle.extend_one_bwa(q, t, h0, sc, flags=BWA_NO_TRIM | BWA_NO_NARROW | 0,
                                   trace=True) if w == sc.w else full
        m = min(len(nb.row_m), len(d.row_m))
        assert np.all(nb.H[1:m + 1, 1:] <= d.H[1:m + 1, 1:])


def test_batch_runner_width_limit_and_checks():
    # the batch runner rejects pairs whose rows would exceed 8,192 columns
    # (min(qlen, 2w'+1)), invalid offsets and h0 < 1, and agrees with the
    # single-pair call on the rest
    rng = np.random.default_rng(11)
    qs = [rng.integers(0, 4, 9000), rng.integers(0, 4, 8192), rng.integers(0, 4, 40),
          rng.integers(0, 4, 30)]
    ts = [rng.integers(0, 4, 40), rng.integers(0, 4, 30), rng.integers(0, 4, 60),
          rng.integers(0, 4, 30)]
    h0 = np.array([20, 20, 20, 0], np.int32)
    ql = np.array([q.size for q in qs], np.int32)
    tl = np.array([t.size for t in ts], np.int32)
    qo = np.concatenate([[0], np.cumsum(ql[:-1])]).astype(np.int64)
    to = np.concatenate([[0], np.cumsum(tl[:-1])]).astype(np.int64)
    q_seq = np.concatenate(qs).astype(np.uint8)
    t_seq = np.concatenate(ts).astype(np.uint8)
    sc = BwaScoring(w=5000, zdrop=0)
    out, cells = oracle.extend_batch_bwa(q_seq, qo, ql, t_seq, to, tl, h0, sc, nthreads=2)
    assert out[0, 6] == 1 and cells[0] == 0          # 9,000 columns
    assert out[3, 6] == 1                             # h0 = 0
    for k in (1, 2):                                  # 8,192 columns is still accepted
        assert out[k, 6] == 0
        res, c = oracle.extend_one_bwa(qs[k], ts[k], 20, sc)
        assert tuple(out[k]) == res and cells[k] == c
    # with a narrow band the long query fits
    out2, _ = oracle.extend_batch_bwa(q_seq, qo, ql, t_seq, to, tl, h0, BwaScoring(w=100))
    assert out2[0, 6] == 0
    with pytest.raises(ValueError):
        oracle.extend_batch_bwa(q_seq, qo, ql, t_seq, to, tl, h0, BwaScoring(e_ins=0))
