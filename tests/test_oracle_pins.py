"""Pins for the CPU oracle, each independent of the oracle's own code.

* hand-worked tables (tests/golden/handworked_*.json): every H/E/F value of
  small extensions, derived on paper from Eq. 1 (Sec. II-A) under the
  seed-extension reading;
* closed forms: identical sequences, identical prefix, all-mismatch, a single
  deletion;
* independent path enumeration: every alignment path from the seed is scored
  move by move (no recurrence), which fixes every H/E/F value of tiny
  extensions, and from them score, positions, gscore and cells;
* invariants: monotonicity in zdrop and w, output ranges.
"""
import json
import os
import random

import numpy as np
import pytest

import oracle
from oracle import Scoring

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CODES = {"A": 0, "C": 1, "G": 2, "T": 3, "N": 4}


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def scoring_of(d, **kw):
    d = dict(d)
    d.update(kw)
    return Scoring(**d)


# ---------------------------------------------------------------- hand-worked
@pytest.mark.parametrize("name", ["handworked_identical_3x3.json", "handworked_anchoring_3x3.json",
                                  "handworked_band_n_3x4.json"])
def test_handworked_tables(name):
    g = load(name)
    tr = oracle.extend_one(g["q"], g["t"], g["h0"], scoring_of(g["scoring"]), trace=True)
    assert tr.H.tolist() == g["H"]
    assert tr.E.tolist() == g["E"]
    assert tr.F.tolist() == g["F"]
    assert tr.row_m.tolist() == g["row_m"]
    assert tr.row_mj.tolist() == g["row_mj"]
    assert list(tr.result) == g["result"]
    assert tr.cells == g["cells"]


def test_handworked_zdrop_tail():
    g = load("handworked_zdrop_tail.json")
    for case in g["cases"]:
        sc = scoring_of(g["scoring"], zdrop=case["zdrop"])
        tr = oracle.extend_one(g["q"], g["t"], g["h0"], sc, trace=True)
        assert list(tr.result) == case["result"], case
        assert tr.cells == case["cells"], case
        n_rows = len(g["t"]) if case["stop_row"] is None else case["stop_row"] + 1
        assert len(tr.row_m) == n_rows
        assert tr.row_m.tolist() == g["row_m_prefix"][:n_rows]
        assert tr.row_mj.tolist() == g["row_mj_prefix"][:n_rows]


# --------------------------------------------------------------- closed forms
def rand_seq(rng, n, alphabet="ACGT"):
    return "".join(rng.choice(alphabet) for _ in range(n))


@pytest.mark.parametrize("L", [1, 2, 7, 40, 150])
def test_identical_sequences(L):
    rng = random.Random(L)
    s = rand_seq(rng, L)
    for h0 in (1, 5, 37):
        res, cells = oracle.extend_one(s, s, h0, Scoring(w=100, zdrop=100))
        assert res == (h0 + L, L, L, h0 + L, L, 0, 0)
        # every row is live and the band covers min(L, i + 101) - max(0, i - 100) columns
        assert cells == sum(min(L, i + 101) - max(0, i - 100) for i in range(L))


def test_identical_prefix_longer_target():
    rng = random.Random(7)
    s = rand_seq(rng, 30)
    t = s + rand_seq(rng, 9)
    res, _ = oracle.extend_one(s, t, 25, Scoring(w=100, zdrop=100))
    assert res[:5] == (25 + 30, 30, 30, 25 + 30, 30)


def test_match_score_scales():
    s = "ACGTTGCAAC"
    res, _ = oracle.extend_one(s, s, 4, Scoring(match=3, w=20, zdrop=0))
    assert res[:5] == (4 + 3 * len(s), len(s), len(s), 4 + 3 * len(s), len(s))


def test_all_mismatch_small_h0():
    res, cells = oracle.extend_one("AAAA", "CCCC", 3, Scoring())
    assert res == (3, 0, 0, -1, 0, 0, 0) and cells == 0


def test_all_mismatch_single_cell_gscore():
    # one mismatching cell with h0 >= 5: the local best stays at the seed, but
    # the end-to-end alignment exists with score h0 - 4.
    for h0 in (5, 9, 30):
        res, cells = oracle.extend_one("A", "C", h0, Scoring())
        assert res == (h0, 0, 0, h0 - 4, 1, 0, 0)
        assert cells == 1


def test_single_deletion_closed_form():
    # q = P + S2, t = P + X + S2: the best alignment deletes X once (cost
    # alpha = gap_open + gap_extend = 7).  P and S2 have no equal neighbours and
    # X differs from both flanks, so no other one-gap path matches as many bases.
    P, X, S2 = "ACGTCA", "G", "TCAGTACG"
    q, t = P + S2, P + X + S2
    L = len(q)
    res, cells = oracle.extend_one(q, t, 20, Scoring(w=100, zdrop=100))
    assert res == (20 + L - 7, L, L + 1, 20 + L - 7, L + 1, 1, 0)
    assert cells == len(t) * len(q)


def test_degenerate_lengths():
    assert oracle.extend_one("", "ACGT", 7, Scoring()) == ((7, 0, 0, 7, 0, 0, 0), 0)
    assert oracle.extend_one("ACGT", "", 7, Scoring()) == ((7, 0, 0, -1, 0, 0, 0), 0)
    assert oracle.extend_one("", "", 7, Scoring()) == ((7, 0, 0, 7, 0, 0, 0), 0)


def test_band_zero_is_diagonal_only():
    # w = 0: only the diagonal is in band, so the extension is ungapped.
    q, t = "ACGTAC", "ACCTAC"
    res, cells = oracle.extend_one(q, t, 10, Scoring(w=0, zdrop=0))
    # running diagonal scores 11, 12, 8, 9, 10, 11: best 12 at (1,1), end 11
    assert res == (12, 2, 2, 11, 6, 0, 0)
    assert cells == 6


# ----------------------------------------------------------- path enumeration
def enumerate_paths(q, t, h0, sc: Scoring):
    """Score every alignment path that leaves the seed (cell (-1,-1)) move by
    move and keep, for each interior cell, the best score of a path ending
    there with a diagonal step (M), an insertion step (E) or a deletion step (F).
    A path is kept only while all cells it visits are in band and every prefix
    score stays > 0.  Gap runs cost alpha for the first base and beta after."""
    alpha, beta = sc.gap_open + sc.gap_extend, sc.gap_extend
    ql, tl = len(q), len(t)
    best = {}  # (r, c, kind) -> max score

    def S(i, j):
        a, b = CODES[t[i]], CODES[q[j]]
        if a >= 4 or b >= 4:
            return sc.n_score
        return sc.match if a == b else sc.mismatch

    def inb(r, c):
        return abs(r - c) <= sc.w

    def walk(r, c, s, last):
        for kind, dr, dc in (("M", 1, 1), ("E", 0, 1), ("F", 1, 0)):
            nr, nc = r + dr, c + dc
            if nr >= tl or nc >= ql or not inb(nr, nc):
                continue
            if kind == "M":
                ns = s + S(nr, nc)
            elif kind == "E":
                ns = s - (beta if last == "E" else alpha)
            else:
                ns = s - (beta if last == "F" else alpha)
            if ns <= 0:
                continue
            key = (nr, nc, kind)
            if best.get(key, -10 ** 9) < ns:
                best[key] = ns
            walk(nr, nc, ns, kind)

    walk(-1, -1, h0, "M")
    H = np.zeros((tl, ql), np.int64)
    E = np.zeros((tl, ql), np.int64)
    F = np.zeros((tl, ql), np.int64)
    for (r, c, kind), v in best.items():
        if r < 0 or c < 0:
            continue
        H[r, c] = max(H[r, c], v)
        if kind == "E":
            E[r, c] = max(E[r, c], v)
        if kind == "F":
            F[r, c] = max(F[r, c], v)
    return H, E, F


def outputs_from_H(H, q, t, h0, sc):
    """score/positions/gscore/max_off/cells from an interior H matrix: rows in
    order, largest column within a row, strictly greater to move the best.
    With sc.zdrop > 0 a row that does not raise the best ends the extension
    when best - m - |(i - bi) - (mj - bj)| * beta > zdrop, after that row's
    gscore update; rows after it count for nothing (Q6).  H is the full
    matrix, so the cut-off is applied here and nowhere else."""
    beta = sc.gap_extend
    tl, ql = H.shape
    if ql == 0:
        return (h0, 0, 0, h0, 0, 0, 0), 0
    if tl == 0:
        return (h0, 0, 0, -1, 0, 0, 0), 0
    best, bi, bj, max_off, g, gtle, last_live = h0, -1, -1, 0, -1, 0, -1
    for i in range(tl):
        cols = [j for j in range(ql) if abs(i - j) <= sc.w]
        m, mj = 0, -1
        for j in cols:
            if H[i, j] >= m:
                m, mj = int(H[i, j]), j
            if H[i, j] > 0:
                last_live = i
        if abs(i - (ql - 1)) <= sc.w and H[i, ql - 1] > 0 and H[i, ql - 1] > g:
            g, gtle = int(H[i, ql - 1]), i + 1
        if m > best:
            best, bi, bj = m, i, mj
            max_off = max(max_off, abs(mj - i))
        elif sc.zdrop > 0:
            d = (i - bi) - (mj - bj)
            if best - m - abs(d) * beta > sc.zdrop:
                break
    cells = sum(len([j for j in range(ql) if abs(i - j) <= sc.w]) for i in range(last_live + 1))
    return (best, bj + 1, bi + 1, g, gtle, max_off, 0), cells


def random_case(rng):
    ql, tl = rng.randint(0, 5), rng.randint(0, 5)
    alph = "ACGT" if rng.random() < 0.6 else "ACGTN"
    q, t = rand_seq(rng, ql, alph), rand_seq(rng, tl, alph)
    if rng.random() < 0.3 and ql and tl:
        t = q[: min(ql, tl)] + t[min(ql, tl):]
    sc = Scoring(match=rng.randint(1, 3), mismatch=-rng.randint(0, 5), gap_open=rng.randint(0, 6),
                 gap_extend=rng.randint(0, 3), w=rng.choice([0, 1, 2, 3, 10]), zdrop=0,
                 n_score=-rng.randint(0, 3))
    return q, t, rng.randint(1, 14), sc


def test_path_enumeration_fixes_every_cell():
    rng = random.Random(2301)
    n_nontrivial = 0
    for _ in range(400):
        q, t, h0, sc = random_case(rng)
        tr = oracle.extend_one(q, t, h0, sc, trace=True)
        H, E, F = enumerate_paths(q, t, h0, sc)
        if len(q) and len(t):
            assert tr.H[1:, 1:].tolist() == H.tolist(), (q, t, h0, sc)
            assert tr.E[1:, 1:].tolist() == E.tolist(), (q, t, h0, sc)
            assert tr.F[1:, 1:].tolist() == F.tolist(), (q, t, h0, sc)
            n_nontrivial += int(H.max() > 0)
        res, cells = outputs_from_H(H, q, t, h0, sc)
        assert tr.result == res, (q, t, h0, sc)
        assert tr.cells == cells, (q, t, h0, sc)
    assert n_nontrivial > 100


def test_path_enumeration_fixes_zdrop():
    """Z-drop pinned independently of the oracle: the enumerated (full) H of
    each random tiny case, cut off in row order by the rule above, against
    the oracle run with the same cutoff, on every field and on cells."""
    rng = random.Random(2302)
    n_cut = 0
    for _ in range(400):
        q, t, h0, sc0 = random_case(rng)
        H, _, _ = enumerate_paths(q, t, h0, sc0)
        full, full_cells = outputs_from_H(H, q, t, h0, sc0)
        for z in (1, 3, 8):
            sc = Scoring(match=sc0.match, mismatch=sc0.mismatch, gap_open=sc0.gap_open,
                         gap_extend=sc0.gap_extend, w=sc0.w, zdrop=z, n_score=sc0.n_score)
            res, cells = oracle.extend_one(q, t, h0, sc)
            want, want_cells = outputs_from_H(H, q, t, h0, sc)
            assert res == want, (q, t, h0, sc)
            assert cells == want_cells, (q, t, h0, sc)
            n_cut += int((want, want_cells) != (full, full_cells))
    # the cutoff changed the outputs of a good share of the cases
    assert n_cut > 50, n_cut


def test_boundary_runs_match_enumeration():
    # row -1 / column -1 values are pure gap runs from the seed
    sc = Scoring(w=3, zdrop=0)
    tr = oracle.extend_one("ACGTA", "ACGTA", 12, sc, trace=True)
    alpha, beta = 7, 1
    for c in range(5):
        want = max(0, 12 - alpha - beta * c) if c + 1 <= sc.w else 0
        assert tr.H[0, c + 1] == want and tr.E[0, c + 1] == want and tr.F[0, c + 1] == 0
    for r in range(5):
        want = max(0, 12 - alpha - beta * r) if r + 1 <= sc.w else 0
        assert tr.H[r + 1, 0] == want and tr.F[r + 1, 0] == want and tr.E[r + 1, 0] == 0


# ----------------------------------------------------------------- invariants
def batch_of(rng, n, qmax, extra):
    qs, ts = [], []
    for _ in range(n):
        ql = rng.randint(0, qmax)
        q = rand_seq(rng, ql, "ACGTACGTACGTN")
        t = list(q)
        for k in range(len(t)):
            if rng.random() < 0.08:
                t[k] = rng.choice("ACGT")
        t = "".join(t) + rand_seq(rng, rng.randint(0, extra))
        if rng.random() < 0.1:
            t = rand_seq(rng, len(t))
        qs.append(q)
        ts.append(t)
    return qs, ts


def pack(seqs):
    off = np.zeros(len(seqs), np.int64)
    lens = np.array([len(s) for s in seqs], np.int32)
    off[1:] = np.cumsum(lens)[:-1] if len(seqs) > 1 else off[1:]
    data = np.array([CODES[ch] for s in seqs for ch in s], np.uint8)
    return data, off, lens


def test_monotone_in_zdrop_and_band():
    rng = random.Random(11)
    qs, ts = batch_of(rng, 300, 60, 30)
    qd, qo, qlen = pack(qs)
    td, to, tlen = pack(ts)
    h0 = np.array([rng.randint(1, 40) for _ in qs], np.int32)
    prev = None
    for z in (1, 5, 20, 60, 0):  # 0 disables z-drop: the largest effective cutoff
        out, _ = oracle.extend_batch(qd, qo, qlen, td, to, tlen, h0, Scoring(w=30, zdrop=z))
        if prev is not None:
            assert np.all(out[:, 0] >= prev[:, 0])
        prev = out
    prev = None
    for w in (0, 2, 8, 30, 200):
        out, _ = oracle.extend_batch(qd, qo, qlen, td, to, tlen, h0, Scoring(w=w, zdrop=0))
        if prev is not None:
            assert np.all(out[:, 0] >= prev[:, 0])
        prev = out


def test_output_ranges():
    rng = random.Random(12)
    qs, ts = batch_of(rng, 400, 80, 40)
    qd, qo, qlen = pack(qs)
    td, to, tlen = pack(ts)
    h0 = np.array([rng.randint(1, 60) for _ in qs], np.int32)
    for sc in (Scoring(w=10, zdrop=20), Scoring(w=100, zdrop=100), Scoring(w=3, zdrop=0)):
        out, cells = oracle.extend_batch(qd, qo, qlen, td, to, tlen, h0, sc)
        score, qle, tle, gscore, gtle, max_off, status = out.T
        assert np.all(status == 0)
        assert np.all(score >= h0)
        assert np.all((qle >= 0) & (qle <= qlen) & (tle >= 0) & (tle <= tlen))
        assert np.all(np.abs(qle - tle) <= sc.w)
        assert np.all(gscore <= score)
        assert np.all((gscore == -1) | (gscore > 0) | (qlen == 0))
        assert np.all(max_off <= sc.w)
        assert np.all((cells >= 0) & (cells <= qlen.astype(np.int64) * tlen))


def test_band_beyond_every_pair_changes_nothing():
    """An invariant of the static band (Q5), not a pin: once w exceeds every
    pair's lengths no cell leaves the band, so any larger w gives the same
    results.  (The band itself is pinned by path enumeration with w in
    {0, 1, 2, 3, 10} and by the hand-worked band table.)"""
    rng = random.Random(13)
    qs, ts = batch_of(rng, 200, 40, 20)
    qd, qo, qlen = pack(qs)
    td, to, tlen = pack(ts)
    h0 = np.array([rng.randint(1, 60) for _ in qs], np.int32)
    a, ca = oracle.extend_batch(qd, qo, qlen, td, to, tlen, h0, Scoring(w=100, zdrop=0))
    b, cb = oracle.extend_batch(qd, qo, qlen, td, to, tlen, h0, Scoring(w=10 ** 6, zdrop=0))
    assert np.array_equal(a, b) and np.array_equal(ca, cb)


def test_batch_equals_single_and_threads():
    rng = random.Random(14)
    qs, ts = batch_of(rng, 120, 50, 30)
    qd, qo, qlen = pack(qs)
    td, to, tlen = pack(ts)
    h0 = np.array([rng.randint(1, 60) for _ in qs], np.int32)
    sc = Scoring(w=20, zdrop=30)
    o1, c1 = oracle.extend_batch(qd, qo, qlen, td, to, tlen, h0, sc, nthreads=1)
    o4, c4 = oracle.extend_batch(qd, qo, qlen, td, to, tlen, h0, sc, nthreads=4)
    assert np.array_equal(o1, o4) and np.array_equal(c1, c4)
    for k in range(len(qs)):
        res, cells = oracle.extend_one(qs[k], ts[k], int(h0[k]), sc)
        assert tuple(o1[k]) == res and c1[k] == cells


def test_invalid_pairs_and_scoring():
    qd, qo, qlen = pack(["ACGT", "ACG", "AC"])
    td, to, tlen = pack(["ACGT", "ACG", "AC"])
    h0 = np.array([5, 0, 5], np.int32)           # h0 < 1 is rejected per pair
    qo2 = qo.copy()
    qo2[2] = 100                                 # out of the buffer
    out, cells = oracle.extend_batch(qd, qo2, qlen, td, to, tlen, h0, Scoring())
    assert out[0, 6] == 0 and out[1, 6] == 1 and out[2, 6] == 1
    assert out[1, :6].tolist() == [0] * 6 and cells[1] == 0
    with pytest.raises(ValueError):
        oracle.extend_batch(qd, qo, qlen, td, to, tlen, h0, Scoring(match=0))
    assert not oracle.check_scoring(Scoring(mismatch=1))
    assert oracle.check_scoring(Scoring())
