"""Host-side check of how the BWA-MEM-compatible kernel splits a row.

The kernel (csrc/xt_bwa.cu) extends a pair with a group of G lanes, one row at a
time, computing only the row's live columns [beg, end): lane l takes k >= ceil(
(end - beg) / G) consecutive columns from beg + l*k.  The row above lives in a
buffer of G*K + 2 elements (x = H of column j, y = query code << 28 | F of
column j) at index j - o(r), o(r) = max(-1, r - w' - 1), with boundary elements
at columns beg - 1 and end.  This test replays that decomposition lane by lane
in Python (a model of the indexing, not the CUDA code) and checks it against
the oracle: every buffer index in range, no element read before it is written,
each column's query code carried with it, F words written while the row above is
still being read landing only on words their own lane has read, and the
oracle's result for several group sizes and for odd as well as exact column
counts per lane.
"""
import random

import numpy as np
import pytest

import oracle
from oracle import BwaScoring

K = 32  # most columns a lane computes in a row


def score(sc, ti, qc):
    if ti == 4 or qc == 4:
        return sc.n_score
    return sc.match if ti == qc else sc.mismatch


def extend_by_rows(q, t, h0, sc, G, odd, early_f=False):
    """Extend one pair the way the kernel's lanes do; returns the oracle's tuple."""
    qlen, tlen = len(q), len(t)
    w = oracle.bwa_band(sc, qlen)
    width = min(qlen, 2 * w + 1)
    cap = 64
    while cap < width:
        cap *= 2
    kmax = max(K, -(-cap // G))
    oe_ins, oe_del = sc.o_ins + sc.e_ins, sc.o_del + sc.e_del
    code = lambda j: min(q[j], 4) if j < qlen else 4
    buf = [None] * (cap + 2)

    def read(idx):
        assert 0 <= idx < len(buf) and buf[idx] is not None, idx
        return buf[idx]

    def write(idx, v):
        assert 0 <= idx < len(buf), idx
        buf[idx] = v

    origin = lambda r: max(-1, r - w - 1)
    end = min(qlen, w + 1)
    for u in range(end + 2):  # row -1
        j = u - 1
        x = h0
        if j >= 0:
            v = h0 - oe_ins - sc.e_ins * j
            x = v if (j < qlen and j + 1 <= w and v > 0) else 0
        write(u, (x, (code(j) if j >= 0 else 4) << 28))
    beg = 0
    best, bi, bj, max_off, gscore, gtle, cells = h0, -1, -1, 0, -1, 0, 0
    for i in range(tlen):
        if beg >= end:
            break
        o_up, o_row = origin(i - 1), origin(i)
        ti = min(t[i], 4)
        kq = -(-(end - beg) // G)
        if odd:
            kq = min(kq | 1, kmax)
        assert kq <= kmax
        lanes = []
        shifted = o_row != o_up
        y_readers = {}  # buffer index -> lane that reads its y word in pass 1
        early = []      # (lane, index, y) written during pass 1
        for lane in range(G):  # pass 1: reads of the row above, early F words
            first = beg + lane * kq
            cnt = max(0, min(kq, end - first))
            Y, Hp, Yn = 0, [], []
            if cnt:
                Dn = read(first - 1 - o_up)[0]
                for kk in range(cnt):
                    x, y = read(first + kk - o_up)
                    y_readers[first + kk - o_up] = lane
                    D, Dn = Dn, x
                    c, F = y >> 28, y & ((1 << 28) - 1)
                    assert c == code(first + kk)
                    M = D + score(sc, ti, c) if D > 0 else 0
                    Fn = max(M - oe_del, F - sc.e_del, 0)
                    Yn.append((c << 28) | Fn)
                    Hp.append(max(M, Y, F))
                    Y = max(M - oe_ins, Y - sc.e_ins, 0)
                    if early_f and (kk > 0 or not shifted):
                        early.append((lane, first + kk - o_row, Yn[-1]))
            lanes.append((first, cnt, Y, Hp, Yn))
        # an F word written during pass 1 lands on a y word that only its own
        # lane reads, and that lane has read it already (an earlier or the
        # same column); x words are not written before the barrier
        for lane, idx, y in early:
            assert y_readers.get(idx, lane) == lane, (i, lane, idx)
            assert 0 <= idx < len(buf)
            buf[idx] = (buf[idx][0] if buf[idx] is not None else None, y)
        decay = sc.e_ins * kq
        best_lane = (-1, 0)
        dead = []
        for lane, (first, cnt, _, Hp, Yn) in enumerate(lanes):  # pass 2: writes
            ex = max((lanes[u][2] + decay * u for u in range(lane)), default=None)
            E = 0 if lane == 0 else max(0, ex - decay * (lane - 1))
            dm = 0
            for kk in range(cnt):
                H = max(Hp[kk], E)
                E -= sc.e_ins
                if (H, first + kk) > best_lane:
                    best_lane = (H, first + kk)
                dm |= (H == 0) << kk
                if early_f and (kk > 0 or not shifted):
                    assert buf[first + kk - o_row][1] == Yn[kk]
                write(first + kk - o_row, (H, Yn[kk]))
            dead.append(dm)
        hb = max(0, h0 - oe_del - sc.e_del * i) if (beg == 0 and i + 1 <= w) else 0
        write(beg - 1 - o_row, (hb, 4 << 28))
        write(end - o_row, (0, code(end) << 28))
        m, mj = best_lane
        if end == qlen:
            gv = read(qlen - 1 - o_row)[0]
            if gv >= gscore:
                gscore, gtle = gv, i + 1
        if m == 0:
            break
        cells += end - beg
        if m > best:
            best, bi, bj = m, i, mj
            max_off = max(max_off, abs(mj - i))
        elif sc.zdrop > 0:
            di, dj = i - bi, mj - bj
            drop = best - m - ((di - dj) * sc.e_del if di > dj else (dj - di) * sc.e_ins)
            if drop > sc.zdrop:
                break
        ll, fl = -1, None
        for (first, cnt, _, _, _), dm in zip(lanes, dead):
            for kk in range(cnt):
                if not dm >> kk & 1:
                    j = first + kk
                    ll = max(ll, j)
                    fl = j if fl is None else min(fl, j)
        beg = max(fl, i + 1 - w)
        end = min(ll + 2, i + w + 2, qlen)
    return (best, bj + 1, bi + 1, gscore, gtle, max_off, 0), cells


SCORINGS = [
    BwaScoring(),
    BwaScoring(o_del=2, e_del=3, o_ins=5, e_ins=1, w=10, zdrop=20, end_bonus=0),
    BwaScoring(match=2, mismatch=-3, o_del=0, e_del=2, o_ins=1, e_ins=4, w=3, zdrop=0,
               end_bonus=100, n_score=-2),
    BwaScoring(w=0, zdrop=5),
    BwaScoring(w=1000, zdrop=0, end_bonus=1000),
]


def random_pair(rng):
    ql, tl = rng.randint(1, 90), rng.randint(1, 120)
    q = [rng.randint(0, 3) for _ in range(ql)]
    if rng.random() < 0.6:
        t = q[:tl] + [rng.randint(0, 3) for _ in range(max(0, tl - ql))]
        t = [x if rng.random() > 0.05 else rng.randint(0, 5) for x in t]
    else:
        t = [rng.randint(0, 4) for _ in range(tl)]
    q = [x if rng.random() > 0.03 else 4 for x in q]
    return q, t, rng.choice([1, 5, 20, rng.randint(1, 80)])


@pytest.mark.parametrize("si", range(len(SCORINGS)))
def test_row_split_matches_oracle(si):
    sc = SCORINGS[si]
    rng = random.Random(900 + si)
    for _ in range(40):
        q, t, h0 = random_pair(rng)
        want = oracle.extend_one_bwa(np.array(q, np.uint8), np.array(t, np.uint8), h0, sc)
        for G, odd, early_f in ((2, True, False), (8, True, True), (3, False, True),
                                (64, True, False)):
            got = extend_by_rows(q, t, h0, sc, G, odd, early_f)
            assert got == want, (si, G, odd, early_f, q, t, h0)


def test_row_split_long_pair_full_width_rows():
    # unbanded equal-length pair: rows as wide as the class, 32 columns per lane
    rng = random.Random(5)
    q = [rng.randint(0, 3) for _ in range(250)]
    t = [x if rng.random() > 0.03 else rng.randint(0, 3) for x in q]
    sc = BwaScoring(w=250, zdrop=0)
    want = oracle.extend_one_bwa(np.array(q, np.uint8), np.array(t, np.uint8), 30, sc)
    assert extend_by_rows(q, t, 30, sc, 8, True) == want
