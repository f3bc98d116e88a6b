"""Both-direction extension of seeds (xt_extend_seeds): each side equals the
CPU oracle on that side's sequences -- the reversed prefixes from the seed's
score, then the suffixes from the left side's best."""
import numpy as np
import pytest

from paper_2301_09310_gb300 import synth
from paper_2301_09310_gb300.synth import Batch, ScoringParams

from tests.gpu_util import assert_same, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    import paper_2301_09310_gb300 as xt
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = xt.Context(0)
    yield c
    c.close()


def _batch(qs, ts, h0):
    ql = np.array([q.size for q in qs], np.int32)
    tl = np.array([t.size for t in ts], np.int32)
    qo = np.zeros(len(qs), np.int64)
    to = np.zeros(len(ts), np.int64)
    if len(qs) > 1:
        qo[1:] = np.cumsum(ql[:-1])
        to[1:] = np.cumsum(tl[:-1])
    cat = lambda xs: np.concatenate(xs).astype(np.uint8) if xs else np.zeros(0, np.uint8)  # noqa: E731
    return Batch(cat(qs), qo, ql, cat(ts), to, tl, np.asarray(h0, np.int32))


def expected(b, q_beg, t_beg, seed_len, h0, sc):
    """The oracle on each side, pair by pair (invalid seeds: XT_EINVAL)."""
    n = b.n
    ok = np.zeros(n, bool)
    lq, lt, rq, rt = [], [], [], []
    for k in range(n):
        qo, to, ql, tl = int(b.q_off[k]), int(b.t_off[k]), int(b.q_len[k]), int(b.t_len[k])
        qb, tb, sl = int(q_beg[k]), int(t_beg[k]), int(seed_len[k])
        valid = (ql >= 0 and tl >= 0 and qo >= 0 and to >= 0 and qo + ql <= b.q_seq.size
                 and to + tl <= b.t_seq.size and qb >= 0 and tb >= 0 and sl >= 0
                 and qb + sl <= ql and tb + sl <= tl)
        ok[k] = valid
        q = b.q_seq[qo:qo + ql] if valid else np.zeros(0, np.uint8)
        t = b.t_seq[to:to + tl] if valid else np.zeros(0, np.uint8)
        lq.append(q[:qb][::-1] if valid else q)
        lt.append(t[:tb][::-1] if valid else t)
        rq.append(q[qb + sl:] if valid else q)
        rt.append(t[tb + sl:] if valid else t)
    lo, lc = run_oracle(_batch(lq, lt, h0), sc)
    rh0 = np.where(lo[:, 6] == 0, lo[:, 0], h0).astype(np.int32)
    ro, rc = run_oracle(_batch(rq, rt, rh0), sc)
    bad = ~ok
    for o, c in ((lo, lc), (ro, rc)):
        o[bad] = 0
        o[bad, 6] = 1
        c[bad] = 0
    return (lo, lc), (ro, rc)


def make_seeds(b, rng, per_pair=3, seed_len=19):
    """Several seeds per pair (the pairs' sequences are shared by their seeds)."""
    idx, qb, tb, sl = [], [], [], []
    for k in range(b.n):
        ql, tl = int(b.q_len[k]), int(b.t_len[k])
        for _ in range(per_pair):
            L = min(seed_len, ql, tl)
            q0 = int(rng.integers(0, ql - L + 1))
            idx.append(k)
            qb.append(q0)
            tb.append(min(q0, tl - L))
            sl.append(L)
    idx = np.asarray(idx)
    seeds = Batch(b.q_seq, b.q_off[idx].copy(), b.q_len[idx].copy(), b.t_seq,
                  b.t_off[idx].copy(), b.t_len[idx].copy(), np.asarray(sl, np.int32) * 1)
    return seeds, np.asarray(qb, np.int32), np.asarray(tb, np.int32), np.asarray(sl, np.int32)


def run_seeds(ctx, b, q_beg, t_beg, seed_len, h0, sc):
    import torch
    dev = torch.device("cuda", ctx.device)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    left, right, lc, rc = ctx.extend_seeds(T(b.q_seq), T(b.q_off), T(b.q_len), T(b.t_seq),
                                           T(b.t_off), T(b.t_len), T(q_beg), T(t_beg),
                                           T(seed_len), T(h0), sc)
    torch.cuda.synchronize()
    return (left.cpu().numpy(), lc.cpu().numpy()), (right.cpu().numpy(), rc.cpu().numpy())


@pytest.mark.parametrize("name,sc", [("c3_mixed", None), ("c5_stream", None),
                                     ("c3_mixed", ScoringParams(w=10, zdrop=20))])
def test_seeds_match_oracle(ctx, name, sc):
    wl = synth.WORKLOADS[name]
    sc = sc or wl.scoring
    rng = np.random.default_rng(7)
    b = synth.generate(wl, n=1500, first=4000)
    keep = (b.q_len >= 1) & (b.t_len >= 1)
    b = b.take(np.nonzero(keep)[0])
    seeds, q_beg, t_beg, seed_len = make_seeds(b, rng)
    h0 = (seed_len * sc.match).astype(np.int32)
    # edge seeds: at the start of the pair, at its end, and outside it
    q_beg[0], t_beg[0] = 0, 0
    q_beg[1] = seeds.q_len[1] - seed_len[1]
    t_beg[1] = seeds.t_len[1] - seed_len[1]
    q_beg[2] = seeds.q_len[2] - seed_len[2] + 1      # one base too far
    t_beg[3] = -1
    seeds.q_off[4] = seeds.q_seq.size + 5            # pair outside its buffer
    want_l, want_r = expected(seeds, q_beg, t_beg, seed_len, h0, sc)
    got_l, got_r = run_seeds(ctx, seeds, q_beg, t_beg, seed_len, h0, sc)
    assert np.all(want_l[0][2:5, 6] == 1)
    assert_same(got_l, want_l, f"{name} left")
    assert_same(got_r, want_r, f"{name} right")


def test_seeds_empty_and_bad_args(ctx):
    import paper_2301_09310_gb300 as xt
    b = synth.generate(synth.WORKLOADS["c1_tiny"], n=10)
    z = np.zeros(0, np.int32)
    empty = Batch(b.q_seq, np.zeros(0, np.int64), z, b.t_seq, np.zeros(0, np.int64), z, z)
    got_l, got_r = run_seeds(ctx, empty, z, z, z, z, synth.WORKLOADS["c1_tiny"].scoring)
    assert got_l[0].shape == (0, 7) and got_r[0].shape == (0, 7)
    with pytest.raises(xt.XtError) as e:
        run_seeds(ctx, b, np.zeros(10, np.int32), np.zeros(10, np.int32),
                  np.full(10, 5, np.int32), np.full(10, 5, np.int32), ScoringParams(match=0))
    assert e.value.status == xt.XT_EINVAL


def test_seeds_packed4_equal_codes(ctx):
    # the 4-bit alphabet: both sides equal the call on base codes
    import paper_2301_09310_gb300 as xt
    wl = synth.WORKLOADS["c3_mixed"]
    rng = np.random.default_rng(9)
    b = synth.generate(wl, n=800, first=9000)
    keep = (b.q_len >= 1) & (b.t_len >= 1)
    b = b.take(np.nonzero(keep)[0])
    seeds, q_beg, t_beg, seed_len = make_seeds(b, rng)
    h0 = (seed_len * wl.scoring.match).astype(np.int32)
    want = run_seeds(ctx, seeds, q_beg, t_beg, seed_len, h0, wl.scoring)
    other = xt.Context(0)
    try:
        other.set_alphabet(xt.XT_ALPHABET_PACKED4)
        packed = Batch(xt.pack4(seeds.q_seq), seeds.q_off, seeds.q_len, xt.pack4(seeds.t_seq),
                       seeds.t_off, seeds.t_len, seeds.h0)
        got = run_seeds(other, packed, q_beg, t_beg, seed_len, h0, wl.scoring)
    finally:
        other.close()
    assert_same(got[0], want[0], "packed4 left")
    assert_same(got[1], want[1], "packed4 right")
