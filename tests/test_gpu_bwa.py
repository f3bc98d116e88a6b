"""The BWA-MEM-compatible extension (xt_extend_batch_bwa) against the CPU
oracle's variant, field by field and cell count by cell count: every width
class (64 to 8,192 columns, 2 to 256 lanes per pair), the paper-shaped
workloads, edge cases, the width limit, raw reads."""
import numpy as np
import pytest

import oracle
from paper_2301_09310_gb300 import synth
from paper_2301_09310_gb300.synth import BwaScoringParams

from tests.gpu_util import assert_same, batch_from_lists, fuzz_batch, to_dev

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


def run_gpu_bwa(ctx, b, sc):
    import torch
    out, cells = ctx.extend_bwa(*to_dev(b, torch.device("cuda", ctx.device)), sc)
    torch.cuda.synchronize()
    return out.cpu().numpy(), cells.cpu().numpy()


def run_oracle_bwa(b, sc):
    return oracle.extend_batch_bwa(b.q_seq, b.q_off, b.q_len, b.t_seq, b.t_off, b.t_len, b.h0,
                                   oracle.BwaScoring(*sc.as_tuple()))


FUZZ_SCORINGS = [
    BwaScoringParams(),
    BwaScoringParams(o_del=2, e_del=3, o_ins=5, e_ins=1, w=10, zdrop=20, end_bonus=0),
    BwaScoringParams(match=2, mismatch=-3, o_del=0, e_del=2, o_ins=1, e_ins=4, w=3, zdrop=0,
                     end_bonus=100, n_score=-2),
    BwaScoringParams(w=0, zdrop=5),
    BwaScoringParams(w=1000, zdrop=0, end_bonus=1000),
]


@pytest.mark.parametrize("si", range(len(FUZZ_SCORINGS)))
def test_fuzz_matches_oracle(ctx, si):
    sc = FUZZ_SCORINGS[si]
    b = fuzz_batch(300 + si, 4000, max_len=70, tail=40)
    assert_same(run_gpu_bwa(ctx, b, sc), run_oracle_bwa(b, sc), f"fuzz {sc}")


@pytest.mark.parametrize("name,n", [("c1_tiny", 1000), ("c2_short", 20000), ("c3_mixed", 20000),
                                    ("c5_stream", 20000), ("c4_long", 120)])
def test_workloads_match_oracle(ctx, name, n):
    wl = synth.WORKLOADS[name]
    b = synth.generate(wl, n=n, first=77)
    sc = BwaScoringParams.from_scoring(wl.scoring)
    want = run_oracle_bwa(b, sc)
    assert np.all(want[0][:, 6] == 0)
    assert_same(run_gpu_bwa(ctx, b, sc), want, name)


@pytest.mark.parametrize("L,n", [(64, 64), (200, 64), (700, 24), (1500, 8), (3000, 4),
                                 (4096, 3), (6000, 2)])
def test_every_group_size(ctx, L, n):
    # equal-length unbanded pairs: the row width is qlen, so L picks the class
    # (2 lanes up to 64 columns ... 256 lanes up to 8192; rows as wide as the
    # class, 32 columns per lane); some pairs ragged
    wl = synth.x2_workload(L, n_pairs=n)
    b = synth.generate(wl)
    b.q_len[::2] = np.maximum(1, b.q_len[::2] - np.arange(b.q_len[::2].size) * 7 % 50)
    for sc in (BwaScoringParams(w=L, zdrop=0), BwaScoringParams(w=L, zdrop=40, o_ins=3, e_ins=2)):
        assert_same(run_gpu_bwa(ctx, b, sc), run_oracle_bwa(b, sc), f"L={L} {sc}")


def test_large_scores_and_row_widths(ctx):
    # seed scores past 16 bits, and rows of 209..256 columns (8-lane groups,
    # up to 32 columns per lane)
    wl = synth.WORKLOADS["c3_mixed"]
    b = synth.generate(wl, n=6000, first=31)
    sc = BwaScoringParams.from_scoring(wl.scoring)
    big = synth.Batch(b.q_seq, b.q_off, b.q_len, b.t_seq, b.t_off, b.t_len, b.h0 + 16400)
    assert_same(run_gpu_bwa(ctx, big, sc), run_oracle_bwa(big, sc), "large h0")
    b2 = synth.generate(synth.x2_workload(250, n_pairs=40))
    sc2 = BwaScoringParams(w=250, zdrop=0)
    assert_same(run_gpu_bwa(ctx, b2, sc2), run_oracle_bwa(b2, sc2), "209..256 columns")


def test_width_limit_and_invalid_pairs(ctx):
    import paper_2301_09310_gb300 as xt
    rng = np.random.default_rng(3)
    qs = [rng.integers(0, 4, 9000), rng.integers(0, 4, 9000), rng.integers(0, 4, 50), [], [1, 2],
          rng.integers(0, 4, 30), rng.integers(0, 4, 8192)]
    ts = [rng.integers(0, 4, 60), rng.integers(0, 4, 60), rng.integers(0, 4, 80), [0, 1], [],
          rng.integers(0, 4, 30), rng.integers(0, 4, 12)]
    b = batch_from_lists(qs, ts, [30, 30, 30, 7, 9, 0, 25])
    wide = BwaScoringParams(w=5000, zdrop=0)      # 9000-base queries: rows of 9000 > 8192 columns
    b2 = batch_from_lists(qs[:1], ts[:1], [30])
    want = run_oracle_bwa(b, wide)
    assert want[0][0, 6] == xt.XT_EINVAL and want[0][1, 6] == xt.XT_EINVAL
    assert want[0][5, 6] == xt.XT_EINVAL            # h0 = 0
    assert want[0][6, 6] == 0                       # exactly 8192 columns
    assert tuple(want[0][3]) == (7, 0, 0, 7, 0, 0, 0)
    assert tuple(want[0][4]) == (9, 0, 0, -1, 0, 0, 0)
    assert_same(run_gpu_bwa(ctx, b, wide), want, "limits")
    narrow = BwaScoringParams(w=100)                # the same queries fit with a 100-base band
    assert_same(run_gpu_bwa(ctx, b2, narrow), run_oracle_bwa(b2, narrow), "narrow")
    # a pair pointing outside its buffer
    b.q_off[2] = b.q_seq.size
    assert_same(run_gpu_bwa(ctx, b, narrow), run_oracle_bwa(b, narrow), "outside")


def test_bad_scoring_and_empty(ctx):
    import paper_2301_09310_gb300 as xt
    b = synth.generate(synth.WORKLOADS["c1_tiny"], n=10)
    for bad in (BwaScoringParams(e_del=0), BwaScoringParams(match=0),
                BwaScoringParams(end_bonus=-1), BwaScoringParams(o_ins=2000)):
        with pytest.raises(xt.XtError) as e:
            run_gpu_bwa(ctx, b, bad)
        assert e.value.status == xt.XT_EINVAL
        assert xt.xt_bwa_scoring_check(bad) == xt.XT_EINVAL
    assert xt.xt_bwa_scoring_check(BwaScoringParams()) == xt.XT_OK
    z = np.zeros(0, np.int32)
    empty = synth.Batch(b.q_seq, np.zeros(0, np.int64), z, b.t_seq, np.zeros(0, np.int64), z, z)
    out, cells = run_gpu_bwa(ctx, empty, BwaScoringParams())
    assert out.shape == (0, 7)


def test_ascii_reads(ctx):
    import paper_2301_09310_gb300 as xt
    wl = synth.WORKLOADS["c3_mixed"]
    b = synth.generate(wl, n=3000, first=5)
    sc = BwaScoringParams.from_scoring(wl.scoring)
    letters = np.frombuffer(b"ACGTN", np.uint8)
    asc = synth.Batch(letters[np.minimum(b.q_seq, 4)], b.q_off, b.q_len,
                      np.frombuffer(b"acgtn", np.uint8)[np.minimum(b.t_seq, 4)], b.t_off,
                      b.t_len, b.h0)
    c = xt.Context(0)
    try:
        c.set_alphabet(xt.XT_ALPHABET_ASCII)
        assert_same(run_gpu_bwa(c, asc, sc), run_oracle_bwa(b, sc), "ascii")
    finally:
        c.close()


def test_default_call_unchanged_after_bwa(ctx):
    # the two entry points share a context: a default call after a BWA call
    # still gives the default definition's results
    from tests.gpu_util import run_gpu, run_oracle
    wl = synth.WORKLOADS["c3_mixed"]
    b = synth.generate(wl, n=5000, first=11)
    run_gpu_bwa(ctx, b, BwaScoringParams.from_scoring(wl.scoring))
    assert_same(run_gpu(ctx, b, wl.scoring), run_oracle(b, wl.scoring), "default after bwa")
