"""Full-size runs in the launch configuration bench.py times (xt_extend_batch
on the whole batch, default schedule): a random sample of pairs is compared
field by field with the CPU oracle, and properties that hold for every pair
are checked on all of them."""
import numpy as np
import pytest

from paper_2301_09310_gb300 import synth

from tests.gpu_util import run_gpu, run_oracle

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


def check_properties(b, out, cells, sc):
    score, qle, tle, gscore, gtle, max_off, status = out.T
    assert np.all(status == 0)
    assert np.all(score >= b.h0)
    assert np.all((qle >= 0) & (qle <= b.q_len) & (tle >= 0) & (tle <= b.t_len))
    assert np.all(np.abs(qle.astype(np.int64) - tle) <= sc.w)
    assert np.all(gscore <= score)
    assert np.all((gscore == -1) | (gscore > 0))
    assert np.all((gtle >= 0) & (gtle <= b.t_len))
    assert np.all(max_off <= sc.w)
    # cells never exceed the in-band cells of the whole pair
    ql = b.q_len.astype(np.int64)
    tl = b.t_len.astype(np.int64)
    assert np.all((cells >= 0) & (cells <= ql * np.minimum(tl, ql + sc.w)))


@pytest.mark.parametrize("name,sample", [("c3_mixed", 6000), ("c2_short", 6000)])
def test_full_batch_sampled_against_oracle(ctx, name, sample):
    wl = synth.WORKLOADS[name]
    b = synth.generate(wl)
    out, cells = run_gpu(ctx, b, wl.scoring)
    check_properties(b, out, cells, wl.scoring)
    rng = np.random.default_rng(2301)
    idx = np.sort(rng.choice(b.n, size=sample, replace=False))
    sub = b.take(idx)
    want_out, want_cells = run_oracle(sub, wl.scoring)
    got_out, got_cells = out[idx], cells[idx]
    bad = np.nonzero(np.any(got_out != want_out, axis=1) | (got_cells != want_cells))[0]
    assert bad.size == 0, (f"{bad.size} of {sample} sampled pairs differ; first pair "
                           f"#{idx[bad[0]]}: gpu {got_out[bad[0]].tolist()} cells {got_cells[bad[0]]}"
                           f" oracle {want_out[bad[0]].tolist()} cells {want_cells[bad[0]]}")
    # the plain kernel agrees with the batched one on every pair
    pout, pcells = run_gpu(ctx, b, wl.scoring, plain=True)
    assert np.array_equal(pout, out) and np.array_equal(pcells, cells)


def test_bwa_full_batch_sampled_against_oracle(ctx):
    # the BWA-MEM-compatible call on the whole c3 batch, as bench.py times it
    import torch
    from paper_2301_09310_gb300.synth import BwaScoringParams

    import oracle
    from tests.gpu_util import to_dev
    wl = synth.WORKLOADS["c3_mixed"]
    b = synth.generate(wl)
    sc = BwaScoringParams.from_scoring(wl.scoring)
    o, c = ctx.extend_bwa(*to_dev(b, torch.device("cuda", ctx.device)), sc)
    torch.cuda.synchronize()
    out, cells = o.cpu().numpy(), c.cpu().numpy()
    score, qle, tle, gscore, gtle, max_off, status = out.T
    assert np.all(status == 0) and np.all(score >= b.h0) and np.all(cells >= 0)
    assert np.all((qle <= b.q_len) & (tle <= b.t_len) & (gscore <= score) & (gscore >= -1))
    rng = np.random.default_rng(2302)
    idx = np.sort(rng.choice(b.n, size=6000, replace=False))
    sub = b.take(idx)
    want_out, want_cells = oracle.extend_batch_bwa(sub.q_seq, sub.q_off, sub.q_len, sub.t_seq,
                                                   sub.t_off, sub.t_len, sub.h0,
                                                   oracle.BwaScoring(*sc.as_tuple()))
    bad = np.nonzero(np.any(out[idx] != want_out, axis=1) | (cells[idx] != want_cells))[0]
    assert bad.size == 0, (f"{bad.size} of 6000 sampled pairs differ; first pair #{idx[bad[0]]}: "
                           f"gpu {out[idx][bad[0]].tolist()} oracle {want_out[bad[0]].tolist()}")


def test_c4_full_batch_sampled_against_oracle(ctx):
    """All 250,000 long pairs of c4_long (w = 500, z-drop 400) in one call, as
    bench.py's c4 leg times it.  Together the long buckets hold more than two
    full waves of one-lane slots, so the count-aware plan takes one lane per
    pair with 16-row strips for every bucket of queries over 510 bases; 2,000
    sampled pairs are compared with the oracle on every field and on cells,
    and every pair is checked for the properties above."""
    wl = synth.WORKLOADS["c4_long"]
    b = synth.generate(wl)
    assert b.n == 250_000
    out, cells = run_gpu(ctx, b, wl.scoring)
    check_properties(b, out, cells, wl.scoring)
    rng = np.random.default_rng(2304)
    idx = np.sort(rng.choice(b.n, size=2000, replace=False))
    sub = b.take(idx)
    want_out, want_cells = run_oracle(sub, wl.scoring)
    got_out, got_cells = out[idx], cells[idx]
    bad = np.nonzero(np.any(got_out != want_out, axis=1) | (got_cells != want_cells))[0]
    assert bad.size == 0, (f"{bad.size} of 2000 sampled pairs differ; first pair "
                           f"#{idx[bad[0]]}: gpu {got_out[bad[0]].tolist()} cells {got_cells[bad[0]]}"
                           f" oracle {want_out[bad[0]].tolist()} cells {want_cells[bad[0]]}")


def test_c5_long_queries_packed_with_short_tags(ctx):
    """A 600,000-pair call of the c5 mix: at 2^19 pairs and more, queries of
    511 bases and longer (h0 + match * length above 511) run packed with
    4-bit row-key tags.  1,500 of them and 500 other pairs are compared with
    the oracle on every field and on cells, and every pair must equal the
    same pairs extended in two calls of 300,000 (below that size the long
    queries take the 32-bit engines)."""
    wl = synth.WORKLOADS["c5_stream"]
    b = synth.generate(wl, n=600_000)
    out, cells = run_gpu(ctx, b, wl.scoring)
    check_properties(b, out, cells, wl.scoring)
    rng = np.random.default_rng(2305)
    long_ = np.nonzero(b.q_len >= 511)[0]
    assert long_.size > 1500
    idx = np.unique(np.concatenate([rng.choice(long_, size=1500, replace=False),
                                    rng.choice(b.n, size=500, replace=False)]))
    sub = b.take(idx)
    want_out, want_cells = run_oracle(sub, wl.scoring)
    got_out, got_cells = out[idx], cells[idx]
    bad = np.nonzero(np.any(got_out != want_out, axis=1) | (got_cells != want_cells))[0]
    assert bad.size == 0, (f"{bad.size} of {idx.size} sampled pairs differ; first pair "
                           f"#{idx[bad[0]]}: gpu {got_out[bad[0]].tolist()} cells {got_cells[bad[0]]}"
                           f" oracle {want_out[bad[0]].tolist()} cells {want_cells[bad[0]]}")
    half = b.n // 2
    for lo, hi in ((0, half), (half, b.n)):
        part = b.take(np.arange(lo, hi))
        pout, pcells = run_gpu(ctx, part, wl.scoring)
        assert np.array_equal(pout, out[lo:hi]) and np.array_equal(pcells, cells[lo:hi])
