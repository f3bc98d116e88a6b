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
