"""Per-bucket schedules and the autotuner: every schedule a bucket can take
gives the oracle's results bit for bit, and a tuned table survives a round
trip through its JSON file."""
import json

import numpy as np
import pytest

from paper_2301_09310_gb300 import synth
from paper_2301_09310_gb300.synth import ScoringParams

from tests.gpu_util import assert_same, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture()
def xt():
    import torch
    import paper_2301_09310_gb300 as xt
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return xt


def test_bucket_schedule_api(xt):
    ctx = xt.Context(0)
    try:
        assert ctx.bucket_schedule(100, 7) == (0, 0)
        ctx.set_bucket_schedule(100, 7, 4, 8)
        assert ctx.bucket_schedule(100, 7) == (4, 8)
        assert ctx.bucket_schedule(50, 7) == (0, 0)       # kept per band
        for P, R in ((3, 8), (8, 16), (1, 5), (64, 8)):
            with pytest.raises(xt.XtError) as e:
                ctx.set_bucket_schedule(100, 7, P, R)
            assert e.value.status == xt.XT_EINVAL
        with pytest.raises(xt.XtError):
            ctx.set_bucket_schedule(100, 4, 1, 8)            # no bucket 4
        ctx.set_bucket_schedule(100, 7, 0, 0)
        assert ctx.bucket_schedule(100, 7) == (0, 0)
    finally:
        ctx.close()


# (bucket range, P, R): group schedules on short buckets, the one-lane engine
# on long ones (queries up to 16382 bases)
PLANS = [
    [((5, 9), 4, 8), ((10, 14), 1, 8)],
    [((5, 9), 16, 4), ((10, 14), 1, 16)],
    [((5, 9), 1, 4), ((10, 14), 8, 8)],
]


@pytest.mark.parametrize("plan", range(len(PLANS)))
def test_explicit_schedules_match_oracle(xt, plan):
    c3 = synth.WORKLOADS["c3_mixed"]
    c4 = synth.WORKLOADS["c4_long"]
    c5 = synth.WORKLOADS["c5_stream"]
    cases = [(synth.generate(c3, n=3000), c3.scoring), (synth.generate(c4, n=24), c4.scoring),
             (synth.generate(c5, n=3000, first=777), c5.scoring)]
    ctx = xt.Context(0)
    try:
        for b, sc in cases:
            n_set = 0
            for (lo, hi), P, R in PLANS[plan]:
                for j in range(lo, hi + 1):
                    try:
                        ctx.set_bucket_schedule(sc.w, j, P, R)
                        n_set += 1
                    except xt.XtError as e:   # ring too large for this band: built-in rule
                        assert e.status == xt.XT_EINVAL
            assert n_set >= 5
            assert_same(run_gpu(ctx, b, sc), run_oracle(b, sc), f"plan {plan} w={sc.w}")
    finally:
        ctx.close()


def test_autotune_round_trip(xt, tmp_path):
    path = str(tmp_path / "tuning.json")
    sc = ScoringParams()
    ctx = xt.Context(0)
    try:
        ctx.autotune(sc, j_max=8, cells_per_trial=3e7, table_path=path)
        chosen = {(j, k): ctx.bucket_schedule(sc.w, j, k) for j in range(5, 9)
                  for k in (xt.XT_BATCH_LARGE, xt.XT_BATCH_SMALL)}
        assert all(P >= 1 for P, _ in chosen.values())
        # a second band goes into the same file
        ctx.autotune(ScoringParams(w=20, zdrop=30), j_max=6, cells_per_trial=1e7, table_path=path)
    finally:
        ctx.close()
    doc = json.load(open(path))
    assert doc["format"] == "xt-tuning" and len(doc["entries"]) == 2
    e = [x for x in doc["entries"] if x["w"] == sc.w][0]
    assert [b["j"] for b in e["buckets"]] == [5, 6, 7, 8]
    assert all(b["gcups"] > 0 and b["gcups_s"] > 0 and b["Ps"] >= 1 for b in e["buckets"])
    ctx = xt.Context(0)
    try:
        ctx.load_tuning(path)
        assert {(j, k): ctx.bucket_schedule(sc.w, j, k) for j in range(5, 9)
                for k in (xt.XT_BATCH_LARGE, xt.XT_BATCH_SMALL)} == chosen
        wl = synth.WORKLOADS["c3_mixed"]
        b = synth.generate(wl, n=4000, first=123)
        assert_same(run_gpu(ctx, b, wl.scoring), run_oracle(b, wl.scoring), "tuned")
    finally:
        ctx.close()


def test_load_tuning_ignores_other_devices_and_rejects_garbage(xt, tmp_path):
    other = tmp_path / "other.json"
    other.write_text(json.dumps({"format": "xt-tuning", "version": 1, "entries": [
        {"device": "some other GPU", "sms": 7, "w": 100, "scoring": [1, -4, 6, 1, 100, 100, -1],
         "buckets": [{"j": 6, "P": 4, "R": 8, "gcups": 1.0}]}]}))
    bad = tmp_path / "bad.json"
    bad.write_text("{\"entries\": [ {\"device\": ")
    ctx = xt.Context(0)
    try:
        ctx.load_tuning(str(other))
        assert ctx.bucket_schedule(100, 6) == (0, 0)
        for p in (str(bad), str(tmp_path / "missing.json")):
            with pytest.raises(xt.XtError) as e:
                ctx.load_tuning(p)
            assert e.value.status == xt.XT_EINVAL
    finally:
        ctx.close()


def test_small_and_large_batch_classes(xt):
    # different schedules for small and large calls; both sizes stay exact
    wl = synth.WORKLOADS["c5_stream"]
    small = synth.generate(wl, n=3000, first=4242)
    large = synth.generate(wl, n=40000, first=9000)
    ctx = xt.Context(0)
    try:
        for j in range(5, 12):
            ctx.set_bucket_schedule_for(wl.scoring.w, j, xt.XT_BATCH_LARGE, 1, 8)
            ctx.set_bucket_schedule_for(wl.scoring.w, j, xt.XT_BATCH_SMALL, 8, 8)
        assert ctx.bucket_schedule(wl.scoring.w, 9, xt.XT_BATCH_SMALL) == (8, 8)
        assert ctx.bucket_schedule(wl.scoring.w, 9, xt.XT_BATCH_LARGE) == (1, 8)
        for b in (small, large):
            assert_same(run_gpu(ctx, b, wl.scoring), run_oracle(b, wl.scoring), f"n={b.n}")
        with pytest.raises(xt.XtError):
            ctx.set_bucket_schedule_for(wl.scoring.w, 9, 2, 1, 8)   # no such class
    finally:
        ctx.close()
