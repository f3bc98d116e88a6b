"""The serving loop (xt_serve_*): requests of host pairs, continuously batched.

Every request's results must equal the CPU oracle on that request alone,
whatever else shared its batch; admission, pausing, timeouts and the drain
at destroy behave as include/xt.h states."""
import threading

import numpy as np
import pytest

from paper_2301_09310_gb300 import synth
from paper_2301_09310_gb300.synth import Batch, ScoringParams

from tests.gpu_util import run_oracle

pytestmark = pytest.mark.gpu

WL = synth.WORKLOADS["c5_stream"]
OTHER = ScoringParams(w=3, zdrop=5)


@pytest.fixture(scope="module")
def xt():
    import torch
    import paper_2301_09310_gb300 as xt
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return xt


def as_batch(req) -> Batch:
    return Batch(*[np.array(a, copy=True) for a in req])


def oracle_of(req, sc):
    return run_oracle(as_batch(req), sc)


def check(out, cells, want, what):
    w_out, w_cells = want
    assert out.shape == w_out.shape, what
    bad = np.nonzero(np.any(out != w_out, axis=1) | (cells != w_cells))[0]
    assert bad.size == 0, (f"{what}: {bad.size} pairs differ, first #{bad[0]}: "
                           f"{out[bad[0]].tolist()} vs {w_out[bad[0]].tolist()}")


def stream(n, sizes=None, seed=5):
    b = synth.generate(WL, n=n, first=seed * 1000)
    return synth.request_stream(b, 1e6, max_request=512, seed=seed, sizes=sizes)


def test_requests_match_oracle_mixed_scorings(xt):
    sizes = [1, 7, 0, 300, 1024, 13, 2048, 5, 600, 2, 0, 1]
    rs = stream(sum(sizes), sizes)
    reqs = [rs.request(r) for r in range(len(sizes))]
    # a pair whose query lies outside its own request's buffer (but inside
    # the stream's) must be rejected, not read from a neighbouring request
    r3 = list(reqs[3])
    r3[1] = r3[1].copy()
    r3[1][4] = r3[0].size + 10
    reqs[3] = tuple(r3)
    scorings = [WL.scoring if k % 3 else OTHER for k in range(len(reqs))]
    srv = xt.Server(0, slots=3)
    try:
        tickets = [srv.submit(*req, sc) for req, sc in zip(reqs, scorings)]
        for k, (t, req, sc) in enumerate(zip(tickets, reqs, scorings)):
            out, cells, times = srv.wait(t, timeout_s=120)
            assert times["status"] == xt.XT_OK
            assert times["submit_ns"] <= times["launch_ns"] <= times["done_ns"]
            check(out, cells, oracle_of(req, sc), f"request {k}")
        assert out is not None
        st = srv.stats()
        assert st["requests"] == len(reqs) and st["pairs"] == sum(sizes)
    finally:
        srv.close()
    # the planted bad pair
    assert oracle_of(reqs[3], scorings[3])[0][4, 6] == xt.XT_EINVAL


def test_alone_equals_mix(xt):
    rs = stream(9000)
    reqs = [rs.request(r) for r in range(rs.size.size)]
    k = len(reqs) // 2
    srv = xt.Server(0, slots=1)
    try:
        alone = srv.wait(srv.submit(*reqs[k], WL.scoring), timeout_s=120)
    finally:
        srv.close()
    srv = xt.Server(0, slots=2)
    try:
        srv.pause(True)
        tickets = [srv.submit(*r, WL.scoring) for r in reqs]
        srv.pause(False)
        got = [srv.wait(t, timeout_s=120) for t in tickets]
    finally:
        srv.close()
    out, cells, times = got[k]
    assert times["batch_pairs"] > reqs[k][2].size   # it shared its batch
    assert np.array_equal(out, alone[0]) and np.array_equal(cells, alone[1])
    check(out, cells, oracle_of(reqs[k], WL.scoring), "mixed request")


def test_admission_pause_timeout(xt):
    rs = stream(600, [200, 200, 200])
    reqs = [rs.request(r) for r in range(3)]
    one = sum(a.nbytes for a in reqs[0]) + 2048
    srv = xt.Server(0, slots=1, max_batch_pairs=250, max_queued_bytes=one)
    try:
        srv.pause(True)
        t0 = srv.submit(*reqs[0], WL.scoring)
        with pytest.raises(xt.XtError) as e:
            srv.submit(*reqs[1], WL.scoring)        # queue full while paused
        assert e.value.status == xt.XT_EBUSY
        with pytest.raises(xt.XtError) as e:
            srv.wait(t0, timeout_s=0.05)              # not launched while paused
        assert e.value.status == xt.XT_ETIMEOUT
        assert not srv.poll(t0)
        big = stream(251, [251]).request(0)
        with pytest.raises(xt.XtError) as e:
            srv.submit(*big, WL.scoring)              # larger than one batch
        assert e.value.status == xt.XT_EINVAL
        with pytest.raises(xt.XtError) as e:
            srv.submit(*reqs[1], ScoringParams(match=0))
        assert e.value.status == xt.XT_EINVAL
        srv.pause(False)
        out, cells, _ = srv.wait(t0, timeout_s=120)
        check(out, cells, oracle_of(reqs[0], WL.scoring), "after resume")
        t1 = srv.submit(*reqs[1], WL.scoring, retry_busy=True)
        out, cells, _ = srv.wait(t1, timeout_s=120)
        check(out, cells, oracle_of(reqs[1], WL.scoring), "after admission")
        with pytest.raises(xt.XtError) as e:
            srv.wait(t1)                              # released ticket
        assert e.value.status == xt.XT_EINVAL
    finally:
        srv.close()


def test_destroy_drains_queue(xt):
    rs = stream(3000)
    reqs = [rs.request(r) for r in range(rs.size.size)]
    srv = xt.Server(0, slots=2)
    srv.pause(True)
    tickets = [srv.submit(*r, WL.scoring) for r in reqs]
    outs = [srv._live[t][1:] for t in tickets]
    srv.close()                                       # resumes and finishes the queue
    for k, ((out, cells), req) in enumerate(zip(outs, reqs)):
        check(out, cells, oracle_of(req, WL.scoring), f"drained request {k}")


def test_concurrent_submitters(xt):
    rs = stream(12000)
    reqs = [rs.request(r) for r in range(rs.size.size)]
    srv = xt.Server(0, slots=3)
    results = {}
    errors = []

    def client(idx):
        try:
            for k in idx:
                results[k] = srv.wait(srv.submit(*reqs[k], WL.scoring, retry_busy=True),
                                      timeout_s=120)
        except Exception as ex:  # noqa: BLE001
            errors.append(ex)

    ths = [threading.Thread(target=client, args=(range(c, len(reqs), 4),)) for c in range(4)]
    try:
        for th in ths:
            th.start()
        for th in ths:
            th.join()
    finally:
        srv.close()
    assert not errors, errors
    want = run_oracle(rs.batch, WL.scoring)
    for k, req in enumerate(reqs):
        a, n = int(rs.start[k]), int(rs.size[k])
        out, cells, _ = results[k]
        check(out, cells, (want[0][a:a + n], want[1][a:a + n]), f"request {k}")


def test_server_with_tuning_table(xt, tmp_path):
    path = str(tmp_path / "tuning.json")
    ctx = xt.Context(0)
    try:
        ctx.autotune(WL.scoring, j_max=8, cells_per_trial=2e7, table_path=path)
    finally:
        ctx.close()
    rs = stream(6000, seed=6)
    reqs = [rs.request(r) for r in range(rs.size.size)]
    srv = xt.Server(0, slots=2, tuning_path=path)
    try:
        tickets = [srv.submit(*r, WL.scoring) for r in reqs]
        for k, (t, req) in enumerate(zip(tickets, reqs)):
            out, cells, _ = srv.wait(t, timeout_s=120)
            check(out, cells, oracle_of(req, WL.scoring), f"tuned request {k}")
    finally:
        srv.close()
    with pytest.raises(xt.XtError) as e:
        xt.Server(0, slots=1, tuning_path=str(tmp_path / "missing.json"))
    assert e.value.status == xt.XT_EINVAL


def test_full_stream_10m_equals_batched(xt):
    """The served stream at its stated size: 10,000,000 c5 pairs cut into
    requests of U[1, 4096] pairs, all submitted as fast as the queue admits
    them (as the 90% load level does when it falls behind).  Every request's
    results equal one batched call on the whole stream; a sample of pairs is
    also compared with the oracle."""
    import torch
    from tests.gpu_util import to_dev
    b = synth.generate(WL, n=10_000_000)
    rs = synth.request_stream(b, 1e9, seed=5)
    ctx = xt.Context(0)
    try:
        o, c = ctx.extend(*to_dev(b, torch.device("cuda", 0)), WL.scoring)
        torch.cuda.synchronize()
        ref_out, ref_cells = o.cpu().numpy(), c.cpu().numpy()
        del o, c
    finally:
        ctx.close()
    torch.cuda.empty_cache()
    nreq = int(rs.size.size)
    got = [None] * nreq
    srv = xt.Server(0, slots=3, mem_budget_bytes=40 * 10**9)
    try:
        tickets = []

        def waiter():
            for k in range(nreq):
                while k >= len(tickets):
                    threading.Event().wait(1e-4)
                got[k] = srv.wait(tickets[k], timeout_s=300)[:2]

        th = threading.Thread(target=waiter)
        th.start()
        for k in range(nreq):
            tickets.append(srv.submit(*rs.request(k), WL.scoring, retry_busy=True))
        th.join()
    finally:
        srv.close()
    for k in range(nreq):
        a, n = int(rs.start[k]), int(rs.size[k])
        check(got[k][0], got[k][1], (ref_out[a:a + n], ref_cells[a:a + n]), f"request {k}")
    rng = np.random.default_rng(2305)
    idx = np.sort(rng.choice(b.n, size=3000, replace=False))
    want_out, want_cells = run_oracle(b.take(idx), WL.scoring)
    check(ref_out[idx], ref_cells[idx], (want_out, want_cells), "sampled pairs vs oracle")
