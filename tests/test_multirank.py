"""The N > 1 path on CPU: two gloo ranks run the same shard, barrier and
reduction code the GPU ranks run under NCCL.  Pairs are independent, so the
only cross-rank traffic is the timing max and the work sums of the
weak-scaling line, and (here, to check the split) the results gathered back
into input order.

The split is the library's LPT partitioner (xt_shard_lpt) on estimated
cells.  The batch is skewed on purpose -- its pairs ordered by query length
-- so that the contiguous halves a naive split would take differ several
fold in work, while the LPT parts differ by at most a pair.  Each rank
extends its part with the CPU oracle (no GPU here); the gathered results
must equal one oracle run on the whole batch."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

N_PER_RANK = 1500


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def skewed_workload():
    """c5_stream pairs (lognormal query lengths, a heavy tail) with the
    stream indices ordered by query length: the second half holds the
    long queries."""
    from paper_2301_09310_gb300 import synth
    wl = synth.WORKLOADS["c5_stream"]
    q_len, _, _ = synth.shapes(wl, n=2 * N_PER_RANK)
    order = np.argsort(q_len, kind="stable").astype(np.int64)
    return wl, order


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    import oracle
    import paper_2301_09310_gb300 as xt
    from paper_2301_09310_gb300 import synth

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        class A:
            gpus = world
        w, r, local = bench.dist_setup(A())
        wl, order = skewed_workload()
        q_len, t_len, _ = synth.shapes(wl, n=world * N_PER_RANK)
        # the job in skewed order: position p is stream pair order[p]
        shard, part_cells = xt.xt_shard_lpt(q_len[order], t_len[order], wl.scoring.w, world)
        mine = np.nonzero(shard == r)[0]
        b = synth.generate_at(wl, order[mine])
        out, cells = oracle.extend_batch(b.q_seq, b.q_off, b.q_len, b.t_seq, b.t_off, b.t_len,
                                         b.h0, oracle.Scoring(*wl.scoring.as_tuple()))
        units = float(cells.sum())
        seconds = 0.5 + r                        # rank 1 is the slowest
        bench.barrier(w)
        total, slowest, rate = bench.aggregate(w, units, seconds)
        parts = [None] * w
        dist.all_gather_object(parts, (mine, out, cells))
        q.put((r, w, local, units, total, slowest, rate, part_cells.tolist(), parts))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_lpt_shards_and_reduce():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=300) for _ in range(world)), key=lambda g: g[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, u0, t0, s0, v0, pc0, parts0), (r1, w1, l1, u1, t1, s1, v1, pc1, _) = got
    assert (r0, r1, w0, w1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert t0 == t1 == pytest.approx(u0 + u1)          # work summed over ranks
    assert s0 == s1 == pytest.approx(1.5)              # the slowest rank's time
    assert v0 == pytest.approx((u0 + u1) / 1.5)
    assert pc0 == pc1                                  # every rank computed the same split

    import oracle
    import paper_2301_09310_gb300 as xt
    from paper_2301_09310_gb300 import synth
    wl, order = skewed_workload()
    n = world * N_PER_RANK
    # the parts cover the job exactly once
    idx = np.concatenate([p[0] for p in parts0])
    assert np.array_equal(np.sort(idx), np.arange(n))
    # balance: LPT parts within one pair's estimate of each other, while the
    # contiguous halves of the same order differ several fold
    q_len, t_len, _ = synth.shapes(wl, n=n)
    est = _estimated_cells(q_len[order], t_len[order], wl.scoring.w)
    assert abs(pc0[0] - pc0[1]) <= est.max()
    assert sum(pc0) == est.sum()
    halves = est[:n // 2].sum(), est[n // 2:].sum()
    assert max(halves) > 3 * min(halves)
    # results gathered back into input order equal one run on the whole batch
    out = np.zeros((n, 7), np.int32)
    cells = np.zeros(n, np.int64)
    for mine, o, c in parts0:
        out[mine], cells[mine] = o, c
    whole = synth.generate_at(wl, order)
    want_out, want_cells = oracle.extend_batch(
        whole.q_seq, whole.q_off, whole.q_len, whole.t_seq, whole.t_off, whole.t_len, whole.h0,
        oracle.Scoring(*wl.scoring.as_tuple()))
    assert np.array_equal(out, want_out) and np.array_equal(cells, want_cells)
    assert xt is not None


def _estimated_cells(q_len, t_len, w):
    """In-band cells of each whole pair, counted row by row."""
    est = np.zeros(q_len.size, np.int64)
    for k, (ql, tl) in enumerate(zip(q_len.tolist(), t_len.tolist())):
        est[k] = sum(max(0, min(ql, i + w + 1) - max(0, i - w)) for i in range(tl))
    return est
