"""The N > 1 path of bench.py on CPU: two gloo ranks run the same shard,
barrier and reduction code the GPU ranks run under NCCL (pairs are
independent, so the only cross-rank traffic is the timing max and the
work sums of the weak-scaling line)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    from paper_2301_09310_gb300 import synth

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        class A:
            gpus = world
        w, r, local = bench.dist_setup(A())
        first, n = bench.shard_of(r, 500)
        b = synth.generate(synth.WORKLOADS["c2_short"], n=n, first=first)
        units = float(b.q_len.sum())            # any per-rank work count
        seconds = 0.5 + r                        # rank 1 is the slowest
        bench.barrier(w)
        total, slowest, rate = bench.aggregate(w, units, seconds)
        q.put((r, w, local, first, n, units, total, slowest, rate, b.q_len[:4].tolist()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, f0, n0, u0, t0, s0, v0, h0), (r1, w1, l1, f1, n1, u1, t1, s1, v1, h1) = got
    assert (r0, r1, w0, w1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert (f0, n0, f1, n1) == (0, 500, 500, 500)       # disjoint, contiguous shards
    assert t0 == t1 == pytest.approx(u0 + u1)          # work summed over ranks
    assert s0 == s1 == pytest.approx(1.5)              # the slowest rank's time
    assert v0 == pytest.approx((u0 + u1) / 1.5)
    # a rank's pairs do not depend on how many ranks there are
    from paper_2301_09310_gb300 import synth
    alone = synth.generate(synth.WORKLOADS["c2_short"], n=1000, first=0)
    assert alone.q_len[500:504].tolist() == h1 and alone.q_len[:4].tolist() == h0
