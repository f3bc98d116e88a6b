"""Helpers shared by the GPU tests: run a batch through libxt (the CUDA path)
and through the CPU oracle on the same arrays."""
import random

import numpy as np

import oracle
from paper_2301_09310_gb300 import synth

CODES = "ACGTN"


def to_dev(b, dev):
    import torch
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    return (t(b.q_seq), t(b.q_off), t(b.q_len), t(b.t_seq), t(b.t_off), t(b.t_len), t(b.h0))


def run_gpu(ctx, b, scoring, plain=False):
    import torch
    args = to_dev(b, torch.device("cuda", ctx.device))
    out, cells = ctx.extend(*args, scoring, plain=plain)
    torch.cuda.synchronize()
    return out.cpu().numpy(), cells.cpu().numpy()


def run_oracle(b, scoring):
    return oracle.extend_batch(b.q_seq, b.q_off, b.q_len, b.t_seq, b.t_off, b.t_len, b.h0,
                               oracle.Scoring(*scoring.as_tuple()))


def assert_same(got, want, what=""):
    (go, gc), (wo, wc) = got, want
    if not np.array_equal(go, wo):
        bad = np.nonzero(np.any(go != wo, axis=1))[0]
        k = bad[0]
        raise AssertionError(f"{what}: {bad.size} pairs differ; first #{k}: gpu {go[k].tolist()} "
                             f"oracle {wo[k].tolist()}")
    if not np.array_equal(gc, wc):
        bad = np.nonzero(gc != wc)[0]
        k = bad[0]
        raise AssertionError(f"{what}: cells differ on {bad.size} pairs; first #{k}: gpu {gc[k]} "
                             f"oracle {wc[k]}")


def batch_from_lists(qs, ts, h0s):
    """Pack lists of code arrays into a synth.Batch."""
    ql = np.array([len(q) for q in qs], np.int32)
    tl = np.array([len(t) for t in ts], np.int32)
    qo = np.zeros(len(qs), np.int64)
    to = np.zeros(len(ts), np.int64)
    if len(qs) > 1:
        qo[1:] = np.cumsum(ql[:-1], dtype=np.int64)
        to[1:] = np.cumsum(tl[:-1], dtype=np.int64)
    qs_ = np.concatenate([np.asarray(q, np.uint8) for q in qs]) if ql.sum() else np.zeros(0, np.uint8)
    ts_ = np.concatenate([np.asarray(t, np.uint8) for t in ts]) if tl.sum() else np.zeros(0, np.uint8)
    return synth.Batch(qs_, qo, ql, ts_, to, tl, np.asarray(h0s, np.int32))


def fuzz_batch(seed, n, max_len=40, tail=30):
    """Edge-heavy random pairs: lengths 0..3 often, identical, related,
    unrelated, all-N, query much longer than target and the reverse."""
    rng = random.Random(seed)
    qs, ts, hs = [], [], []
    for _ in range(n):
        kind = rng.random()
        if kind < 0.15:
            ql, tl = rng.randint(0, 3), rng.randint(0, 3)
        elif kind < 0.25:
            ql, tl = rng.randint(20, max_len), rng.randint(0, 4)
        elif kind < 0.35:
            ql, tl = rng.randint(0, 4), rng.randint(20, max_len + tail)
        else:
            ql = rng.randint(1, max_len)
            tl = ql + rng.randint(0, tail)
        q = [rng.randint(0, 3) for _ in range(ql)]
        style = rng.random()
        if style < 0.1:
            q = [4] * ql
            t = [rng.randint(0, 4) for _ in range(tl)]
        elif style < 0.3:
            t = [rng.randint(0, 3) for _ in range(tl)]
        else:
            t = list(q[:tl]) + [rng.randint(0, 3) for _ in range(max(0, tl - ql))]
            for k in range(len(t)):
                r = rng.random()
                if r < 0.06:
                    t[k] = rng.randint(0, 3)
                elif r < 0.07:
                    t[k] = 4 + rng.randint(0, 20)  # any byte >= 4 is N
        h = rng.choice([1, 2, 5, rng.randint(1, 80)])
        qs.append(q)
        ts.append(t)
        hs.append(h)
    return batch_from_lists(qs, ts, hs)
