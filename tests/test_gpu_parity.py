"""GPU parity: every field of every pair, bit-exact against the CPU oracle
(integer DP: the tolerance is zero), called through the C ABI."""
import numpy as np
import pytest

from paper_2301_09310_gb300 import synth
from paper_2301_09310_gb300.synth import ScoringParams

from tests.gpu_util import assert_same, batch_from_lists, fuzz_batch, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

SCHEDULES = [(1, 4), (1, 8), (1, 16), (2, 8), (4, 4), (4, 8), (4, 16), (8, 8), (16, 4), (32, 8)]

SCORINGS = [
    ScoringParams(),                                           # the workloads' scoring
    ScoringParams(w=3, zdrop=5),
    ScoringParams(w=0, zdrop=0),
    ScoringParams(match=2, mismatch=-3, gap_open=2, gap_extend=2, w=12, zdrop=20, n_score=-2),
    ScoringParams(match=3, mismatch=0, gap_open=0, gap_extend=0, w=7, zdrop=0, n_score=0),
    ScoringParams(w=1000, zdrop=-1),
]


@pytest.fixture(scope="module")
def ctx():
    import torch
    import paper_2301_09310_gb300 as xt
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = xt.Context(0)
    yield c
    c.close()


def test_c1_tiny_batched_and_plain(ctx):
    wl = synth.WORKLOADS["c1_tiny"]
    b = synth.generate(wl)
    want = run_oracle(b, wl.scoring)
    assert_same(run_gpu(ctx, b, wl.scoring), want, "batched")
    assert_same(run_gpu(ctx, b, wl.scoring, plain=True), want, "plain")


@pytest.mark.parametrize("si", range(len(SCORINGS)))
def test_fuzz_edges(ctx, si):
    sc = SCORINGS[si]
    b = fuzz_batch(100 + si, 1500)
    want = run_oracle(b, sc)
    assert_same(run_gpu(ctx, b, sc), want, f"batched {sc}")
    assert_same(run_gpu(ctx, b, sc, plain=True), want, f"plain {sc}")


@pytest.mark.parametrize("P,R", SCHEDULES)
def test_schedule_invariance(ctx, P, R):
    wl = synth.WORKLOADS["c3_mixed"]
    b = synth.generate(wl, n=3000)
    fz = fuzz_batch(7, 800, max_len=70, tail=60)
    try:
        ctx.set_schedule(P, R)
        for batch, sc in ((b, wl.scoring), (fz, SCORINGS[1]), (fz, SCORINGS[3])):
            assert_same(run_gpu(ctx, batch, sc), run_oracle(batch, sc), f"P={P} R={R} {sc}")
    finally:
        ctx.set_schedule(0)


@pytest.mark.parametrize("name,n", [("c2_short", 40000), ("c3_mixed", 40000), ("c5_stream", 8000)])
def test_workload_samples(ctx, name, n):
    wl = synth.WORKLOADS[name]
    b = synth.generate(wl, n=n)
    want = run_oracle(b, wl.scoring)
    assert_same(run_gpu(ctx, b, wl.scoring), want, f"{name} batched")
    assert_same(run_gpu(ctx, b, wl.scoring, plain=True), want, f"{name} plain")


def test_long_extensions(ctx):
    wl = synth.WORKLOADS["c4_long"]
    b = synth.generate(wl, n=48)
    want = run_oracle(b, wl.scoring)
    assert_same(run_gpu(ctx, b, wl.scoring), want, "c4 batched")
    assert_same(run_gpu(ctx, b, wl.scoring, plain=True), want, "c4 plain")


def test_huge_band_global_ring(ctx):
    # a band wider than any shared-memory ring: queries longer than 4094
    # with w = 6000 go to the global-slab kernel
    rng = np.random.default_rng(5)
    qs, ts, hs = [], [], []
    for k in range(4):
        q = rng.integers(0, 4, 4200 + 300 * k)
        t = q.copy()
        mut = rng.random(t.size) < 0.03
        t[mut] = rng.integers(0, 4, int(mut.sum()))
        qs.append(q)
        ts.append(np.concatenate([t, rng.integers(0, 4, 500)]))
        hs.append(30)
    # 2,200-base queries with w = 1000: a shared ring would leave one CTA per
    # SM, so these take the global slabs too
    for k in range(3):
        q = rng.integers(0, 4, 2200 + 100 * k)
        t = q.copy()
        mut = rng.random(t.size) < 0.03
        t[mut] = rng.integers(0, 4, int(mut.sum()))
        qs.append(q)
        ts.append(np.concatenate([t, rng.integers(0, 4, 500)]))
        hs.append(30)
    # and two of them again with a seed score that makes them WIDE: a bucket
    # whose group ring does not fit runs its narrow pairs on one-lane strips
    # and only its WIDE pairs on the global slabs
    for k in (4, 5):
        qs.append(qs[k])
        ts.append(ts[k])
        hs.append(40000)
    b = batch_from_lists(qs, ts, hs)
    import paper_2301_09310_gb300 as xt
    for sc in (ScoringParams(w=6000, zdrop=300), ScoringParams(w=1000, zdrop=300)):
        want = run_oracle(b, sc)
        assert_same(run_gpu(ctx, b, sc), want, f"huge batched w={sc.w}")
        assert_same(run_gpu(ctx, b, sc, plain=True), want, f"huge plain w={sc.w}")
        fresh = xt.Context(0)      # a new context's first plan, on a fresh stack
        try:
            assert_same(run_gpu(fresh, b, sc), want, f"huge fresh context w={sc.w}")
        finally:
            fresh.close()


def test_wide_scores(ctx):
    # h0 near the limit pushes the score bound past 16 bits: the WIDE path
    b = fuzz_batch(11, 600, max_len=60)
    b.h0[:] = np.where(np.arange(b.n) % 2 == 0, 40000 + np.arange(b.n), b.h0)
    b.h0[:] = np.minimum(b.h0, 1 << 20)
    sc = SCORINGS[0]
    want = run_oracle(b, sc)
    assert_same(run_gpu(ctx, b, sc), want, "wide batched")
    assert_same(run_gpu(ctx, b, sc, plain=True), want, "wide plain")


def test_invalid_pairs(ctx):
    b = fuzz_batch(12, 200)
    b.h0[3] = 0
    b.h0[4] = -5
    b.h0[5] = (1 << 20) + 1
    b.q_off[6] = b.q_seq.size + 10
    b.t_len[7] = -1
    b.q_len[8] = (1 << 20) + 1
    b.t_off[9] = -1
    sc = SCORINGS[0]
    want = run_oracle(b, sc)
    assert np.all(want[0][3:10, 6] == 1)
    assert_same(run_gpu(ctx, b, sc), want, "invalid batched")
    assert_same(run_gpu(ctx, b, sc, plain=True), want, "invalid plain")


def test_bad_scoring_rejected(ctx):
    import paper_2301_09310_gb300 as xt
    b = fuzz_batch(13, 10)
    with pytest.raises(xt.XtError) as e:
        run_gpu(ctx, b, ScoringParams(match=0))
    assert e.value.status == xt.XT_EINVAL


def test_empty_batch(ctx):
    b = batch_from_lists([], [], [])
    out, cells = run_gpu(ctx, b, SCORINGS[0])
    assert out.shape == (0, 7) and cells.shape == (0,)


def test_host_variant(ctx):
    wl = synth.WORKLOADS["c3_mixed"]
    b = synth.generate(wl, n=5000)
    out, cells = ctx.extend_host(b.q_seq, b.q_off, b.q_len, b.t_seq, b.t_off, b.t_len, b.h0,
                                 wl.scoring)
    assert_same((out, cells), run_oracle(b, wl.scoring), "host variant")


def test_host_variant_in_chunks(ctx):
    # 2.2M pairs: the host call runs in chunks whose sequence bytes are copied
    # while earlier chunks extend.  Its results must equal the device call's
    # (itself pinned to the oracle), for pairs in buffer order and for pairs
    # whose offsets jump around the buffers (every chunk then reads far ahead)
    import torch
    import paper_2301_09310_gb300 as xt
    wl = synth.WORKLOADS["c3_mixed"]
    b = synth.generate(wl, n=2_200_000, first=999)
    sample = np.random.default_rng(1).choice(b.n, 4000, replace=False)
    want_dev = run_gpu(ctx, b, wl.scoring)
    sub = b.take(np.sort(sample))
    assert_same((want_dev[0][np.sort(sample)], want_dev[1][np.sort(sample)]),
                run_oracle(sub, wl.scoring), "device sample")

    def pinned(a):
        t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True)
        t.numpy()[...] = a
        return t.numpy()

    perm = np.random.default_rng(2).permutation(b.n)
    for order in (np.arange(b.n), perm):
        h = [pinned(a) for a in (b.q_seq, b.q_off[order], b.q_len[order], b.t_seq,
                                 b.t_off[order], b.t_len[order], b.h0[order])]
        out, cells = ctx.extend_host(*h, wl.scoring)
        assert_same((out, cells), (want_dev[0][order], want_dev[1][order]), "chunked host call")
    # pairs outside their buffers (in the first and the last chunk) are
    # rejected, the rest unchanged
    qo, to = b.q_off.copy(), b.t_off.copy()
    qo[5] = b.q_seq.size + 100
    to[b.n - 3] = -7
    h = [pinned(a) for a in (b.q_seq, qo, b.q_len, b.t_seq, to, b.t_len, b.h0)]
    out, cells = ctx.extend_host(*h, wl.scoring)
    assert out[5, 6] == xt.XT_EINVAL and out[b.n - 3, 6] == xt.XT_EINVAL
    keep = np.ones(b.n, bool)
    keep[[5, b.n - 3]] = False
    assert np.array_equal(out[keep], want_dev[0][keep]) and np.array_equal(cells[keep],
                                                                           want_dev[1][keep])


def test_host_chunks_under_a_budget(ctx):
    # a context with a memory budget runs its chunks one after another on its
    # own workspace (a context without one spreads them over two internal
    # contexts): both must return the device call's results
    import torch
    import paper_2301_09310_gb300 as xt
    wl = synth.WORKLOADS["c3_mixed"]
    b = synth.generate(wl, n=2_100_000, first=4242)
    want = run_gpu(ctx, b, wl.scoring)

    def pinned(a):
        t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True)
        t.numpy()[...] = a
        return t.numpy()

    h = [pinned(a) for a in (b.q_seq, b.q_off, b.q_len, b.t_seq, b.t_off, b.t_len, b.h0)]
    budgeted = xt.Context(0, mem_budget_bytes=16 << 30)
    try:
        for _ in range(2):
            out, cells = budgeted.extend_host(*h, wl.scoring)
            assert_same((out, cells), want, "chunked host call under a budget")
    finally:
        budgeted.close()
    for _ in range(2):
        out, cells = ctx.extend_host(*h, wl.scoring)
        assert_same((out, cells), want, "chunked host call on chunk contexts")


def test_shared_ring_pool_under_a_budget(ctx):
    # a 1M-pair call of the c5 mix runs several global-ring launches: with no
    # budget each has a pool region of its own and they run side by side; a
    # 400 MB budget holds the largest of them but not their sum, so they
    # share one region and run one after another.  Both give the same results.
    import paper_2301_09310_gb300 as xt
    wl = synth.WORKLOADS["c5_stream"]
    b = synth.generate(wl, n=1_000_000, first=77)
    want = run_gpu(ctx, b, wl.scoring)
    budgeted = xt.Context(0, mem_budget_bytes=400 << 20)
    try:
        for _ in range(2):
            assert_same(run_gpu(budgeted, b, wl.scoring), want, "shared ring pool")
    finally:
        budgeted.close()


def test_repeat_calls_reuse_workspace(ctx):
    wl = synth.WORKLOADS["c2_short"]
    b1 = synth.generate(wl, n=2000, first=0)
    b2 = synth.generate(wl, n=7000, first=50000)
    for b in (b2, b1, b2):
        assert_same(run_gpu(ctx, b, wl.scoring), run_oracle(b, wl.scoring), "repeat")


def test_graph_replay_matches_direct(ctx):
    # the second call of a (scoring, size class) is captured, later ones replay
    # the graph; each call brings its own arrays through the device descriptor
    import paper_2301_09310_gb300 as xt
    wl = synth.WORKLOADS["c3_mixed"]
    # sizes grow within a capacity class after its capture (2200 -> 4000 in
    # the 4096 class, 1100 -> 2048 in the 2048 class): the workspace layout
    # baked into a graph must hold every size of its class
    sizes = (2100, 2200, 4000, 3000, 1500, 1100, 2048, 1025, 4096)
    batches = [synth.generate(wl, n=n, first=10000 * k) for k, n in enumerate(sizes)]
    want = []
    direct = xt.Context(0)
    direct.set_graphs(False)
    try:
        for b in batches:
            want.append(run_gpu(direct, b, wl.scoring))
    finally:
        direct.close()
    ctx.set_graphs(True)
    for rep in range(2):
        for b, w in zip(batches, want):
            assert_same(run_gpu(ctx, b, wl.scoring), w, f"graph replay {rep}")
    for b in batches[2:4]:
        assert_same(run_gpu(ctx, b, wl.scoring), run_oracle(b, wl.scoring), "graph vs oracle")


@pytest.mark.parametrize("L", [64, 300, 1100])
def test_equal_length_unbanded(ctx, L):
    # the paper's kernel comparison regime: qlen = tlen, band = whole table,
    # z-drop off; built-in schedule and explicit one-lane / group schedules
    import paper_2301_09310_gb300 as xt
    wl = synth.x2_workload(L)
    b = synth.generate(wl, n=40 if L < 1000 else 12)
    want = run_oracle(b, wl.scoring)
    assert np.all(want[1] == (want[1] > 0) * L * L)   # full tables while alive
    assert_same(run_gpu(ctx, b, wl.scoring), want, f"x2 {L} built-in")
    j = int(np.ceil(np.log2(L + 2)))
    other = xt.Context(0)
    try:
        for P, R in ((1, 8), (8, 8), (32, 4)):
            try:
                other.set_bucket_schedule(wl.scoring.w, j, P, R)
            except xt.XtError:
                continue
            assert_same(run_gpu(other, b, wl.scoring), want, f"x2 {L} P{P}R{R}")
    finally:
        other.close()


def test_two_step_call(ctx):
    # xt_extend_batch_begin / _ready / _finish give the one-call results; the
    # context refuses a second call while one is pending
    import time
    import torch
    import paper_2301_09310_gb300 as xt
    from tests.gpu_util import to_dev
    wl = synth.WORKLOADS["c5_stream"]
    b = synth.generate(wl, n=5000, first=31337)
    d = to_dev(b, torch.device("cuda", ctx.device))
    out = torch.empty((b.n, 7), dtype=torch.int32, device="cuda")
    cells = torch.empty(b.n, dtype=torch.int64, device="cuda")
    st = torch.cuda.current_stream()
    args = (d[0].data_ptr(), d[0].numel(), d[1].data_ptr(), d[2].data_ptr(), d[3].data_ptr(),
            d[3].numel(), d[4].data_ptr(), d[5].data_ptr(), d[6].data_ptr(), b.n,
            xt._scoring(wl.scoring), out.data_ptr(), cells.data_ptr(), st.cuda_stream)
    assert xt.xt_extend_batch_begin(ctx.handle, *args) == xt.XT_OK
    assert xt.xt_extend_batch(ctx.handle, *args) == xt.XT_EBUSY
    # every other call of the context waits its turn too (they share the
    # context's count read-back)
    assert xt.xt_extend_batch_bwa(ctx.handle, *args[:10], (1, -4, -1, 6, 1, 6, 1, 100, 100, 5),
                                  *args[11:]) == xt.XT_EBUSY
    z = torch.zeros(b.n, dtype=torch.int32, device="cuda")
    assert xt.xt_extend_seeds(ctx.handle, *args[:8], z.data_ptr(), z.data_ptr(), z.data_ptr(),
                              d[6].data_ptr(), b.n, wl.scoring, out.data_ptr(), out.data_ptr(),
                              0, 0, st.cuda_stream) == xt.XT_EBUSY
    for _ in range(20000):
        s, ready = xt.xt_extend_batch_ready(ctx.handle)
        assert s == xt.XT_OK
        if ready:
            break
        time.sleep(0.0005)
    assert ready
    assert xt.xt_extend_batch_finish(ctx.handle) == xt.XT_OK
    assert xt.xt_extend_batch_finish(ctx.handle) == xt.XT_EINVAL
    torch.cuda.synchronize()
    assert_same((out.cpu().numpy(), cells.cpu().numpy()), run_oracle(b, wl.scoring), "two-step")


def _to_ascii(codes, rng):
    """Base codes as raw read letters: A/C/G/T in random case, N as an
    assortment of other bytes (N, n, IUPAC letters, '-', '.')."""
    upper = np.frombuffer(b"ACGT", np.uint8)
    lower = np.frombuffer(b"acgt", np.uint8)
    other = np.frombuffer(b"NnRYKMSWBDHV-.", np.uint8)
    out = np.where(rng.random(codes.size) < 0.5, upper[np.minimum(codes, 3)],
                   lower[np.minimum(codes, 3)]).astype(np.uint8)
    n = codes >= 4
    out[n] = other[rng.integers(0, other.size, int(n.sum()))]
    return out


@pytest.mark.parametrize("shift", [0, 1])
def test_ascii_reads(ctx, shift):
    # raw reads go through the on-GPU packing pass; results equal the oracle
    # on the base codes; shift = 1 starts both buffers one byte off (the
    # conversion's byte path)
    import torch
    import paper_2301_09310_gb300 as xt
    rng = np.random.default_rng(99 + shift)
    wl = synth.WORKLOADS["c3_mixed"]
    b = synth.generate(wl, n=4000, first=555)
    fz = fuzz_batch(21, 600, max_len=80, tail=40)
    other = xt.Context(0)
    try:
        other.set_alphabet(xt.XT_ALPHABET_ASCII)
        for batch, sc in ((b, wl.scoring), (fz, SCORINGS[3])):
            want = run_oracle(batch, sc)
            qa = np.concatenate([np.zeros(shift, np.uint8), _to_ascii(batch.q_seq, rng)])
            ta = np.concatenate([np.zeros(shift, np.uint8), _to_ascii(batch.t_seq, rng)])
            dev = torch.device("cuda", 0)
            T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
            qd, td = T(qa)[shift:], T(ta)[shift:]
            args = (qd, T(batch.q_off), T(batch.q_len), td, T(batch.t_off), T(batch.t_len),
                    T(batch.h0))
            for plain in (False, True):
                out, cells = other.extend(*args, sc, plain=plain)
                torch.cuda.synchronize()
                assert_same((out.cpu().numpy(), cells.cpu().numpy()), want,
                            f"ascii shift={shift} plain={plain}")
    finally:
        other.close()


def _odd_start(batch):
    """The same pairs with every sequence moved one base later in its buffer,
    so half of them start on the high nibble of a byte in the 4-bit layout."""
    from paper_2301_09310_gb300.synth import Batch
    return Batch(np.concatenate([np.full(1, 2, np.uint8), batch.q_seq]), batch.q_off + 1,
                 batch.q_len, np.concatenate([np.full(1, 3, np.uint8), batch.t_seq]),
                 batch.t_off + 1, batch.t_len, batch.h0)


@pytest.mark.parametrize("odd", [0, 1])
def test_packed4_reads(ctx, odd):
    # two 4-bit codes per byte, unpacked on the GPU: batched, plain and
    # BWA-compatible calls equal the oracle on the base codes
    import torch
    import oracle
    import paper_2301_09310_gb300 as xt
    from paper_2301_09310_gb300.synth import BwaScoringParams
    wl = synth.WORKLOADS["c3_mixed"]
    batches = [(synth.generate(wl, n=4000, first=777), wl.scoring),
               (fuzz_batch(23, 600, max_len=80, tail=40), SCORINGS[3])]
    other = xt.Context(0)
    try:
        other.set_alphabet(xt.XT_ALPHABET_PACKED4)
        dev = torch.device("cuda", 0)
        T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
        for batch, sc in batches:
            if odd:
                batch = _odd_start(batch)
            want = run_oracle(batch, sc)
            args = (T(xt.pack4(batch.q_seq)), T(batch.q_off), T(batch.q_len),
                    T(xt.pack4(batch.t_seq)), T(batch.t_off), T(batch.t_len), T(batch.h0))
            for plain in (False, True):
                out, cells = other.extend(*args, sc, plain=plain)
                torch.cuda.synchronize()
                assert_same((out.cpu().numpy(), cells.cpu().numpy()), want,
                            f"packed4 odd={odd} plain={plain}")
            bsc = BwaScoringParams.from_scoring(sc)
            out, cells = other.extend_bwa(*args, bsc)
            torch.cuda.synchronize()
            bwant = oracle.extend_batch_bwa(batch.q_seq, batch.q_off, batch.q_len, batch.t_seq,
                                            batch.t_off, batch.t_len, batch.h0,
                                            oracle.BwaScoring(*bsc.as_tuple()))
            assert_same((out.cpu().numpy(), cells.cpu().numpy()), bwant, f"packed4 bwa odd={odd}")
    finally:
        other.close()


def test_packed4_host_chunks_equal_codes():
    # 2.1M pairs on host buffers: the call runs in chunks, copies packed
    # bytes (half of the codes) and unpacks each chunk's bytes on the GPU;
    # every result equals the same call on base codes
    import paper_2301_09310_gb300 as xt
    wl = synth.WORKLOADS["c2_short"]
    b = synth.generate(wl, n=2_100_000)
    sub = np.arange(0, b.n, 700)
    want_sub = run_oracle(b.take(sub), wl.scoring)
    res = {}
    for alphabet in (xt.XT_ALPHABET_CODES, xt.XT_ALPHABET_PACKED4):
        c = xt.Context(0)
        try:
            c.set_alphabet(alphabet)
            q = b.q_seq if alphabet == xt.XT_ALPHABET_CODES else xt.pack4(b.q_seq)
            t = b.t_seq if alphabet == xt.XT_ALPHABET_CODES else xt.pack4(b.t_seq)
            res[alphabet] = c.extend_host(q, b.q_off, b.q_len, t, b.t_off, b.t_len, b.h0,
                                          wl.scoring)
        finally:
            c.close()
    (oc, cc), (op, cp) = res[xt.XT_ALPHABET_CODES], res[xt.XT_ALPHABET_PACKED4]
    assert np.array_equal(oc, op) and np.array_equal(cc, cp)
    assert_same((op[sub], cp[sub]), want_sub, "packed4 host chunks vs oracle")
