"""The allocation-free entry point, xt_extend_batch_static.

It is meant for callers that may not allocate device memory themselves (code
inside another framework's memory pool, a process that reserved the device
memory up front, an allocator-free hot loop).  This file checks, through the
C ABI, that it returns exactly what xt_extend_batch returns on the same
inputs, on two calls in a row that share its fixed scratch array, and that it
refuses work beyond its limits.  It is collected last, so a run that stops at
the first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

from paper_2301_09310_gb300 import synth
from paper_2301_09310_gb300.synth import ScoringParams

from tests.gpu_util import fuzz_batch, to_dev

pytestmark = pytest.mark.gpu


def _static_call(args, n, sc, stream):
    import torch
    import paper_2301_09310_gb300 as xt
    q_seq, q_off, q_len, t_seq, t_off, t_len, h0 = args
    out = torch.full((n, 7), -7, dtype=torch.int32, device=q_len.device)
    cells = torch.full((n,), -7, dtype=torch.int64, device=q_len.device)
    s = xt.xt_extend_batch_static(q_seq.data_ptr(), q_seq.numel(), q_off.data_ptr(),
                                  q_len.data_ptr(), t_seq.data_ptr(), t_seq.numel(),
                                  t_off.data_ptr(), t_len.data_ptr(), h0.data_ptr(), n, sc,
                                  out.data_ptr(), cells.data_ptr(), stream.cuda_stream)
    return s, out, cells


def test_static_matches_batched_on_two_calls():
    import torch
    import paper_2301_09310_gb300 as xt
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    wl = synth.WORKLOADS["c3_mixed"]
    batches = [(synth.generate(wl, n=30000), wl.scoring),
               (fuzz_batch(21, 4000, max_len=120, tail=80), ScoringParams(w=12, zdrop=20))]
    ctx = xt.Context(0)
    try:
        refs = []
        for b, sc in batches:
            args = to_dev(b, dev)
            out, cells = ctx.extend(*args, sc)
            torch.cuda.synchronize()
            refs.append((args, b.n, sc, out.cpu().numpy(), cells.cpu().numpy()))
        free_before = None
        for k, (args, n, sc, want_out, want_cells) in enumerate(refs):
            if k == 1:
                free_before = torch.cuda.mem_get_info(dev)[0]
            s, out, cells = _static_call(args, n, sc, stream)
            assert s == xt.XT_OK, xt.xt_status_str(s)
            torch.cuda.synchronize()
            assert np.array_equal(out.cpu().numpy(), want_out), f"call {k}: results differ"
            assert np.array_equal(cells.cpu().numpy(), want_cells), f"call {k}: cells differ"
        # the second call took no device memory
        assert torch.cuda.mem_get_info(dev)[0] == free_before
    finally:
        ctx.close()


def test_static_refuses_beyond_limits():
    import torch
    import paper_2301_09310_gb300 as xt
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    b = fuzz_batch(22, 16)
    args = to_dev(b, dev)
    # more pairs than the fixed scratch holds: refused before anything runs
    s, _, _ = _static_call(args, xt.XT_STATIC_MAX_PAIRS + 1, ScoringParams(), stream)
    assert s == xt.XT_EINVAL
    # a band too wide for shared-memory rings needs the context's ring pool
    s, _, _ = _static_call(args, b.n, ScoringParams(w=5000), stream)
    assert s == xt.XT_EINVAL
    # the same small batch within the limits runs
    s, out, _ = _static_call(args, b.n, ScoringParams(), stream)
    torch.cuda.synchronize()
    assert s == xt.XT_OK and int(out[:, 6].max().item()) <= 1


def test_static_at_its_pair_limit():
    """XT_STATIC_MAX_PAIRS short pairs: the carved tables come closest to the
    end of the fixed array; results equal xt_extend_batch's."""
    import torch
    import paper_2301_09310_gb300 as xt
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    n = xt.XT_STATIC_MAX_PAIRS
    wl = synth.WORKLOADS["c2_short"]
    b = synth.generate(wl, n=n)
    sc = wl.scoring
    args = to_dev(b, dev)
    ctx = xt.Context(0)
    try:
        want_out, want_cells = ctx.extend(*args, sc)
        torch.cuda.synchronize()
        want_out, want_cells = want_out.cpu().numpy(), want_cells.cpu().numpy()
    finally:
        ctx.close()
    for k in range(2):
        s, out, cells = _static_call(args, n, sc, stream)
        assert s == xt.XT_OK, xt.xt_status_str(s)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), want_out), f"call {k}: results differ"
        assert np.array_equal(cells.cpu().numpy(), want_cells), f"call {k}: cells differ"


def _capture_static(graph, args, n, sc, out, cells, stream):
    """Capture one static call into `graph`; the call's host-side arguments
    (its batch descriptor included) live in this frame only."""
    import torch
    import paper_2301_09310_gb300 as xt
    q_seq, q_off, q_len, t_seq, t_off, t_len, h0 = args
    with torch.cuda.graph(graph, stream=stream, capture_error_mode="thread_local"):
        s = xt.xt_extend_batch_static(q_seq.data_ptr(), q_seq.numel(), q_off.data_ptr(),
                                      q_len.data_ptr(), t_seq.data_ptr(), t_seq.numel(),
                                      t_off.data_ptr(), t_len.data_ptr(), h0.data_ptr(), n, sc,
                                      out.data_ptr(), cells.data_ptr(), stream.cuda_stream)
    return s


def test_static_replays_from_a_captured_graph():
    # the documented use under stream capture: a first call outside capture,
    # then a captured call whose graph replays after the capturing frame is gone
    import torch
    import paper_2301_09310_gb300 as xt
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    wl = synth.WORKLOADS["c3_mixed"]
    b = synth.generate(wl, n=20000)
    args = to_dev(b, dev)
    ctx = xt.Context(0)
    try:
        want_out, want_cells = ctx.extend(*args, wl.scoring)
        torch.cuda.synchronize()
        want_out, want_cells = want_out.cpu().numpy(), want_cells.cpu().numpy()
    finally:
        ctx.close()
    stream = torch.cuda.Stream(dev)
    s, _, _ = _static_call(args, b.n, wl.scoring, stream)
    assert s == xt.XT_OK, xt.xt_status_str(s)
    torch.cuda.synchronize()
    out = torch.empty((b.n, 7), dtype=torch.int32, device=dev)
    cells = torch.empty(b.n, dtype=torch.int64, device=dev)
    graph = torch.cuda.CUDAGraph()
    s = _capture_static(graph, args, b.n, wl.scoring, out, cells, stream)
    assert s == xt.XT_OK, xt.xt_status_str(s)
    for k in range(2):
        out.fill_(-7)
        cells.fill_(-7)
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), want_out), f"replay {k}: results differ"
        assert np.array_equal(cells.cpu().numpy(), want_cells), f"replay {k}: cells differ"
