"""Batched seed extension on GB300: Python binding of the libxt C ABI.

Argument marshalling only.  Every step of the extension runs in the CUDA
kernels of libxt (csrc/); there is no CPU implementation here and no
fallback: if the library is not built or no GPU is present, calls raise.
The functions carry the C names of include/xt.h (xt_ctx_create,
xt_extend_batch, ...); ``Context`` is a small convenience wrapper over them
taking torch CUDA tensors.
"""
from __future__ import annotations

import ctypes
import os
import time
from dataclasses import dataclass

from . import build as _build

XT_OK, XT_EINVAL, XT_ENOMEM, XT_ECUDA, XT_ETIMEOUT, XT_EBUSY = range(6)
XT_MAX_LEN = 1 << 20
XT_MAX_H0 = 1 << 20
RESULT_FIELDS = ("score", "qle", "tle", "gscore", "gtle", "max_off", "status")

EXPORTED = ("xt_ctx_create", "xt_ctx_destroy", "xt_ctx_sync", "xt_extend_batch",
            "xt_extend_batch_plain", "xt_extend_batch_host", "xt_status_str",
            "xt_ctx_last_error", "xt_ctx_set_schedule", "xt_ctx_set_timing", "xt_ctx_stats",
            "xt_extend_batch_static", "xt_ctx_set_graphs", "xt_scoring_check", "xt_now_ns",
            "xt_serve_create", "xt_serve_submit", "xt_serve_poll", "xt_serve_wait",
            "xt_serve_pause", "xt_serve_get_stats", "xt_serve_destroy", "xt_ctx_set_streams",
            "xt_ctx_set_bucket_schedule", "xt_ctx_get_bucket_schedule", "xt_autotune",
            "xt_ctx_load_tuning", "xt_ctx_set_bucket_schedule_for",
            "xt_ctx_get_bucket_schedule_for", "xt_extend_batch_begin", "xt_extend_batch_ready",
            "xt_extend_batch_finish", "xt_ctx_set_alphabet", "xt_extend_seeds",
            "xt_extend_batch_bwa", "xt_bwa_scoring_check", "xt_int_rate", "xt_shard_lpt")
XT_STATIC_MAX_PAIRS = 1 << 20
# instruction kinds of xt_int_rate (measurement aid)
XT_RATE_ADD16X2, XT_RATE_MAX3_16X2, XT_RATE_ADDMAX_16X2, XT_RATE_PRMT = 0, 1, 2, 3
XT_RATE_IADD3, XT_RATE_MAX3_32, XT_RATE_IMAD, XT_RATE_MIX, XT_RATE_CELL_P16 = 4, 5, 6, 7, 8
XT_RATE_HMAX2 = 9
RATE_NAMES = {XT_RATE_ADD16X2: "add.s16x2", XT_RATE_MAX3_16X2: "max3.s16x2",
              XT_RATE_ADDMAX_16X2: "addmax.relu.s16x2", XT_RATE_PRMT: "prmt",
              XT_RATE_IADD3: "iadd3.s32", XT_RATE_MAX3_32: "max3.s32", XT_RATE_IMAD: "imad.u32",
              XT_RATE_MIX: "max3.s16x2 + add.s16x2 by chain",
              XT_RATE_CELL_P16: "packed cell update (cells)",
              XT_RATE_HMAX2: "max.f16x2"}


class xt_scoring(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("match", "mismatch", "gap_open", "gap_extend", "w", "zdrop", "n_score")]


class xt_bwa_scoring(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("match", "mismatch", "n_score", "o_del", "e_del", "o_ins", "e_ins", "w", "zdrop",
                 "end_bonus")]


XT_BWA_MAX_WIDTH = 8192


class xt_stats(ctypes.Structure):
    _fields_ = [("calls", ctypes.c_int32), ("launches", ctypes.c_int32),
                ("dp_launches", ctypes.c_int32), ("timed_calls", ctypes.c_int32),
                ("dp_ms", ctypes.c_double)]


class xt_serve_config(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("max_batch_pairs", ctypes.c_int32),
                ("max_batch_bytes", ctypes.c_int64), ("max_queued_bytes", ctypes.c_int64),
                ("mem_budget_bytes", ctypes.c_size_t), ("gather_threads", ctypes.c_int32),
                ("tuning_path", ctypes.c_char_p), ("alphabet", ctypes.c_int32)]


class xt_serve_times(ctypes.Structure):
    _fields_ = [("submit_ns", ctypes.c_int64), ("launch_ns", ctypes.c_int64),
                ("done_ns", ctypes.c_int64), ("batch_pairs", ctypes.c_int32),
                ("status", ctypes.c_int32)]


class xt_serve_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in
                ("requests", "pairs", "cells", "batches", "waiting", "in_flight",
                 "gather_ns", "device_ns")]


class XtError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        self.status = status
        super().__init__(f"{_status_name(status)}: {msg}" if msg else _status_name(status))


_LIB = None


def _status_name(s: int) -> str:
    names = ["XT_OK", "XT_EINVAL", "XT_ENOMEM", "XT_ECUDA", "XT_ETIMEOUT", "XT_EBUSY"]
    return names[s] if 0 <= s < len(names) else f"XT_STATUS_{s}"


def lib_path() -> str:
    return _build.lib_path()


def load_library(path: str | None = None):
    """Load libxt (built by build.build()); raises if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libxt is not built ({path} missing): run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    batch_args = [P, P, I64, P, P, P, I64, P, P, P, I32, ctypes.POINTER(xt_scoring), P, P, P]
    lib.xt_ctx_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.c_size_t]
    lib.xt_ctx_destroy.argtypes = [P]
    lib.xt_ctx_sync.argtypes = [P, P]
    for fn in ("xt_extend_batch", "xt_extend_batch_plain", "xt_extend_batch_host",
               "xt_extend_batch_begin"):
        getattr(lib, fn).argtypes = batch_args
    lib.xt_extend_batch_begin.restype = ctypes.c_int
    lib.xt_extend_batch_ready.argtypes = [P, ctypes.POINTER(ctypes.c_int)]
    lib.xt_extend_batch_ready.restype = ctypes.c_int
    lib.xt_extend_batch_finish.argtypes = [P]
    lib.xt_extend_batch_finish.restype = ctypes.c_int
    for fn in ("xt_ctx_create", "xt_ctx_destroy", "xt_ctx_sync", "xt_extend_batch",
               "xt_extend_batch_plain", "xt_extend_batch_host"):
        getattr(lib, fn).restype = ctypes.c_int
    lib.xt_status_str.argtypes = [ctypes.c_int]
    lib.xt_status_str.restype = ctypes.c_char_p
    lib.xt_ctx_set_schedule.argtypes = [P, ctypes.c_int, ctypes.c_int]
    lib.xt_ctx_set_schedule.restype = ctypes.c_int
    lib.xt_extend_batch_static.argtypes = batch_args[1:]
    lib.xt_extend_batch_static.restype = ctypes.c_int
    lib.xt_ctx_set_graphs.argtypes = [P, ctypes.c_int]
    lib.xt_ctx_set_graphs.restype = ctypes.c_int
    lib.xt_ctx_set_bucket_schedule.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int]
    lib.xt_ctx_get_bucket_schedule.argtypes = [P, ctypes.c_int, ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(ctypes.c_int)]
    lib.xt_ctx_set_bucket_schedule_for.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_int, ctypes.c_int]
    lib.xt_ctx_get_bucket_schedule_for.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   ctypes.POINTER(ctypes.c_int),
                                                   ctypes.POINTER(ctypes.c_int)]
    lib.xt_ctx_set_bucket_schedule_for.restype = ctypes.c_int
    lib.xt_ctx_get_bucket_schedule_for.restype = ctypes.c_int
    lib.xt_autotune.argtypes = [P, ctypes.POINTER(xt_scoring), ctypes.c_int, ctypes.c_double,
                                ctypes.c_char_p]
    lib.xt_ctx_load_tuning.argtypes = [P, ctypes.c_char_p]
    for fn in ("xt_ctx_set_bucket_schedule", "xt_ctx_get_bucket_schedule", "xt_autotune",
               "xt_ctx_load_tuning"):
        getattr(lib, fn).restype = ctypes.c_int
    lib.xt_extend_seeds.argtypes = [P, P, I64, P, P, P, I64, P, P, P, P, P, P, I32,
                                    ctypes.POINTER(xt_scoring), P, P, P, P, P]
    lib.xt_extend_seeds.restype = ctypes.c_int
    lib.xt_extend_batch_bwa.argtypes = batch_args[:11] + [ctypes.POINTER(xt_bwa_scoring), P, P, P]
    lib.xt_extend_batch_bwa.restype = ctypes.c_int
    lib.xt_bwa_scoring_check.argtypes = [ctypes.POINTER(xt_bwa_scoring)]
    lib.xt_bwa_scoring_check.restype = ctypes.c_int
    lib.xt_ctx_set_alphabet.argtypes = [P, ctypes.c_int]
    lib.xt_ctx_set_alphabet.restype = ctypes.c_int
    lib.xt_ctx_set_streams.argtypes = [P, ctypes.c_int]
    lib.xt_ctx_set_streams.restype = ctypes.c_int
    lib.xt_ctx_set_timing.argtypes = [P, ctypes.c_int]
    lib.xt_ctx_set_timing.restype = ctypes.c_int
    lib.xt_ctx_stats.argtypes = [P, ctypes.POINTER(xt_stats)]
    lib.xt_ctx_stats.restype = ctypes.c_int
    lib.xt_ctx_last_error.argtypes = [P]
    lib.xt_ctx_last_error.restype = ctypes.c_char_p
    lib.xt_scoring_check.argtypes = [ctypes.POINTER(xt_scoring)]
    lib.xt_scoring_check.restype = ctypes.c_int
    lib.xt_int_rate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]
    lib.xt_int_rate.restype = ctypes.c_int
    lib.xt_shard_lpt.argtypes = [P, P, I32, I32, I32, P, P]
    lib.xt_shard_lpt.restype = ctypes.c_int
    lib.xt_now_ns.argtypes = []
    lib.xt_now_ns.restype = ctypes.c_int64
    lib.xt_serve_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(xt_serve_config)]
    lib.xt_serve_submit.argtypes = [P] + batch_args[1:-1] + [ctypes.POINTER(ctypes.c_uint64)]
    lib.xt_serve_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)]
    lib.xt_serve_wait.argtypes = [P, ctypes.c_uint64, ctypes.c_int64,
                                  ctypes.POINTER(xt_serve_times)]
    lib.xt_serve_pause.argtypes = [P, ctypes.c_int]
    lib.xt_serve_get_stats.argtypes = [P, ctypes.POINTER(xt_serve_stats)]
    lib.xt_serve_destroy.argtypes = [P]
    for fn in ("xt_serve_create", "xt_serve_submit", "xt_serve_poll", "xt_serve_wait",
               "xt_serve_pause", "xt_serve_get_stats", "xt_serve_destroy", "xt_ctx_set_streams",
            "xt_ctx_set_bucket_schedule", "xt_ctx_get_bucket_schedule", "xt_autotune",
            "xt_ctx_load_tuning", "xt_ctx_set_bucket_schedule_for",
            "xt_ctx_get_bucket_schedule_for", "xt_extend_batch_begin", "xt_extend_batch_ready",
            "xt_extend_batch_finish", "xt_ctx_set_alphabet", "xt_extend_seeds"):
        getattr(lib, fn).restype = ctypes.c_int
    _LIB = lib
    return lib


# ------------------------------------------------------------ C-ABI mirrors
def xt_ctx_create(device: int = 0, mem_budget_bytes: int = 0) -> int:
    h = ctypes.c_void_p()
    s = load_library().xt_ctx_create(ctypes.byref(h), int(device), int(mem_budget_bytes))
    if s != XT_OK:
        raise XtError(s, "xt_ctx_create")
    return h.value


def xt_ctx_destroy(ctx: int) -> int:
    return load_library().xt_ctx_destroy(ctypes.c_void_p(ctx))


def xt_ctx_sync(ctx: int, stream: int = 0) -> int:
    return load_library().xt_ctx_sync(ctypes.c_void_p(ctx), ctypes.c_void_p(stream))


def xt_ctx_set_schedule(ctx: int, P: int, R: int) -> int:
    return load_library().xt_ctx_set_schedule(ctypes.c_void_p(ctx), int(P), int(R))


def xt_ctx_set_graphs(ctx: int, enable: bool) -> int:
    return load_library().xt_ctx_set_graphs(ctypes.c_void_p(ctx), int(bool(enable)))


def xt_ctx_set_bucket_schedule(ctx: int, w: int, j: int, P: int, R: int) -> int:
    return load_library().xt_ctx_set_bucket_schedule(ctypes.c_void_p(ctx), int(w), int(j), int(P),
                                                     int(R))


def xt_ctx_get_bucket_schedule(ctx: int, w: int, j: int) -> tuple[int, int, int]:
    P, R = ctypes.c_int(0), ctypes.c_int(0)
    s = load_library().xt_ctx_get_bucket_schedule(ctypes.c_void_p(ctx), int(w), int(j),
                                                  ctypes.byref(P), ctypes.byref(R))
    return s, P.value, R.value


XT_BATCH_LARGE, XT_BATCH_SMALL, XT_SMALL_BUCKET = 0, 1, 8192


def xt_ctx_set_bucket_schedule_for(ctx: int, w: int, j: int, batch_class: int, P: int,
                                   R: int) -> int:
    return load_library().xt_ctx_set_bucket_schedule_for(ctypes.c_void_p(ctx), int(w), int(j),
                                                         int(batch_class), int(P), int(R))


def xt_ctx_get_bucket_schedule_for(ctx: int, w: int, j: int,
                                   batch_class: int) -> tuple[int, int, int]:
    P, R = ctypes.c_int(0), ctypes.c_int(0)
    s = load_library().xt_ctx_get_bucket_schedule_for(ctypes.c_void_p(ctx), int(w), int(j),
                                                      int(batch_class), ctypes.byref(P),
                                                      ctypes.byref(R))
    return s, P.value, R.value


def xt_autotune(ctx: int, sc, j_max: int = 14, cells_per_trial: float = 0.0,
                table_path: str | None = None) -> int:
    return load_library().xt_autotune(ctypes.c_void_p(ctx), ctypes.byref(_scoring(sc)), int(j_max),
                                      float(cells_per_trial),
                                      table_path.encode() if table_path else None)


def xt_ctx_load_tuning(ctx: int, table_path: str) -> int:
    return load_library().xt_ctx_load_tuning(ctypes.c_void_p(ctx), table_path.encode())


XT_ALPHABET_CODES, XT_ALPHABET_ASCII, XT_ALPHABET_PACKED4 = 0, 1, 2


def pack4(codes):
    """Host-side packing of base codes into the 4-bit layout of
    XT_ALPHABET_PACKED4: base p is the low nibble of byte p // 2 when p is
    even and the high nibble when p is odd (codes above 15 become 15, N).
    Offsets and lengths of the pairs stay in bases."""
    import numpy as np
    c = np.minimum(np.asarray(codes, np.uint8), 15)
    if c.size % 2:
        c = np.concatenate([c, np.zeros(1, np.uint8)])
    return (c[0::2] | (c[1::2] << 4)).astype(np.uint8)


def xt_ctx_set_alphabet(ctx: int, alphabet: int) -> int:
    return load_library().xt_ctx_set_alphabet(ctypes.c_void_p(ctx), int(alphabet))


def xt_ctx_set_streams(ctx: int, branches: int) -> int:
    return load_library().xt_ctx_set_streams(ctypes.c_void_p(ctx), int(branches))


def xt_shard_lpt(q_len, t_len, w: int, parts: int):
    """(shard int32[n], part_cells int64[parts]): the LPT split of a batch
    over `parts` devices by estimated cells (host arrays in, host arrays out)."""
    import numpy as np
    ql = np.ascontiguousarray(q_len, np.int32)
    tl = np.ascontiguousarray(t_len, np.int32)
    if ql.shape != tl.shape:
        raise ValueError("q_len and t_len differ in length")
    shard = np.empty(ql.size, np.int32)
    cells = np.empty(max(int(parts), 1), np.int64)
    s = load_library().xt_shard_lpt(ql.ctypes.data, tl.ctypes.data, int(ql.size), int(w),
                                    int(parts), shard.ctypes.data, cells.ctypes.data)
    if s != XT_OK:
        raise XtError(s, "xt_shard_lpt")
    return shard, cells


def xt_int_rate(device: int, op: int, reps: int = 3):
    """(status, units, ms): one instruction kind's throughput probe."""
    units, ms = ctypes.c_int64(0), ctypes.c_double(0.0)
    s = load_library().xt_int_rate(int(device), int(op), int(reps), ctypes.byref(units),
                                   ctypes.byref(ms))
    return s, units.value, ms.value


def xt_ctx_set_timing(ctx: int, enable: bool) -> int:
    return load_library().xt_ctx_set_timing(ctypes.c_void_p(ctx), int(bool(enable)))


def xt_ctx_stats(ctx: int) -> xt_stats:
    st = xt_stats()
    s = load_library().xt_ctx_stats(ctypes.c_void_p(ctx), ctypes.byref(st))
    if s != XT_OK:
        raise XtError(s, "xt_ctx_stats")
    return st


def xt_scoring_check(sc) -> int:
    return load_library().xt_scoring_check(ctypes.byref(_scoring(sc)))


def xt_now_ns() -> int:
    """The serving loop's clock (CLOCK_MONOTONIC, ns)."""
    return load_library().xt_now_ns()


def xt_serve_create(device: int = 0, cfg: xt_serve_config | None = None) -> int:
    h = ctypes.c_void_p()
    s = load_library().xt_serve_create(ctypes.byref(h), int(device),
                                       ctypes.byref(cfg) if cfg is not None else None)
    if s != XT_OK:
        raise XtError(s, "xt_serve_create")
    return h.value


def xt_serve_submit(server, q_seq, q_bytes, q_off, q_len, t_seq, t_bytes, t_off, t_len, h0, n, sc,
                    out, cells) -> tuple[int, int]:
    """Raw host pointers (ints) as in include/xt.h; returns (xt_status, ticket)."""
    ticket = ctypes.c_uint64(0)
    s = load_library().xt_serve_submit(
        ctypes.c_void_p(server), ctypes.c_void_p(q_seq), int(q_bytes), ctypes.c_void_p(q_off),
        ctypes.c_void_p(q_len), ctypes.c_void_p(t_seq), int(t_bytes), ctypes.c_void_p(t_off),
        ctypes.c_void_p(t_len), ctypes.c_void_p(h0), int(n), ctypes.byref(_scoring(sc)),
        ctypes.c_void_p(out), ctypes.c_void_p(cells), ctypes.byref(ticket))
    return s, ticket.value


def xt_serve_poll(server, ticket: int) -> tuple[int, bool]:
    done = ctypes.c_int(0)
    s = load_library().xt_serve_poll(ctypes.c_void_p(server), ticket, ctypes.byref(done))
    return s, bool(done.value)


def xt_serve_wait(server, ticket: int, timeout_us: int = -1) -> tuple[int, xt_serve_times]:
    t = xt_serve_times()
    s = load_library().xt_serve_wait(ctypes.c_void_p(server), ticket, int(timeout_us),
                                     ctypes.byref(t))
    return s, t


def xt_serve_pause(server, paused: bool) -> int:
    return load_library().xt_serve_pause(ctypes.c_void_p(server), int(bool(paused)))


def xt_serve_get_stats(server) -> xt_serve_stats:
    st = xt_serve_stats()
    s = load_library().xt_serve_get_stats(ctypes.c_void_p(server), ctypes.byref(st))
    if s != XT_OK:
        raise XtError(s, "xt_serve_get_stats")
    return st


def xt_serve_destroy(server) -> int:
    return load_library().xt_serve_destroy(ctypes.c_void_p(server))


def xt_status_str(s: int) -> str:
    return load_library().xt_status_str(int(s)).decode()


def xt_ctx_last_error(ctx: int) -> str:
    return load_library().xt_ctx_last_error(ctypes.c_void_p(ctx)).decode()


def _call(fn: str, ctx, q_seq, q_bytes, q_off, q_len, t_seq, t_bytes, t_off, t_len, h0, n,
          sc: xt_scoring, out, cells, stream) -> int:
    f = getattr(load_library(), fn)
    return f(ctypes.c_void_p(ctx), ctypes.c_void_p(q_seq), int(q_bytes), ctypes.c_void_p(q_off),
             ctypes.c_void_p(q_len), ctypes.c_void_p(t_seq), int(t_bytes), ctypes.c_void_p(t_off),
             ctypes.c_void_p(t_len), ctypes.c_void_p(h0), int(n), ctypes.byref(sc),
             ctypes.c_void_p(out), ctypes.c_void_p(cells), ctypes.c_void_p(stream))


def xt_extend_batch(ctx, q_seq, q_bytes, q_off, q_len, t_seq, t_bytes, t_off, t_len, h0, n, sc,
                    out, cells, stream) -> int:
    """Raw pointers (ints) as in include/xt.h; returns the xt_status."""
    return _call("xt_extend_batch", ctx, q_seq, q_bytes, q_off, q_len, t_seq, t_bytes, t_off,
                 t_len, h0, n, sc, out, cells, stream)


def xt_extend_batch_plain(ctx, q_seq, q_bytes, q_off, q_len, t_seq, t_bytes, t_off, t_len, h0, n,
                          sc, out, cells, stream) -> int:
    return _call("xt_extend_batch_plain", ctx, q_seq, q_bytes, q_off, q_len, t_seq, t_bytes, t_off,
                 t_len, h0, n, sc, out, cells, stream)


def xt_extend_batch_host(ctx, q_seq, q_bytes, q_off, q_len, t_seq, t_bytes, t_off, t_len, h0, n,
                         sc, out, cells, stream) -> int:
    return _call("xt_extend_batch_host", ctx, q_seq, q_bytes, q_off, q_len, t_seq, t_bytes, t_off,
                 t_len, h0, n, sc, out, cells, stream)


def xt_extend_seeds(ctx, q_seq, q_bytes, q_off, q_len, t_seq, t_bytes, t_off, t_len, q_beg, t_beg,
                    seed_len, h0, n, sc, left, right, left_cells, right_cells, stream) -> int:
    """Both-direction extension of seeds; raw device pointers as in include/xt.h."""
    V = ctypes.c_void_p
    return load_library().xt_extend_seeds(
        V(ctx), V(q_seq), int(q_bytes), V(q_off), V(q_len), V(t_seq), int(t_bytes), V(t_off),
        V(t_len), V(q_beg), V(t_beg), V(seed_len), V(h0), int(n), ctypes.byref(_scoring(sc)),
        V(left), V(right), V(left_cells), V(right_cells), V(stream))


def _bwa_scoring(sc) -> xt_bwa_scoring:
    if isinstance(sc, xt_bwa_scoring):
        return sc
    if hasattr(sc, "as_tuple"):
        return xt_bwa_scoring(*sc.as_tuple())
    return xt_bwa_scoring(*sc)


def xt_bwa_scoring_check(sc) -> int:
    return load_library().xt_bwa_scoring_check(ctypes.byref(_bwa_scoring(sc)))


def xt_extend_batch_bwa(ctx, q_seq, q_bytes, q_off, q_len, t_seq, t_bytes, t_off, t_len, h0, n,
                        sc, out, cells, stream) -> int:
    """BWA-MEM-compatible extension; raw device pointers as in include/xt.h."""
    V = ctypes.c_void_p
    return load_library().xt_extend_batch_bwa(
        V(ctx), V(q_seq), int(q_bytes), V(q_off), V(q_len), V(t_seq), int(t_bytes), V(t_off),
        V(t_len), V(h0), int(n), ctypes.byref(_bwa_scoring(sc)), V(out), V(cells), V(stream))


def xt_extend_batch_begin(ctx, q_seq, q_bytes, q_off, q_len, t_seq, t_bytes, t_off, t_len, h0, n,
                          sc, out, cells, stream) -> int:
    return _call("xt_extend_batch_begin", ctx, q_seq, q_bytes, q_off, q_len, t_seq, t_bytes,
                 t_off, t_len, h0, n, sc, out, cells, stream)


def xt_extend_batch_ready(ctx) -> tuple[int, bool]:
    r = ctypes.c_int(0)
    s = load_library().xt_extend_batch_ready(ctypes.c_void_p(ctx), ctypes.byref(r))
    return s, bool(r.value)


def xt_extend_batch_finish(ctx) -> int:
    return load_library().xt_extend_batch_finish(ctypes.c_void_p(ctx))


def xt_extend_batch_static(q_seq, q_bytes, q_off, q_len, t_seq, t_bytes, t_off, t_len, h0, n, sc,
                           out, cells, stream) -> int:
    """Allocation-free batched extension on the current device (no context):
    for callers that may not allocate device memory.  Raw device pointers as
    in include/xt.h; returns the xt_status.  Calls share one fixed scratch
    array inside the library, so calls must not overlap on the GPU."""
    return load_library().xt_extend_batch_static(
        ctypes.c_void_p(q_seq), int(q_bytes), ctypes.c_void_p(q_off), ctypes.c_void_p(q_len),
        ctypes.c_void_p(t_seq), int(t_bytes), ctypes.c_void_p(t_off), ctypes.c_void_p(t_len),
        ctypes.c_void_p(h0), int(n), ctypes.byref(_scoring(sc)), ctypes.c_void_p(out),
        ctypes.c_void_p(cells), ctypes.c_void_p(stream))


# ------------------------------------------------------------ convenience
@dataclass(frozen=True)
class Scoring:
    match: int = 1
    mismatch: int = -4
    gap_open: int = 6
    gap_extend: int = 1
    w: int = 100
    zdrop: int = 100
    n_score: int = -1

    def c(self) -> xt_scoring:
        return xt_scoring(self.match, self.mismatch, self.gap_open, self.gap_extend, self.w,
                          self.zdrop, self.n_score)


def _scoring(sc) -> xt_scoring:
    if isinstance(sc, xt_scoring):
        return sc
    if hasattr(sc, "as_tuple"):
        return xt_scoring(*sc.as_tuple())
    if hasattr(sc, "c"):
        return sc.c()
    return xt_scoring(*sc)


class Context:
    """A libxt context on one CUDA device, taking torch tensors.

    Inputs are CUDA tensors (uint8 sequences, int64 offsets, int32 lengths and
    h0); results come back as an int32 [n, 7] CUDA tensor (RESULT_FIELDS) and
    an int64 [n] tensor of useful cells.  Work is enqueued on the current torch
    stream unless a stream is given."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0):
        import torch  # noqa: F401  (device memory and streams)
        self.device = int(device)
        self.handle = xt_ctx_create(self.device, mem_budget_bytes)

    def close(self):
        if self.handle:
            xt_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_graphs(self, enable: bool = True):
        self._check(xt_ctx_set_graphs(self.handle, enable), "xt_ctx_set_graphs")

    def set_bucket_schedule(self, w: int, j: int, P: int, R: int = 8):
        self._check(xt_ctx_set_bucket_schedule(self.handle, w, j, P, R),
                    "xt_ctx_set_bucket_schedule")

    def bucket_schedule(self, w: int, j: int, batch_class: int = XT_BATCH_LARGE) -> tuple[int, int]:
        s, P, R = xt_ctx_get_bucket_schedule_for(self.handle, w, j, batch_class)
        self._check(s, "xt_ctx_get_bucket_schedule_for")
        return P, R

    def set_bucket_schedule_for(self, w: int, j: int, batch_class: int, P: int, R: int = 8):
        self._check(xt_ctx_set_bucket_schedule_for(self.handle, w, j, batch_class, P, R),
                    "xt_ctx_set_bucket_schedule_for")

    def autotune(self, scoring, j_max: int = 14, cells_per_trial: float = 0.0,
                 table_path: str | None = None):
        self._check(xt_autotune(self.handle, scoring, j_max, cells_per_trial, table_path),
                    "xt_autotune")

    def load_tuning(self, table_path: str):
        self._check(xt_ctx_load_tuning(self.handle, table_path), "xt_ctx_load_tuning")

    def set_alphabet(self, alphabet: int):
        """XT_ALPHABET_CODES (base codes 0..3), XT_ALPHABET_ASCII (raw letters) or
        XT_ALPHABET_PACKED4 (two 4-bit codes per byte, see pack4)."""
        self._check(xt_ctx_set_alphabet(self.handle, alphabet), "xt_ctx_set_alphabet")

    def set_streams(self, branches: int):
        self._check(xt_ctx_set_streams(self.handle, branches), "xt_ctx_set_streams")

    def set_timing(self, enable: bool = True):
        self._check(xt_ctx_set_timing(self.handle, enable), "xt_ctx_set_timing")

    def stats(self) -> dict:
        st = xt_ctx_stats(self.handle)
        return {f: getattr(st, f) for f, _ in xt_stats._fields_}

    def set_schedule(self, P: int = 0, R: int = 8):
        self._check(xt_ctx_set_schedule(self.handle, P, R), "xt_ctx_set_schedule")

    def _check(self, s: int, what: str):
        if s != XT_OK:
            raise XtError(s, f"{what}: {xt_ctx_last_error(self.handle)}")

    @staticmethod
    def _dev(t, dtype, name):
        import torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda):
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype != dtype:
            raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        return t

    def extend(self, q_seq, q_off, q_len, t_seq, t_off, t_len, h0, scoring, plain=False,
               out=None, cells=None, want_cells=True, stream=None):
        import torch
        d = self._dev
        q_seq = d(q_seq, torch.uint8, "q_seq")
        t_seq = d(t_seq, torch.uint8, "t_seq")
        q_off = d(q_off, torch.int64, "q_off")
        t_off = d(t_off, torch.int64, "t_off")
        q_len = d(q_len, torch.int32, "q_len")
        t_len = d(t_len, torch.int32, "t_len")
        h0 = d(h0, torch.int32, "h0")
        n = int(q_len.numel())
        for name, t in (("q_off", q_off), ("t_off", t_off), ("t_len", t_len), ("h0", h0)):
            if t.numel() != n:
                raise ValueError(f"{name} has {t.numel()} entries, expected {n}")
        dev = q_len.device
        if out is None:
            out = torch.empty((n, 7), dtype=torch.int32, device=dev)
        if cells is None and want_cells:
            cells = torch.empty(n, dtype=torch.int64, device=dev)
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        fn = "xt_extend_batch_plain" if plain else "xt_extend_batch"
        s = _call(fn, self.handle, q_seq.data_ptr(), q_seq.numel(), q_off.data_ptr(),
                  q_len.data_ptr(), t_seq.data_ptr(), t_seq.numel(), t_off.data_ptr(),
                  t_len.data_ptr(), h0.data_ptr(), n, _scoring(scoring), out.data_ptr(),
                  cells.data_ptr() if cells is not None else 0, stream.cuda_stream)
        self._check(s, fn)
        return out, cells

    def extend_bwa(self, q_seq, q_off, q_len, t_seq, t_off, t_len, h0, scoring, out=None,
                   cells=None, want_cells=True, stream=None):
        """BWA-MEM-compatible extension (xt_extend_batch_bwa): the arguments of
        extend(); scoring is an xt_bwa_scoring, a BwaScoringParams or a tuple
        (match, mismatch, n_score, o_del, e_del, o_ins, e_ins, w, zdrop,
        end_bonus)."""
        import torch
        d = self._dev
        q_seq = d(q_seq, torch.uint8, "q_seq")
        t_seq = d(t_seq, torch.uint8, "t_seq")
        q_off = d(q_off, torch.int64, "q_off")
        t_off = d(t_off, torch.int64, "t_off")
        q_len = d(q_len, torch.int32, "q_len")
        t_len = d(t_len, torch.int32, "t_len")
        h0 = d(h0, torch.int32, "h0")
        n = int(q_len.numel())
        for name, t in (("q_off", q_off), ("t_off", t_off), ("t_len", t_len), ("h0", h0)):
            if t.numel() != n:
                raise ValueError(f"{name} has {t.numel()} entries, expected {n}")
        dev = q_len.device
        if out is None:
            out = torch.empty((n, 7), dtype=torch.int32, device=dev)
        if cells is None and want_cells:
            cells = torch.empty(n, dtype=torch.int64, device=dev)
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        s = xt_extend_batch_bwa(self.handle, q_seq.data_ptr(), q_seq.numel(), q_off.data_ptr(),
                                q_len.data_ptr(), t_seq.data_ptr(), t_seq.numel(),
                                t_off.data_ptr(), t_len.data_ptr(), h0.data_ptr(), n, scoring,
                                out.data_ptr(), cells.data_ptr() if cells is not None else 0,
                                stream.cuda_stream)
        self._check(s, "xt_extend_batch_bwa")
        return out, cells

    def extend_seeds(self, q_seq, q_off, q_len, t_seq, t_off, t_len, q_beg, t_beg, seed_len, h0,
                     scoring, stream=None):
        """Both-direction extension of seeds (xt_extend_seeds): CUDA tensors in,
        (left [n, 7], right [n, 7], left_cells [n], right_cells [n]) out."""
        import torch
        d = self._dev
        q_seq = d(q_seq, torch.uint8, "q_seq")
        t_seq = d(t_seq, torch.uint8, "t_seq")
        q_off = d(q_off, torch.int64, "q_off")
        t_off = d(t_off, torch.int64, "t_off")
        arrs32 = [d(a, torch.int32, nm) for a, nm in ((q_len, "q_len"), (t_len, "t_len"),
                                                      (q_beg, "q_beg"), (t_beg, "t_beg"),
                                                      (seed_len, "seed_len"), (h0, "h0"))]
        q_len, t_len, q_beg, t_beg, seed_len, h0 = arrs32
        n = int(q_len.numel())
        dev = q_len.device
        left = torch.empty((n, 7), dtype=torch.int32, device=dev)
        right = torch.empty((n, 7), dtype=torch.int32, device=dev)
        lc = torch.empty(n, dtype=torch.int64, device=dev)
        rc = torch.empty(n, dtype=torch.int64, device=dev)
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        V = ctypes.c_void_p
        s = load_library().xt_extend_seeds(
            V(self.handle), V(q_seq.data_ptr()), q_seq.numel(), V(q_off.data_ptr()),
            V(q_len.data_ptr()), V(t_seq.data_ptr()), t_seq.numel(), V(t_off.data_ptr()),
            V(t_len.data_ptr()), V(q_beg.data_ptr()), V(t_beg.data_ptr()),
            V(seed_len.data_ptr()), V(h0.data_ptr()), n, ctypes.byref(_scoring(scoring)),
            V(left.data_ptr()), V(right.data_ptr()), V(lc.data_ptr()), V(rc.data_ptr()),
            V(stream.cuda_stream))
        self._check(s, "xt_extend_seeds")
        return left, right, lc, rc

    def extend_host(self, q_seq, q_off, q_len, t_seq, t_off, t_len, h0, scoring, out=None,
                    cells=None, stream=None):
        """Host (numpy, ideally pinned) buffers in and out; returns after completion."""
        import numpy as np
        import torch
        arrs = [np.ascontiguousarray(a, dt) for a, dt in
                ((q_seq, np.uint8), (q_off, np.int64), (q_len, np.int32), (t_seq, np.uint8),
                 (t_off, np.int64), (t_len, np.int32), (h0, np.int32))]
        q_seq, q_off, q_len, t_seq, t_off, t_len, h0 = arrs
        n = int(q_len.size)
        if out is None:
            out = np.empty((n, 7), np.int32)
        if cells is None:
            cells = np.empty(n, np.int64)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        p = lambda a: a.ctypes.data  # noqa: E731
        s = _call("xt_extend_batch_host", self.handle, p(q_seq), q_seq.size, p(q_off), p(q_len),
                  p(t_seq), t_seq.size, p(t_off), p(t_len), p(h0), n, _scoring(scoring), p(out),
                  p(cells), stream.cuda_stream)
        self._check(s, "xt_extend_batch_host")
        return out, cells


class Server:
    """The serving loop (xt_serve_*) on numpy host arrays.

    submit() queues one request and returns its ticket; the arrays passed
    (and the result arrays it allocates) are kept alive here until wait()
    releases the ticket.  wait() returns (out [n, 7] int32, cells [n] int64,
    times dict) or raises XtError with the request's status."""

    def __init__(self, device: int = 0, slots: int = 0, max_batch_pairs: int = 0,
                 max_batch_bytes: int = 0, max_queued_bytes: int = 0, mem_budget_bytes: int = 0,
                 gather_threads: int = 0, tuning_path: str | None = None,
                 alphabet: int = XT_ALPHABET_CODES):
        cfg = xt_serve_config(slots, max_batch_pairs, max_batch_bytes, max_queued_bytes,
                              mem_budget_bytes, gather_threads,
                              tuning_path.encode() if tuning_path else None, alphabet)
        self.handle = xt_serve_create(device, cfg)
        self._live = {}

    def submit(self, q_seq, q_off, q_len, t_seq, t_off, t_len, h0, scoring, want_cells=True,
               retry_busy: bool = False) -> int:
        import numpy as np
        arrs = [np.ascontiguousarray(a, dt) for a, dt in
                ((q_seq, np.uint8), (q_off, np.int64), (q_len, np.int32), (t_seq, np.uint8),
                 (t_off, np.int64), (t_len, np.int32), (h0, np.int32))]
        n = int(arrs[2].size)
        out = np.empty((n, 7), np.int32)
        cells = np.empty(n, np.int64) if want_cells else None
        p = lambda a: a.ctypes.data if a is not None and a.size else 0  # noqa: E731
        backoff = 50e-6
        while True:
            s, ticket = xt_serve_submit(self.handle, p(arrs[0]), arrs[0].size, p(arrs[1]),
                                        p(arrs[2]), p(arrs[3]), arrs[3].size, p(arrs[4]),
                                        p(arrs[5]), p(arrs[6]), n, scoring, p(out), p(cells))
            if s == XT_EBUSY and retry_busy:
                # the queue drains as batches form; sleeping leaves the host
                # cores to the server's gather threads
                time.sleep(backoff)
                backoff = min(2 * backoff, 2e-3)
                continue
            if s != XT_OK:
                raise XtError(s, "xt_serve_submit")
            self._live[ticket] = (arrs, out, cells)
            return ticket

    def poll(self, ticket: int) -> bool:
        s, done = xt_serve_poll(self.handle, ticket)
        if s != XT_OK:
            raise XtError(s, "xt_serve_poll")
        return done

    def wait(self, ticket: int, timeout_s: float | None = None):
        us = -1 if timeout_s is None else int(timeout_s * 1e6)
        s, t = xt_serve_wait(self.handle, ticket, us)
        if s == XT_ETIMEOUT:
            raise XtError(s, "xt_serve_wait")
        _, out, cells = self._live.pop(ticket, (None, None, None))
        if s != XT_OK:
            raise XtError(s, "xt_serve_wait")
        times = {f: getattr(t, f) for f, _ in xt_serve_times._fields_}
        return out, cells, times

    def pause(self, paused: bool = True):
        s = xt_serve_pause(self.handle, paused)
        if s != XT_OK:
            raise XtError(s, "xt_serve_pause")

    def stats(self) -> dict:
        st = xt_serve_get_stats(self.handle)
        return {f: getattr(st, f) for f, _ in xt_serve_stats._fields_}

    def close(self):
        if self.handle:
            xt_serve_destroy(self.handle)
            self.handle = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
