"""Seeded synthetic seed-extension workloads (input generation only).

Stands in for the paper's BWA-MEM seeds on GRCh38 with MiSeq 250 bp and
PacBio ~2 kbp reads (Sec. V-D) and for its wgsim-like equal-length reads
(Sec. V-B), which are not available here.  Shapes follow the five workload
presets below; the C generator (csrc/xt_synth.c) draws every base from a
counter-based SplitMix64 keyed by (seed, pair index), so results are the same
on every host and for every split of the batch.

This module holds none of the extension arithmetic.  It is shared by the
tests, the bench and the oracle runs as a source of inputs.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
from dataclasses import dataclass, field, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "xt_synth.c")
_LIB = None


class _Cfg(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("len_kind", ctypes.c_int32),
                ("qlen_fixed", ctypes.c_int32), ("n_mix", ctypes.c_int32),
                ("mix_len", ctypes.c_int32 * 4), ("mix_frac", ctypes.c_double * 4),
                ("len_lo", ctypes.c_double), ("len_hi", ctypes.c_double),
                ("ln_median", ctypes.c_double), ("ln_sigma", ctypes.c_double),
                ("tlen_extra", ctypes.c_int32), ("p_n", ctypes.c_double),
                ("p_sub", ctypes.c_double), ("p_ins", ctypes.c_double), ("p_del", ctypes.c_double),
                ("indel_max", ctypes.c_int32), ("long_threshold", ctypes.c_int32),
                ("long_p_sub", ctypes.c_double), ("long_p_ins", ctypes.c_double),
                ("long_p_del", ctypes.c_double), ("p_unrelated", ctypes.c_double),
                ("h0_lo", ctypes.c_int32), ("h0_hi", ctypes.c_int32)]


@dataclass(frozen=True)
class ScoringParams:
    """Scoring of a workload (same field meaning as the C ABI's xt_scoring)."""
    match: int = 1
    mismatch: int = -4
    gap_open: int = 6
    gap_extend: int = 1
    w: int = 100
    zdrop: int = 100
    n_score: int = -1

    def as_tuple(self):
        return (self.match, self.mismatch, self.gap_open, self.gap_extend, self.w, self.zdrop,
                self.n_score)


@dataclass(frozen=True)
class BwaScoringParams:
    """Scoring of the BWA-MEM-compatible extension (same field meaning as the
    C ABI's xt_bwa_scoring)."""
    match: int = 1
    mismatch: int = -4
    n_score: int = -1
    o_del: int = 6
    e_del: int = 1
    o_ins: int = 6
    e_ins: int = 1
    w: int = 100
    zdrop: int = 100
    end_bonus: int = 5

    def as_tuple(self):
        return (self.match, self.mismatch, self.n_score, self.o_del, self.e_del, self.o_ins,
                self.e_ins, self.w, self.zdrop, self.end_bonus)

    @staticmethod
    def from_scoring(sc: "ScoringParams", end_bonus: int = 5) -> "BwaScoringParams":
        """The same penalties for insertions and deletions as a default scoring."""
        return BwaScoringParams(sc.match, sc.mismatch, sc.n_score, sc.gap_open, sc.gap_extend,
                                sc.gap_open, sc.gap_extend, sc.w, sc.zdrop, end_bonus)


@dataclass(frozen=True)
class Workload:
    name: str
    n_pairs: int
    seed: int
    len_kind: int                      # 0 fixed, 1 uniform over read-length mix, 2 log-uniform, 3 lognormal
    qlen_fixed: int = 0
    mix: tuple = ()                    # ((read_len, fraction), ...)
    len_lo: float = 0.0
    len_hi: float = 0.0
    ln_median: float = 0.0
    ln_sigma: float = 0.0
    tlen_extra: int = 200
    p_n: float = 0.001
    p_sub: float = 0.01
    p_ins: float = 0.0005
    p_del: float = 0.0005
    indel_max: int = 3
    long_threshold: int = 0
    long_p_sub: float = 0.0
    long_p_ins: float = 0.0
    long_p_del: float = 0.0
    p_unrelated: float = 0.0
    h0_lo: int = 19
    h0_hi: int = 60
    scoring: ScoringParams = field(default_factory=ScoringParams)

    def _c(self) -> _Cfg:
        c = _Cfg()
        c.seed = self.seed
        c.len_kind = self.len_kind
        c.qlen_fixed = self.qlen_fixed
        c.n_mix = len(self.mix)
        for k, (rl, fr) in enumerate(self.mix):
            c.mix_len[k] = rl
            c.mix_frac[k] = fr
        c.len_lo, c.len_hi = self.len_lo, self.len_hi
        c.ln_median, c.ln_sigma = self.ln_median, self.ln_sigma
        c.tlen_extra = self.tlen_extra
        c.p_n, c.p_sub, c.p_ins, c.p_del = self.p_n, self.p_sub, self.p_ins, self.p_del
        c.indel_max = self.indel_max
        c.long_threshold = self.long_threshold
        c.long_p_sub, c.long_p_ins, c.long_p_del = self.long_p_sub, self.long_p_ins, self.long_p_del
        c.p_unrelated = self.p_unrelated
        c.h0_lo, c.h0_hi = self.h0_lo, self.h0_hi
        return c


_C4_ERR = 0.08 / 3.0

WORKLOADS = {
    # 1,000 pairs: 100 bp queries, 116 bp targets, 2% substitutions, 0.2% indels of 1-3 bp.
    "c1_tiny": Workload("c1_tiny", 1000, 1, 0, qlen_fixed=100, tlen_extra=16, p_sub=0.02,
                        p_ins=0.001, p_del=0.001, h0_lo=19, h0_hi=40),
    # 1M pairs: extension length uniform [1,150] (remainder of a 150 bp read past a seed),
    # target = query + 2w; 1% substitutions, 0.1% indels, 5% unrelated pairs.
    "c2_short": Workload("c2_short", 1_000_000, 2, 1, mix=((150, 1.0),), p_unrelated=0.05),
    # 4M pairs: read lengths 100/150/250 at 40/40/20%, extension length uniform [1, read length].
    "c3_mixed": Workload("c3_mixed", 4_000_000, 3, 1, mix=((100, 0.4), (150, 0.4), (250, 0.2)),
                         p_unrelated=0.05),
    # 250k pairs: query length log-uniform [1000, 10000], 8% errors (sub:ins:del = 1:1:1),
    # target = query + 2w with w = 500, zdrop = 400.
    "c4_long": Workload("c4_long", 250_000, 4, 2, len_lo=1000.0, len_hi=10000.0, tlen_extra=1000,
                        p_sub=_C4_ERR, p_ins=_C4_ERR, p_del=_C4_ERR,
                        scoring=ScoringParams(w=500, zdrop=400)),
    # served stream: lognormal length (median 120, sigma 1.0) clipped to [1, 2000];
    # c3's mutation mix up to 300 bp, c4's above.
    "c5_stream": Workload("c5_stream", 10_000_000, 5, 3, len_lo=1.0, len_hi=2000.0, ln_median=120.0,
                          ln_sigma=1.0, long_threshold=300, long_p_sub=_C4_ERR,
                          long_p_ins=_C4_ERR, long_p_del=_C4_ERR, p_unrelated=0.05),
}


# Equal-length reads of the paper's kernel comparison (Sec. V-B): 5,000 pairs per
# call at each length L in 64..4096 from a wgsim-like simulator.  Here: target =
# a reference window of L bases, query = a copy with 2% substitutions (base
# errors) and 0.1% indels, both L long; the whole table is the band (w = L) and
# z-drop is off, so every pair extends over all L x L cells.
X2_LENGTHS = (64, 128, 256, 512, 1024, 2048, 4096)


def x2_workload(L: int, n_pairs: int = 5000) -> Workload:
    return Workload(f"x2_{L}", n_pairs, 100 + L.bit_length(), 0, qlen_fixed=L, tlen_extra=0,
                    p_sub=0.02, p_ins=0.0005, p_del=0.0005, h0_lo=20, h0_hi=40,
                    scoring=ScoringParams(w=L, zdrop=0))


def lib_path() -> str:
    return os.path.join(_HERE, "_build", f"libxt_synth.{platform.machine()}.so")


def build(force: bool = False) -> str:
    out = lib_path()
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(out), exist_ok=True)
        tmp = out + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", _SRC, "-lm",
                        "-o", tmp], check=True)
        os.replace(tmp, out)
    return out


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.xs_shapes.restype = None
        lib.xs_shapes.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_uint64, ctypes.c_int64, P, P, P]
        lib.xs_fill.restype = None
        lib.xs_fill.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_uint64, ctypes.c_int64, P, P, P, P,
                                ctypes.c_int]
        lib.xs_shapes_at.restype = None
        lib.xs_shapes_at.argtypes = [ctypes.POINTER(_Cfg), P, ctypes.c_int64, P, P, P]
        lib.xs_fill_at.restype = None
        lib.xs_fill_at.argtypes = [ctypes.POINTER(_Cfg), P, ctypes.c_int64, P, P, P, P,
                                   ctypes.c_int]
        _LIB = lib
    return _LIB


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Batch:
    """Pairs laid out as the C ABI takes them: concatenated uint8 base codes
    (0..3 = A,C,G,T, 4 = N) with int64 offsets and int32 lengths, and int32 h0."""
    q_seq: np.ndarray
    q_off: np.ndarray
    q_len: np.ndarray
    t_seq: np.ndarray
    t_off: np.ndarray
    t_len: np.ndarray
    h0: np.ndarray

    @property
    def n(self) -> int:
        return int(self.q_len.size)

    def take(self, idx) -> "Batch":
        """Sub-batch of the given pair indices, repacked contiguously."""
        idx = np.asarray(idx, np.int64)
        ql, tl = self.q_len[idx], self.t_len[idx]
        qo = np.zeros(idx.size, np.int64)
        to = np.zeros(idx.size, np.int64)
        if idx.size > 1:
            qo[1:] = np.cumsum(ql[:-1], dtype=np.int64)
            to[1:] = np.cumsum(tl[:-1], dtype=np.int64)
        qs = np.empty(int(ql.sum()), np.uint8)
        ts = np.empty(int(tl.sum()), np.uint8)
        for k, i in enumerate(idx):
            qs[qo[k]:qo[k] + ql[k]] = self.q_seq[self.q_off[i]:self.q_off[i] + ql[k]]
            ts[to[k]:to[k] + tl[k]] = self.t_seq[self.t_off[i]:self.t_off[i] + tl[k]]
        return Batch(qs, qo, ql.copy(), ts, to, tl.copy(), self.h0[idx].copy())

    def nbytes(self) -> int:
        return sum(int(a.nbytes) for a in (self.q_seq, self.q_off, self.q_len, self.t_seq,
                                           self.t_off, self.t_len, self.h0))


def generate(wl: Workload, n: int | None = None, first: int = 0,
             nthreads: int | None = None) -> Batch:
    """Pairs [first, first+n) of workload wl (n defaults to wl.n_pairs)."""
    n = wl.n_pairs if n is None else int(n)
    cfg = wl._c()
    lib = _lib()
    q_len = np.empty(n, np.int32)
    t_len = np.empty(n, np.int32)
    h0 = np.empty(n, np.int32)
    lib.xs_shapes(ctypes.byref(cfg), first, n, _p(q_len), _p(t_len), _p(h0))
    q_off = np.zeros(n, np.int64)
    t_off = np.zeros(n, np.int64)
    if n > 1:
        np.cumsum(q_len[:-1], dtype=np.int64, out=q_off[1:])
        np.cumsum(t_len[:-1], dtype=np.int64, out=t_off[1:])
    q_seq = np.empty(int(q_len.sum(dtype=np.int64)), np.uint8)
    t_seq = np.empty(int(t_len.sum(dtype=np.int64)), np.uint8)
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    lib.xs_fill(ctypes.byref(cfg), first, n, _p(q_off), _p(t_off), _p(q_seq), _p(t_seq),
                int(nthreads))
    return Batch(q_seq, q_off, q_len, t_seq, t_off, t_len, h0)


def shapes(wl: Workload, n: int | None = None, first: int = 0):
    """(q_len, t_len, h0) of pairs [first, first+n) without their sequences."""
    n = wl.n_pairs if n is None else int(n)
    cfg = wl._c()
    q_len = np.empty(n, np.int32)
    t_len = np.empty(n, np.int32)
    h0 = np.empty(n, np.int32)
    _lib().xs_shapes(ctypes.byref(cfg), first, n, _p(q_len), _p(t_len), _p(h0))
    return q_len, t_len, h0


def generate_at(wl: Workload, idx, nthreads: int | None = None) -> Batch:
    """The pairs of workload wl with the given stream indices, in that order
    (pair k is the same pair generate() gives at position k)."""
    idx = np.ascontiguousarray(idx, np.int64)
    n = int(idx.size)
    cfg = wl._c()
    lib = _lib()
    q_len = np.empty(n, np.int32)
    t_len = np.empty(n, np.int32)
    h0 = np.empty(n, np.int32)
    lib.xs_shapes_at(ctypes.byref(cfg), _p(idx), n, _p(q_len), _p(t_len), _p(h0))
    q_off = np.zeros(n, np.int64)
    t_off = np.zeros(n, np.int64)
    if n > 1:
        np.cumsum(q_len[:-1], dtype=np.int64, out=q_off[1:])
        np.cumsum(t_len[:-1], dtype=np.int64, out=t_off[1:])
    q_seq = np.empty(int(q_len.sum(dtype=np.int64)), np.uint8)
    t_seq = np.empty(int(t_len.sum(dtype=np.int64)), np.uint8)
    lib.xs_fill_at(ctypes.byref(cfg), _p(idx), n, _p(q_off), _p(t_off), _p(q_seq), _p(t_seq),
                   int(nthreads or os.cpu_count() or 1))
    return Batch(q_seq, q_off, q_len, t_seq, t_off, t_len, h0)


def with_n(wl: Workload, n: int) -> Workload:
    return replace(wl, n_pairs=int(n))


@dataclass
class RequestStream:
    """A served stream cut from one Batch: request r holds the consecutive
    pairs [start[r], start[r] + size[r]) and arrives at arrival_s[r] seconds
    after the stream starts.  q_rel/t_rel are the pairs' offsets relative to
    the first base of their own request, so a request's arrays are views."""
    batch: Batch
    start: np.ndarray
    size: np.ndarray
    arrival_s: np.ndarray
    q_rel: np.ndarray
    t_rel: np.ndarray

    def request(self, r: int):
        """(q_seq, q_off, q_len, t_seq, t_off, t_len, h0) of request r, as views."""
        b = self.batch
        a, n = int(self.start[r]), int(self.size[r])
        if n == 0:
            e8, e64, e32 = np.empty(0, np.uint8), np.empty(0, np.int64), np.empty(0, np.int32)
            return e8, e64, e32, e8, e64, e32, e32
        qa, ta = int(b.q_off[a]), int(b.t_off[a])
        qe = int(b.q_off[a + n - 1]) + int(b.q_len[a + n - 1])
        te = int(b.t_off[a + n - 1]) + int(b.t_len[a + n - 1])
        s = slice(a, a + n)
        return (b.q_seq[qa:qe], self.q_rel[s], b.q_len[s], b.t_seq[ta:te], self.t_rel[s],
                b.t_len[s], b.h0[s])


def request_stream(b: Batch, rate_pairs_per_s: float, max_request: int = 4096,
                   seed: int = 5, sizes=None) -> RequestStream:
    """Cut b into requests of U[1, max_request] pairs (or the given sizes,
    which must sum to b.n) with Poisson arrivals at an offered load of
    rate_pairs_per_s (exponential gaps between requests, mean request size /
    rate)."""
    rng = np.random.default_rng(seed)
    if sizes is None:
        sizes = []
        left = b.n
        while left > 0:
            k = int(min(left, rng.integers(1, max_request + 1)))
            sizes.append(k)
            left -= k
    size = np.asarray(sizes, np.int64)
    if int(size.sum()) != b.n or np.any(size < 0):
        raise ValueError("request sizes must be >= 0 and sum to the batch's pairs")
    start = np.zeros(size.size, np.int64)
    if size.size > 1:
        np.cumsum(size[:-1], out=start[1:])
    mean_gap = (max_request + 1) / 2.0 / float(rate_pairs_per_s)
    arrival = np.cumsum(rng.exponential(mean_gap, size.size))
    nz = size > 0
    q_rel = b.q_off - np.repeat(b.q_off[start[nz]], size[nz])
    t_rel = b.t_off - np.repeat(b.t_off[start[nz]], size[nz])
    return RequestStream(b, start, size, arrival, q_rel, t_rel)
