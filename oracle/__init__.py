"""Scalar CPU oracle for banded affine-gap seed extension.

TEST INFRASTRUCTURE ONLY.  This package is the correctness oracle that the CUDA
path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it; the
library (``paper_2301_09310_gb300``) never does, and the two share no code.

The arithmetic lives in ``xt_oracle.c`` (plain C, int64, row by row), which
follows arXiv 2301.09310 Sec. II-A, Eq. 1, read as one-directional seed
extension from a seed score h0 with a static band and a z-drop cutoff.  The
file header of ``xt_oracle.c`` states the full definition.  This module only
compiles it with gcc and marshals numpy arrays.

``extend_one_bwa`` / ``extend_batch_bwa`` run the opt-in BWA-MEM-compatible
variant (gaps opened from the match value, separate insertion and deletion
penalties, band narrowing from the end bonus, row trimming, latest-row gscore
ties, direction-dependent z-drop), stated in full in ``xt_oracle.c``.

Parity status: every output field (score, qle, tle, gscore, gtle, max_off,
status) and the useful-cell count are pinned by ``tests/test_oracle_pins.py``
(hand-worked tables, closed forms, independent path enumeration, invariants);
the BWA-MEM-compatible variant by ``tests/test_oracle_bwa_pins.py`` (path
enumeration with its own move rules, a hand-worked trimming table, closed
forms at the narrowing threshold and for the z-drop direction, invariants).
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xt_oracle.c")
_LIB = None


class _Scoring(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("match", "mismatch", "gap_open", "gap_extend", "w", "zdrop", "n_score")]


@dataclass(frozen=True)
class Scoring:
    """Scoring record: match > 0; mismatch, n_score <= 0 (signed scores);
    gap_open, gap_extend >= 0 (a gap of k bases costs gap_open + k*gap_extend);
    w >= 0 band half-width; zdrop <= 0 disables the z-drop cutoff."""
    match: int = 1
    mismatch: int = -4
    gap_open: int = 6
    gap_extend: int = 1
    w: int = 100
    zdrop: int = 100
    n_score: int = -1

    def _c(self) -> _Scoring:
        return _Scoring(self.match, self.mismatch, self.gap_open, self.gap_extend, self.w,
                        self.zdrop, self.n_score)


class _BwaScoring(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("match", "mismatch", "n_score", "o_del", "e_del", "o_ins", "e_ins", "w", "zdrop",
                 "end_bonus")]


@dataclass(frozen=True)
class BwaScoring:
    """Scoring of the BWA-MEM-compatible variant: match > 0; mismatch, n_score
    <= 0; a deletion (insertion) of k bases costs o_del + k*e_del (o_ins +
    k*e_ins), e_del, e_ins >= 1; w >= 0 band half-width before narrowing;
    zdrop <= 0 disables the z-drop; end_bonus >= 0 enters the band narrowing."""
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

    def _c(self) -> _BwaScoring:
        return _BwaScoring(self.match, self.mismatch, self.n_score, self.o_del, self.e_del,
                           self.o_ins, self.e_ins, self.w, self.zdrop, self.end_bonus)


BWA_NO_TRIM = 1     # test-only switches of the BWA-MEM-compatible variant
BWA_NO_NARROW = 2


def lib_path() -> str:
    return os.path.join(_HERE, "_build", f"libxt_oracle.{platform.machine()}.so")


def build(force: bool = False) -> str:
    """Compile xt_oracle.c with gcc into oracle/_build/ (per host architecture)."""
    out = lib_path()
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(out), exist_ok=True)
        tmp = out + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-pthread", _SRC,
                        "-o", tmp], check=True)
        os.replace(tmp, out)
    return out


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.xo_extend_one.restype = None
        lib.xo_extend_one.argtypes = [P, ctypes.c_int32, P, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.POINTER(_Scoring), P, P, P, P, P, P, P, P]
        lib.xo_extend_batch.restype = ctypes.c_int
        lib.xo_extend_batch.argtypes = [P, ctypes.c_int64, P, P, P, ctypes.c_int64, P, P, P,
                                        ctypes.c_int64, ctypes.POINTER(_Scoring), P, P,
                                        ctypes.c_int]
        lib.xo_check_scoring.restype = ctypes.c_int
        lib.xo_check_scoring.argtypes = [ctypes.POINTER(_Scoring)]
        B = ctypes.POINTER(_BwaScoring)
        lib.xo_extend_one_bwa.restype = None
        lib.xo_extend_one_bwa.argtypes = [P, ctypes.c_int32, P, ctypes.c_int32, ctypes.c_int32, B,
                                          ctypes.c_int] + [P] * 11
        lib.xo_extend_batch_bwa.restype = ctypes.c_int
        lib.xo_extend_batch_bwa.argtypes = [P, ctypes.c_int64, P, P, P, ctypes.c_int64, P, P, P,
                                            ctypes.c_int64, B, P, P, ctypes.c_int]
        lib.xo_check_bwa_scoring.restype = ctypes.c_int
        lib.xo_check_bwa_scoring.argtypes = [B]
        lib.xo_bwa_band.restype = ctypes.c_int64
        lib.xo_bwa_band.argtypes = [B, ctypes.c_int64, ctypes.c_int]
        _LIB = lib
    return _LIB


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


FIELDS = ("score", "qle", "tle", "gscore", "gtle", "max_off", "status")


@dataclass
class Trace:
    """Full extended matrices and row summaries of one extension."""
    result: tuple
    cells: int
    H: np.ndarray   # (tlen+1, qlen+1); [r+1, c+1] is cell (r, c)
    E: np.ndarray
    F: np.ndarray
    row_m: np.ndarray   # m_i for each evaluated row
    row_mj: np.ndarray  # mj_i for each evaluated row


def _codes(s) -> np.ndarray:
    if isinstance(s, str):
        table = {"A": 0, "C": 1, "G": 2, "T": 3, "N": 4}
        return np.array([table[ch] for ch in s.upper()], dtype=np.uint8)
    return np.ascontiguousarray(s, dtype=np.uint8)


def extend_one(q, t, h0: int, sc: Scoring, trace: bool = False):
    """Extend one pair.  q, t: code arrays (0..3 bases, >= 4 N) or ACGTN strings.

    Returns (result_tuple, cells) or a Trace when trace=True."""
    qa, ta = _codes(q), _codes(t)
    out = np.zeros(7, np.int32)
    cells = np.zeros(1, np.int64)
    lib = _lib()
    scc = sc._c()
    ql, tl = int(qa.size), int(ta.size)
    if trace:
        shape = (tl + 1, ql + 1)
        H = np.zeros(shape, np.int64); E = np.zeros(shape, np.int64); F = np.zeros(shape, np.int64)
        rm = np.zeros(max(tl, 1), np.int64); rmj = np.zeros(max(tl, 1), np.int64)
        nr = np.zeros(1, np.int32)
        lib.xo_extend_one(_ptr(qa), ql, _ptr(ta), tl, int(h0), ctypes.byref(scc), _ptr(out),
                          _ptr(cells), _ptr(rm), _ptr(rmj), _ptr(nr), _ptr(H), _ptr(E), _ptr(F))
        n = int(nr[0])
        return Trace(tuple(int(x) for x in out), int(cells[0]), H, E, F, rm[:n].copy(),
                     rmj[:n].copy())
    lib.xo_extend_one(_ptr(qa), ql, _ptr(ta), tl, int(h0), ctypes.byref(scc), _ptr(out),
                      _ptr(cells), None, None, None, None, None, None)
    return tuple(int(x) for x in out), int(cells[0])


def check_scoring(sc: Scoring) -> bool:
    return _lib().xo_check_scoring(ctypes.byref(sc._c())) == 0


def extend_batch(q_seq, q_off, q_len, t_seq, t_off, t_len, h0, sc: Scoring,
                 nthreads: int | None = None):
    """Extend a batch of pairs laid out as in the library's C ABI (concatenated
    uint8 codes, int64 offsets, int32 lengths, int32 h0).

    Returns (out int32 [n, 7], cells int64 [n]); raises ValueError when the
    scoring record is rejected."""
    q_seq = np.ascontiguousarray(q_seq, np.uint8)
    t_seq = np.ascontiguousarray(t_seq, np.uint8)
    q_off = np.ascontiguousarray(q_off, np.int64)
    t_off = np.ascontiguousarray(t_off, np.int64)
    q_len = np.ascontiguousarray(q_len, np.int32)
    t_len = np.ascontiguousarray(t_len, np.int32)
    h0 = np.ascontiguousarray(h0, np.int32)
    n = int(q_len.size)
    out = np.zeros((n, 7), np.int32)
    cells = np.zeros(n, np.int64)
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    rc = _lib().xo_extend_batch(_ptr(q_seq), int(q_seq.size), _ptr(q_off), _ptr(q_len),
                                _ptr(t_seq), int(t_seq.size), _ptr(t_off), _ptr(t_len),
                                _ptr(h0), n, ctypes.byref(sc._c()), _ptr(out), _ptr(cells),
                                int(nthreads))
    if rc != 0:
        raise ValueError("oracle rejected the scoring record")
    return out, cells


@dataclass
class BwaTrace:
    """Matrices, per-row column ranges and row summaries of one extension of
    the BWA-MEM-compatible variant (0 where a cell was not computed)."""
    result: tuple
    cells: int
    H: np.ndarray   # (tlen+1, qlen+1); [r+1, c+1] is cell (r, c)
    M: np.ndarray
    E: np.ndarray
    F: np.ndarray
    row_beg: np.ndarray  # first computed column of each evaluated row
    row_end: np.ndarray  # one past the last computed column
    row_m: np.ndarray
    row_mj: np.ndarray


def bwa_band(sc: BwaScoring, qlen: int, flags: int = 0) -> int:
    """The band half-width after narrowing for a query of length qlen."""
    return int(_lib().xo_bwa_band(ctypes.byref(sc._c()), int(qlen), int(flags)))


def check_bwa_scoring(sc: BwaScoring) -> bool:
    return _lib().xo_check_bwa_scoring(ctypes.byref(sc._c())) == 0


def extend_one_bwa(q, t, h0: int, sc: BwaScoring, flags: int = 0, trace: bool = False):
    """Extend one pair under the BWA-MEM-compatible variant.

    Returns (result_tuple, cells) or a BwaTrace when trace=True."""
    qa, ta = _codes(q), _codes(t)
    out = np.zeros(7, np.int32)
    cells = np.zeros(1, np.int64)
    lib = _lib()
    scc = sc._c()
    ql, tl = int(qa.size), int(ta.size)
    if not trace:
        lib.xo_extend_one_bwa(_ptr(qa), ql, _ptr(ta), tl, int(h0), ctypes.byref(scc), int(flags),
                              _ptr(out), _ptr(cells), *([None] * 9))
        return tuple(int(x) for x in out), int(cells[0])
    shape = (tl + 1, ql + 1)
    mats = [np.zeros(shape, np.int64) for _ in range(4)]
    rows = [np.zeros(max(tl, 1), np.int64) for _ in range(4)]
    nr = np.zeros(1, np.int32)
    lib.xo_extend_one_bwa(_ptr(qa), ql, _ptr(ta), tl, int(h0), ctypes.byref(scc), int(flags),
                          _ptr(out), _ptr(cells), *[_ptr(r) for r in rows], _ptr(nr),
                          *[_ptr(m) for m in mats])
    n = int(nr[0])
    return BwaTrace(tuple(int(x) for x in out), int(cells[0]), *mats,
                    *[r[:n].copy() for r in rows])


def extend_batch_bwa(q_seq, q_off, q_len, t_seq, t_off, t_len, h0, sc: BwaScoring,
                     nthreads: int | None = None):
    """extend_batch for the BWA-MEM-compatible variant (same layout and outputs)."""
    q_seq = np.ascontiguousarray(q_seq, np.uint8)
    t_seq = np.ascontiguousarray(t_seq, np.uint8)
    q_off = np.ascontiguousarray(q_off, np.int64)
    t_off = np.ascontiguousarray(t_off, np.int64)
    q_len = np.ascontiguousarray(q_len, np.int32)
    t_len = np.ascontiguousarray(t_len, np.int32)
    h0 = np.ascontiguousarray(h0, np.int32)
    n = int(q_len.size)
    out = np.zeros((n, 7), np.int32)
    cells = np.zeros(n, np.int64)
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    rc = _lib().xo_extend_batch_bwa(_ptr(q_seq), int(q_seq.size), _ptr(q_off), _ptr(q_len),
                                    _ptr(t_seq), int(t_seq.size), _ptr(t_off), _ptr(t_len),
                                    _ptr(h0), n, ctypes.byref(sc._c()), _ptr(out), _ptr(cells),
                                    int(nthreads))
    if rc != 0:
        raise ValueError("oracle rejected the scoring record")
    return out, cells
