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

Parity status: every output field (score, qle, tle, gscore, gtle, max_off,
status) and the useful-cell count are pinned by ``tests/test_oracle_pins.py``
(hand-worked tables, closed forms, independent path enumeration, invariants).
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
