"""CPU oracle for the TCR network — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg import this package. The library under test never imports it and never
falls back to it; the two share no code.

It wraps ``oracle.c`` (plain Wagner-Fischer, Methods "Levenshtein distance",
Eq. levenshtein; network rule of Methods "TCR network"; row serialisation of
Methods "Adjacency matrix") through ctypes. Every function here is pinned by
``tests/test_oracle_pins.py`` against things other than itself: a memoised
transcription of the recurrence, hand-worked pairs (the paper's ACCA/ACGG
example), the paper's 5-node adjacency example, metric invariants, the
Hamming special case and the exact lev <= 1 edit-neighbourhood.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False, src: str = _SRC, out: str = _LIB_PATH, extra=()) -> str:
    """Compile oracle.c with gcc (OpenMP) into a shared library."""
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", *extra, "-o", out, src]
        subprocess.run(cmd, check=True)
    return out


class _Lists(ctypes.Structure):
    pass


def _bind(path: str):
    lib = ctypes.CDLL(path)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    i64p = ctypes.POINTER(ctypes.c_int64)
    i32p = ctypes.POINTER(ctypes.c_int32)
    lp = ctypes.POINTER(_Lists)
    lib.oracle_lev.argtypes = [u8p, ctypes.c_int64, u8p, ctypes.c_int64]
    lib.oracle_lev.restype = ctypes.c_int
    lib.oracle_neighbors.argtypes = [u8p, i64p, ctypes.c_int64, u8p, i64p, ctypes.c_int64,
                                     i64p, ctypes.c_int32, ctypes.c_int32]
    lib.oracle_neighbors.restype = lp
    lib.oracle_lists_rows.argtypes = [lp]
    lib.oracle_lists_rows.restype = ctypes.c_int64
    lib.oracle_lists_nnz.argtypes = [lp]
    lib.oracle_lists_nnz.restype = ctypes.c_int64
    lib.oracle_lists_copy.argtypes = [lp, i64p, i32p]
    lib.oracle_lists_copy.restype = None
    lib.oracle_lists_free.argtypes = [lp]
    lib.oracle_lists_free.restype = None
    lib.oracle_max_threads.argtypes = []
    lib.oracle_max_threads.restype = ctypes.c_int
    lib.baseline_within.argtypes = [u8p, ctypes.c_int64, u8p, ctypes.c_int64, ctypes.c_int32]
    lib.baseline_within.restype = ctypes.c_int
    lib.baseline_neighbors.argtypes = lib.oracle_neighbors.argtypes
    lib.baseline_neighbors.restype = lp
    return lib


def load(path: str | None = None):
    """Load (building first if needed) the oracle library. A custom `path`
    loads a separately compiled variant (used by the planted-mistake tests)."""
    global _lib
    if path is not None:
        return _bind(path)
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(_LIB_PATH)
    return _lib


def _u8(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _i64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _i32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _bytes(s) -> np.ndarray:
    if isinstance(s, str):
        s = s.encode("ascii")
    return np.frombuffer(bytes(s) + b"\0", dtype=np.uint8)


def lev(a, b, lib=None) -> int:
    """Levenshtein distance of two strings (Eq. levenshtein, Wagner-Fischer)."""
    lib = lib or load()
    x = _bytes(a)
    y = _bytes(b)
    return int(lib.oracle_lev(_u8(x), len(x) - 1, _u8(y), len(y) - 1))


def neighbors(chars, offsets, qchars=None, qoffsets=None, self_index=None,
              max_dist: int = 1, nthreads: int = 0, lib=None, _fn="oracle_neighbors"):
    """For each query, all repertoire indices within edit distance `max_dist`.

    Without queries, the queries are the repertoire itself with self-exclusion
    (the full network's rows). Returns (offsets int64 [m+1], cols int32 [nnz]).
    """
    lib = lib or load()
    chars = np.ascontiguousarray(chars, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    n = offsets.shape[0] - 1
    if qchars is None:
        qchars, qoffsets = chars, offsets
        if self_index is None:
            self_index = np.arange(n, dtype=np.int64)
    qchars = np.ascontiguousarray(qchars, dtype=np.uint8)
    qoffsets = np.ascontiguousarray(qoffsets, dtype=np.int64)
    m = qoffsets.shape[0] - 1
    if chars.size == 0:
        chars = np.zeros(1, dtype=np.uint8)
    if qchars.size == 0:
        qchars = np.zeros(1, dtype=np.uint8)
    si = None
    if self_index is not None:
        self_index = np.ascontiguousarray(self_index, dtype=np.int64)
        si = _i64(self_index)
    res = getattr(lib, _fn)(_u8(chars), _i64(offsets), n, _u8(qchars), _i64(qoffsets), m,
                            si, int(max_dist), int(nthreads))
    if not res:
        raise MemoryError("oracle_neighbors failed")
    try:
        rows = lib.oracle_lists_rows(res)
        nnz = lib.oracle_lists_nnz(res)
        off = np.zeros(rows + 1, dtype=np.int64)
        cols = np.zeros(max(nnz, 1), dtype=np.int32)
        lib.oracle_lists_copy(res, _i64(off), _i32(cols))
    finally:
        lib.oracle_lists_free(res)
    return off, cols[:nnz]


def network(chars, offsets, max_dist: int = 1, nthreads: int = 0, lib=None):
    """Full network CSR (offsets int64 [n+1], cols int32, degree int32 [n])."""
    off, cols = neighbors(chars, offsets, max_dist=max_dist, nthreads=nthreads, lib=lib)
    return off, cols, np.diff(off).astype(np.int32)


def rows(chars, offsets, row_ids, max_dist: int = 1, nthreads: int = 0, lib=None, _fn="oracle_neighbors"):
    """Complete neighbour lists of selected rows of the network."""
    chars = np.ascontiguousarray(chars, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    row_ids = np.ascontiguousarray(row_ids, dtype=np.int64)
    lens = offsets[row_ids + 1] - offsets[row_ids]
    qoff = np.zeros(row_ids.shape[0] + 1, dtype=np.int64)
    np.cumsum(lens, out=qoff[1:])
    qchars = np.concatenate([chars[offsets[i]:offsets[i + 1]] for i in row_ids]) if row_ids.size \
        else np.zeros(0, dtype=np.uint8)
    return neighbors(chars, offsets, qchars, qoff, self_index=row_ids, max_dist=max_dist,
                     nthreads=nthreads, lib=lib, _fn=_fn)


def max_threads(lib=None) -> int:
    lib = lib or load()
    return int(lib.oracle_max_threads())


# ---------------------------------------------------------------------------
# CPU baseline (not the oracle): the paper's early-abort per-pair test
# (Methods "GPU-based network generation", Listing 1, restated correctly: the
# row-minimum abort plus the length-difference skip). Used only to time the
# paper's own algorithm on the host; pinned to the oracle by the test suite.

def baseline_within(a, b, max_dist: int = 1, lib=None) -> bool:
    """lev(a, b) <= max_dist by the early-abort table."""
    lib = lib or load()
    x = _bytes(a)
    y = _bytes(b)
    r = int(lib.baseline_within(_u8(x), len(x) - 1, _u8(y), len(y) - 1, int(max_dist)))
    if r < 0:
        raise MemoryError("baseline_within failed")
    return bool(r)


def baseline_network(chars, offsets, max_dist: int = 1, nthreads: int = 0, lib=None):
    """Full network by the baseline test (offsets int64, cols int32, degree int32)."""
    off, cols = neighbors(chars, offsets, max_dist=max_dist, nthreads=nthreads, lib=lib,
                          _fn="baseline_neighbors")
    return off, cols, np.diff(off).astype(np.int32)


def baseline_rows(chars, offsets, row_ids, max_dist: int = 1, nthreads: int = 0, lib=None):
    """Neighbour lists of selected rows by the baseline test."""
    return rows(chars, offsets, row_ids, max_dist=max_dist, nthreads=nthreads, lib=lib,
                _fn="baseline_neighbors")
