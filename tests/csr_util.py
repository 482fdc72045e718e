"""Helpers shared by the GPU parity tests (comparison and invariants only)."""

from __future__ import annotations

import numpy as np


def assert_csr_equal(off_a, cols_a, off_b, cols_b, what=""):
    off_a = np.asarray(off_a, dtype=np.int64)
    off_b = np.asarray(off_b, dtype=np.int64)
    assert off_a.shape == off_b.shape, f"{what}: row count differs"
    if not np.array_equal(off_a, off_b):
        bad = np.nonzero(off_a != off_b)[0][0]
        raise AssertionError(f"{what}: offsets differ first at {bad}: {off_a[bad]} vs {off_b[bad]}")
    ca = np.asarray(cols_a, dtype=np.int32)
    cb = np.asarray(cols_b, dtype=np.int32)
    if not np.array_equal(ca, cb):
        bad = np.nonzero(ca != cb)[0][0]
        row = int(np.searchsorted(off_a, bad, side="right") - 1)
        raise AssertionError(f"{what}: cols differ first at entry {bad} (row {row})")


def assert_rows_equal(off, cols, rows, roff, rcols, what=""):
    """Rows `rows` of a full CSR equal the reference lists (roff, rcols)."""
    off = np.asarray(off, dtype=np.int64)
    for k, i in enumerate(rows):
        got = cols[off[i]:off[i + 1]]
        want = rcols[roff[k]:roff[k + 1]]
        if not np.array_equal(got, want):
            raise AssertionError(f"{what}: row {i} differs: got {len(got)} entries, want {len(want)}")


def check_invariants(off, cols, deg, n):
    """Symmetric, no self-loops, strictly ascending rows, degree = row length."""
    off = np.asarray(off, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    assert off.shape[0] == n + 1 and off[0] == 0
    lens = np.diff(off)
    assert (lens >= 0).all()
    assert np.array_equal(np.asarray(deg, dtype=np.int64), lens)
    nnz = int(off[-1])
    assert cols.shape[0] == nnz and nnz % 2 == 0
    if nnz == 0:
        return
    assert cols.min() >= 0 and cols.max() < n
    rows = np.repeat(np.arange(n, dtype=np.int64), lens)
    assert not (rows == cols).any(), "self-loop"
    # strictly ascending inside each row
    inner = np.ones(nnz, dtype=bool)
    inner[off[:-1][lens > 0]] = False
    assert (np.diff(cols)[inner[1:]] > 0).all(), "row not strictly ascending"
    # symmetry: the multiset of (i, j) equals that of (j, i)
    fwd = np.sort(rows * n + cols)
    bwd = np.sort(cols * n + rows)
    assert np.array_equal(fwd, bwd), "asymmetric"


def sample_rows(deg, count, seed=0, top=100):
    """Seeded uniform sample plus the highest-degree rows."""
    deg = np.asarray(deg)
    n = deg.shape[0]
    rng = np.random.default_rng(seed)
    pick = rng.choice(n, size=min(count, n), replace=False)
    topk = np.argsort(-deg, kind="stable")[:top]
    return np.unique(np.concatenate([pick, topk])).astype(np.int64)
