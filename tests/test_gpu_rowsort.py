"""The per-row ordering step (tcrnet_sort_rows) against numpy's sort, row by row,
for rows in every class of the sort (one lane, warp registers, shared memory,
chunk sorts with pairwise merges above 16,384 values) and for values that
repeat, as the l_max = 2 candidate rows do. Bar: bit-exact."""

from __future__ import annotations

import numpy as np
import pytest
import torch

import paper_2112_06613_b300 as tn

pytestmark = pytest.mark.gpu

LENGTHS = [0, 1, 2, 7, 8, 9, 31, 32, 33, 63, 64, 65, 128, 129, 255, 256, 257, 511, 512, 513,
           1000, 4095, 4096, 4097, 16383, 16384, 16385, 30000, 65537, 140000]


def _rows(kind, rng):
    rows = []
    for L in LENGTHS:
        if kind == "distinct":
            v = rng.choice(10_000_000, size=L, replace=False).astype(np.int32)
        elif kind == "repeats":  # few distinct values: long runs of equal ones
            v = rng.integers(0, 50, size=L).astype(np.int32)
        elif kind == "pairs":  # every value twice, shuffled (repeats straddle the merge runs)
            v = np.repeat(rng.choice(10_000_000, size=(L + 1) // 2, replace=False), 2)[:L].astype(np.int32)
            rng.shuffle(v)
        elif kind == "equal":
            v = np.full(L, 7, np.int32)
        elif kind == "descending":
            v = np.sort(rng.choice(10_000_000, size=L, replace=False).astype(np.int32))[::-1].copy()
        else:
            raise ValueError(kind)
        rows.append(v)
    return rows


@pytest.mark.parametrize("kind", ["distinct", "repeats", "pairs", "equal", "descending"])
def test_sort_rows_every_class(kind):
    rng = np.random.default_rng(hash(kind) % 2**32)
    rows = _rows(kind, rng)
    rng.shuffle(rows)  # classes interleaved
    off = np.zeros(len(rows) + 1, np.int64)
    off[1:] = np.cumsum([len(r) for r in rows])
    flat = np.concatenate(rows).astype(np.int32)
    d_off = torch.from_numpy(off).cuda()
    d_cols = torch.from_numpy(flat).cuda()
    tn.tcrnet_sort_rows(d_off, d_cols)
    got = d_cols.cpu().numpy()
    for i, r in enumerate(rows):
        assert np.array_equal(got[off[i]:off[i + 1]], np.sort(r)), (kind, len(r))


def test_sort_rows_rejects_bad_offsets():
    d_cols = torch.zeros(10, dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):
        tn.tcrnet_sort_rows(torch.tensor([0, 5, 3, 10], dtype=torch.int64, device="cuda"), d_cols)
    with pytest.raises(ValueError):
        tn.tcrnet_sort_rows(torch.tensor([0, 5, 11], dtype=torch.int64, device="cuda"), d_cols)
    with pytest.raises(TypeError):
        tn.tcrnet_sort_rows(torch.tensor([0, 10], dtype=torch.int32, device="cuda"), d_cols)
