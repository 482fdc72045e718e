"""The pins catch plausible mistakes: each mutated copy of the oracle source
(compiled on the CPU into a temporary library) must fail at least one pin."""

from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
from synthgen import ALPHABET, from_strings, generate_config1

from test_oracle_pins import (
    _edit_graph,
    all_strings,
    lev_recursive,
    lists_of,
    read_adjacency_golden,
    read_lev_pairs,
)

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

# (name, original text, mutated text)
MUTATIONS = [
    ("indicator-inverted", "(a[i - 1] != b[j - 1]) ? 1 : 0", "(a[i - 1] != b[j - 1]) ? 0 : 1"),
    ("insertion-cost-2", "cur[j - 1] + 1,", "cur[j - 1] + 2,"),
    ("deletion-term-dropped", "prev[j] + 1,          /* deletion", "1 << 20,          /* deletion"),
    ("base-row-zero", "prev[j] = (int)j;", "prev[j] = 0;"),
    ("base-col-off-by-one", "cur[0] = (int)i;", "cur[0] = (int)i - 1;"),
    ("b-index-reversed", "a[i - 1] != b[j - 1]", "a[i - 1] != b[lb - j]"),
    ("strict-threshold", "if (d <= max_dist)", "if (d < max_dist)"),
    ("self-loops", "if (j == self) continue;", ""),
    ("skip-last-column", "for (int64_t j = 0; j < n; ++j) {", "for (int64_t j = 0; j + 1 < n; ++j) {"),
]


def _pins_pass(lib) -> bool:
    try:
        for a in all_strings("AC", 4):
            for b in all_strings("AC", 4):
                if oracle.lev(a, b, lib=lib) != lev_recursive(a, b):
                    return False
        for a, b, d, _ in read_lev_pairs():
            if oracle.lev(a, b, lib=lib) != d:
                return False
        mat, _, strings = read_adjacency_golden()
        rep = from_strings(strings)
        off, cols, _ = oracle.network(rep.chars, rep.offsets, max_dist=1, lib=lib)
        got = np.zeros((5, 5), dtype=int)
        for i in range(5):
            got[i, cols[off[i]:off[i + 1]]] = 1
        if not (got == mat).all():
            return False
        strs = generate_config1(400, seed=9).strings() + ["CAAAF", "CAAF", "AAB", "AB"]
        rep = from_strings(strs)
        off, cols, _ = oracle.network(rep.chars, rep.offsets, max_dist=1, lib=lib)
        if lists_of(off, cols) != _edit_graph(strs, ALPHABET):
            return False
    except Exception:
        return False
    return True


def test_unmutated_source_passes(oracle_lib):
    assert _pins_pass(oracle_lib)


@pytest.mark.parametrize("name,orig,mut", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, name, orig, mut):
    text = open(SRC).read()
    assert orig in text, f"mutation anchor for {name} not found"
    src = tmp_path / f"oracle_{name}.c"
    src.write_text(text.replace(orig, mut, 1))
    lib_path = oracle.build(force=True, src=str(src), out=str(tmp_path / f"lib_{name}.so"))
    lib = oracle.load(lib_path)
    assert not _pins_pass(lib), f"planted mistake {name} was not caught by any pin"


# Planted mistakes in the CPU baseline (the paper's early-abort test): each must
# fail the baseline's pin against the recurrence.
BASELINE_MUTATIONS = [
    ("abort-at-bound", "if (row_min > max_dist) {", "if (row_min >= max_dist) {"),
    ("length-skip-off-by-one", "if (dl > max_dist) return 0;", "if (dl >= max_dist) return 0;"),
    ("no-final-check", "if (within) within = row[lb] <= max_dist;", ""),
    ("row-min-is-last-entry", "if (v < row_min) row_min = v;", "row_min = v;"),
]


def _baseline_pins_pass(lib) -> bool:
    try:
        strs = all_strings("AC", 5)
        for a in strs:
            for b in strs:
                d = lev_recursive(a, b)
                for t in range(3):
                    if oracle.baseline_within(a, b, t, lib=lib) != (d <= t):
                        return False
    except Exception:
        return False
    return True


def test_unmutated_baseline_passes(oracle_lib):
    assert _baseline_pins_pass(oracle_lib)


@pytest.mark.parametrize("name,orig,mut", BASELINE_MUTATIONS, ids=[m[0] for m in BASELINE_MUTATIONS])
def test_planted_baseline_mistake_is_caught(tmp_path, name, orig, mut):
    text = open(SRC).read()
    assert orig in text, f"mutation anchor for {name} not found"
    src = tmp_path / f"baseline_{name}.c"
    src.write_text(text.replace(orig, mut, 1))
    lib_path = oracle.build(force=True, src=str(src), out=str(tmp_path / f"libb_{name}.so"))
    lib = oracle.load(lib_path)
    assert not _baseline_pins_pass(lib), f"planted baseline mistake {name} was not caught"
