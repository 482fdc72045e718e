"""Pins for the CPU oracle: each check compares it with something other than itself.

- a memoised transcription of the Levenshtein recurrence (Methods "Levenshtein
  distance", Eq. levenshtein), exhaustively over tiny alphabets;
- hand-worked pairs, including the paper's ACCA/ACGG example (golden file);
- metric invariants and bounds of the edit distance;
- the paper's 5-node adjacency example (Methods "Adjacency matrix");
- l_max = 0 reduces to grouping identical strings (a dict group-by);
- l_max = 1 equals the explicit one-edit neighbourhood (every substitution,
  deletion and insertion of each string looked up in a dict).
"""

from __future__ import annotations

import functools
import itertools
import os
import random

import numpy as np
import pytest

import oracle
from synthgen import ALPHABET, from_strings, generate_config1

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# Independent references (test-only code, shares nothing with oracle.c)
# ---------------------------------------------------------------------------

def lev_recursive(a: str, b: str) -> int:
    """Direct transcription of the recurrence: lev(i, j) over prefix lengths,
    lev(i, 0) = i, lev(0, j) = j, else the minimum of the three moves with the
    indicator 1(a_i != b_j) on the diagonal."""

    @functools.lru_cache(maxsize=None)
    def rec(i: int, j: int) -> int:
        if i == 0 or j == 0:
            return max(i, j)
        return min(rec(i - 1, j) + 1, rec(i, j - 1) + 1,
                   rec(i - 1, j - 1) + (0 if a[i - 1] == b[j - 1] else 1))

    return rec(len(a), len(b))


def one_edit_neighbourhood(s: str, alphabet: str) -> set[str]:
    """All strings at edit distance exactly <= 1 from s (s itself included)."""
    out = {s}
    for p in range(len(s)):
        out.add(s[:p] + s[p + 1:])
        for c in alphabet:
            out.add(s[:p] + c + s[p + 1:])
    for p in range(len(s) + 1):
        for c in alphabet:
            out.add(s[:p] + c + s[p:])
    return out


def all_strings(alphabet: str, max_len: int):
    out = []
    for L in range(max_len + 1):
        out.extend("".join(t) for t in itertools.product(alphabet, repeat=L))
    return out


def lists_of(off, cols):
    return [list(cols[off[i]:off[i + 1]]) for i in range(len(off) - 1)]


# ---------------------------------------------------------------------------
# Pins on lev
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("alphabet,max_len", [("AC", 6), ("ACG", 4)])
def test_lev_matches_recurrence_bruteforce(oracle_lib, alphabet, max_len):
    strs = all_strings(alphabet, max_len)
    for a in strs:
        for b in strs:
            assert oracle.lev(a, b, lib=oracle_lib) == lev_recursive(a, b), (a, b)


def read_lev_pairs():
    rows = []
    with open(os.path.join(GOLDEN, "lev_pairs.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            a, b, d, note = line.split()
            rows.append(("" if a == "-" else a, "" if b == "-" else b, int(d), note))
    return rows


@pytest.mark.parametrize("a,b,d,note", read_lev_pairs())
def test_lev_hand_worked(oracle_lib, a, b, d, note):
    assert oracle.lev(a, b, lib=oracle_lib) == d
    assert oracle.lev(b, a, lib=oracle_lib) == d


def test_lev_metric_invariants(oracle_lib):
    rng = random.Random(7)
    rep = generate_config1(600, seed=3).strings()
    strs = rep + ["".join(rng.choice("ACDE") for _ in range(rng.randint(0, 9))) for _ in range(300)]
    for _ in range(4000):
        a, b, c = rng.choice(strs), rng.choice(strs), rng.choice(strs)
        ab = oracle.lev(a, b, lib=oracle_lib)
        assert ab == oracle.lev(b, a, lib=oracle_lib)
        assert oracle.lev(a, a, lib=oracle_lib) == 0
        assert abs(len(a) - len(b)) <= ab <= max(len(a), len(b))
        assert (ab == 0) == (a == b)
        ac = oracle.lev(a, c, lib=oracle_lib)
        cb = oracle.lev(c, b, lib=oracle_lib)
        assert ab <= ac + cb


def test_hamming_special_case(oracle_lib):
    """Equal length: lev <= Hamming always, and lev <= 1 iff Hamming <= 1. The
    paper calls the equal-length distance a Hamming distance; ABAB/BABA shows the
    two differ in general (lev 2, Hamming 4), which is why the oracle never uses
    Hamming."""
    rng = random.Random(11)
    for _ in range(3000):
        L = rng.randint(1, 8)
        a = "".join(rng.choice("ACG") for _ in range(L))
        b = "".join(rng.choice("ACG") for _ in range(L))
        ham = sum(x != y for x, y in zip(a, b))
        d = oracle.lev(a, b, lib=oracle_lib)
        assert d <= ham
        assert (d <= 1) == (ham <= 1)
    assert oracle.lev("ABAB", "BABA", lib=oracle_lib) == 2


# ---------------------------------------------------------------------------
# Pins on the network
# ---------------------------------------------------------------------------

def read_adjacency_golden():
    mat, edges, strings = [], None, None
    with open(os.path.join(GOLDEN, "adjacency_5node.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("edges"):
                edges = [tuple(int(x) for x in e.split("-")) for e in line.split()[1:]]
            elif line.startswith("strings"):
                strings = line.split()[1:]
            else:
                mat.append([int(x) for x in line.split()])
    return np.array(mat), edges, strings


def test_adjacency_example_golden(oracle_lib):
    mat, edges, strings = read_adjacency_golden()
    # the printed matrix is the printed edge set
    rebuilt = np.zeros((5, 5), dtype=int)
    for u, v in edges:
        rebuilt[u - 1, v - 1] = rebuilt[v - 1, u - 1] = 1
    assert (rebuilt == mat).all()
    rep = from_strings(strings)
    off, cols, deg = oracle.network(rep.chars, rep.offsets, max_dist=1, lib=oracle_lib)
    got = np.zeros((5, 5), dtype=int)
    for i in range(5):
        got[i, cols[off[i]:off[i + 1]]] = 1
    assert (got == mat).all()
    assert list(off) == [0, 2, 4, 5, 6, 8]
    assert list(cols) == [1, 2, 0, 4, 0, 4, 1, 3]
    assert list(deg) == [2, 2, 1, 1, 2]


def check_graph_invariants(off, cols, n):
    assert off[0] == 0 and off.shape[0] == n + 1
    assert (np.diff(off) >= 0).all()
    rows = lists_of(off, cols)
    edges = set()
    for i, r in enumerate(rows):
        assert all(r[k] < r[k + 1] for k in range(len(r) - 1)), "row not strictly ascending"
        assert i not in r, "self-loop"
        for j in r:
            edges.add((i, j))
    for (i, j) in edges:
        assert (j, i) in edges, "asymmetric"
    assert len(edges) == off[-1] and len(edges) % 2 == 0


def test_threshold0_is_identical_groups(oracle_lib):
    rep = generate_config1(3000, seed=5)
    strs = rep.strings()
    off, cols, _ = oracle.network(rep.chars, rep.offsets, max_dist=0, lib=oracle_lib)
    groups: dict[str, list[int]] = {}
    for i, s in enumerate(strs):
        groups.setdefault(s, []).append(i)
    for i, s in enumerate(strs):
        assert list(cols[off[i]:off[i + 1]]) == [j for j in groups[s] if j != i]
    check_graph_invariants(off, cols, len(strs))


def _edit_graph(strs, alphabet):
    index: dict[str, list[int]] = {}
    for i, s in enumerate(strs):
        index.setdefault(s, []).append(i)
    rows = []
    for i, s in enumerate(strs):
        nb = set()
        for t in one_edit_neighbourhood(s, alphabet):
            nb.update(index.get(t, ()))
        nb.discard(i)
        rows.append(sorted(nb))
    return rows


def test_threshold1_is_one_edit_neighbourhood(oracle_lib):
    rep = generate_config1(2500, seed=9)
    strs = rep.strings()
    # add homopolymer runs and duplicates, where deletion variants coincide
    extra = ["CAAAF", "CAAF", "CAAAAF", "CAF", "CAAF", "CABAF", "CBAAF", "AAB", "AB", "AAA", "AA"]
    strs = strs + extra
    rep = from_strings(strs)
    off, cols, deg = oracle.network(rep.chars, rep.offsets, max_dist=1, lib=oracle_lib)
    assert lists_of(off, cols) == _edit_graph(strs, ALPHABET + "B")
    check_graph_invariants(off, cols, len(strs))
    assert deg.sum() == off[-1]


def test_threshold2_matches_recurrence_tiny(oracle_lib):
    strs = all_strings("AC", 4)
    rep = from_strings(strs)
    off, cols, _ = oracle.network(rep.chars, rep.offsets, max_dist=2, lib=oracle_lib)
    for i, a in enumerate(strs):
        want = [j for j, b in enumerate(strs) if j != i and lev_recursive(a, b) <= 2]
        assert list(cols[off[i]:off[i + 1]]) == want


def test_queries_against_repertoire(oracle_lib):
    rep = generate_config1(1500, seed=13)
    strs = rep.strings()
    rng = random.Random(3)
    qs = [rng.choice(strs) for _ in range(40)]
    qs += [q[:-1] for q in qs[:10]] + [q + "A" for q in qs[10:20]] + ["CASSF", "W"]
    qrep = from_strings(qs)
    qoff, qcols = oracle.neighbors(rep.chars, rep.offsets, qrep.chars, qrep.offsets,
                                   max_dist=1, lib=oracle_lib)
    index: dict[str, list[int]] = {}
    for i, s in enumerate(strs):
        index.setdefault(s, []).append(i)
    for k, q in enumerate(qs):
        want = set()
        for t in one_edit_neighbourhood(q, ALPHABET):
            want.update(index.get(t, ()))
        assert list(qcols[qoff[k]:qoff[k + 1]]) == sorted(want)


def test_rows_equal_full_network_rows(oracle_lib):
    rep = generate_config1(2000, seed=21)
    off, cols, _ = oracle.network(rep.chars, rep.offsets, lib=oracle_lib)
    pick = np.array([0, 5, 17, 1999, 1000, 3], dtype=np.int64)
    roff, rcols = oracle.rows(rep.chars, rep.offsets, pick, lib=oracle_lib)
    for k, i in enumerate(pick):
        assert list(rcols[roff[k]:roff[k + 1]]) == list(cols[off[i]:off[i + 1]])


def test_empty_and_single(oracle_lib):
    rep = from_strings([])
    off, cols, deg = oracle.network(rep.chars, rep.offsets, lib=oracle_lib)
    assert list(off) == [0] and cols.size == 0
    rep = from_strings(["CASSF"])
    off, cols, deg = oracle.network(rep.chars, rep.offsets, lib=oracle_lib)
    assert list(off) == [0, 0] and cols.size == 0


# ---------------------------------------------------------------------------
# Pins on the CPU baseline (the paper's early-abort test, timed by the bench)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("alphabet,max_len", [("AC", 6), ("ACG", 4)])
def test_baseline_within_matches_recurrence_bruteforce(oracle_lib, alphabet, max_len):
    """The row-minimum abort and the length skip change the work, never the
    answer: lev(a, b) <= T for every pair and every T in 0..3."""
    strs = all_strings(alphabet, max_len)
    for a in strs:
        for b in strs:
            d = lev_recursive(a, b)
            for t in range(4):
                assert oracle.baseline_within(a, b, t, lib=oracle_lib) == (d <= t), (a, b, t)


@pytest.mark.parametrize("threshold", [0, 1, 2])
def test_baseline_network_equals_oracle(oracle_lib, threshold):
    strs = generate_config1(1500, seed=41).strings() + ["CAAAF", "CAAF", "AAB", "AB", "W" * 30, "W" * 29]
    rep = from_strings(strs)
    off, cols, _ = oracle.network(rep.chars, rep.offsets, max_dist=threshold, lib=oracle_lib)
    boff, bcols, _ = oracle.baseline_network(rep.chars, rep.offsets, max_dist=threshold, lib=oracle_lib)
    assert np.array_equal(off, boff) and np.array_equal(cols, bcols)
    # one core gives the same lists
    rows_ = np.array([0, 7, 1499, 1500], dtype=np.int64)
    r1 = oracle.baseline_rows(rep.chars, rep.offsets, rows_, max_dist=threshold, nthreads=1, lib=oracle_lib)
    r2 = oracle.rows(rep.chars, rep.offsets, rows_, max_dist=threshold, lib=oracle_lib)
    assert np.array_equal(r1[0], r2[0]) and np.array_equal(r1[1], r2[1])
