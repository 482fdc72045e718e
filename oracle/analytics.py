"""CPU oracle for the network analytics — TEST INFRASTRUCTURE ONLY.

Plain breadth-first search and averages over a CSR (offsets, cols), following
the definitions of Methods "Overview of network theory concepts" (connected
components, largest connected component, average neighbour degree) and
Methods "Computing LCC" (LCC after node removal and its normalisations).
Pinned against networkx in tests/test_oracle_analytics.py.
"""

from __future__ import annotations

import collections

import numpy as np


def components(off, cols, keep=None):
    """labels[i] = smallest node id of i's component (BFS), -1 if removed."""
    off = np.asarray(off, dtype=np.int64)
    n = off.shape[0] - 1
    keep = np.ones(n, dtype=bool) if keep is None else np.asarray(keep, dtype=bool)
    labels = np.full(n, -1, dtype=np.int64)
    for s in range(n):
        if not keep[s] or labels[s] >= 0:
            continue
        labels[s] = s  # s is the smallest unvisited kept id, so the smallest of its component
        q = collections.deque([s])
        while q:
            i = q.popleft()
            for j in cols[off[i]:off[i + 1]]:
                if keep[j] and labels[j] < 0:
                    labels[j] = s
                    q.append(j)
    return labels


def largest_component(labels):
    lab = labels[labels >= 0]
    if lab.size == 0:
        return 0, 0
    _, counts = np.unique(lab, return_counts=True)
    return int(counts.size), int(counts.max())


def neighbor_degree(off, cols):
    """knn[i] = mean degree of i's neighbours, 0 for isolated nodes."""
    off = np.asarray(off, dtype=np.int64)
    deg = np.diff(off)
    n = deg.shape[0]
    knn = np.zeros(n, dtype=np.float64)
    for i in range(n):
        if deg[i]:
            knn[i] = float(sum(int(deg[j]) for j in cols[off[i]:off[i + 1]])) / float(deg[i])
    return knn


def lcc_normalised(lcc_p, n, p, lcc0):
    """LCC_norm,1(p) = LCC(p) / ((1 - p) N); LCC_norm,2(p) = LCC_norm,1(p) / LCC_norm,1(0)."""
    norm1 = lcc_p / ((1.0 - p) * n)
    return norm1, norm1 / (lcc0 / n)
