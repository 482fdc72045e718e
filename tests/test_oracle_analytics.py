"""Pins for the analytics oracle: networkx on the same graphs."""

import networkx as nx
import numpy as np

import oracle
from oracle import analytics
from synthgen import generate_config1


def _graph(n=1500, seed=3):
    rep = generate_config1(n, seed=seed)
    off, cols, _ = oracle.network(rep.chars, rep.offsets, max_dist=1)
    G = nx.Graph()
    G.add_nodes_from(range(rep.n))
    for i in range(rep.n):
        for j in cols[off[i]:off[i + 1]]:
            G.add_edge(i, int(j))
    return off, cols, G


def test_components_match_networkx():
    off, cols, G = _graph()
    labels = analytics.components(off, cols)
    for comp in nx.connected_components(G):
        m = min(comp)
        assert all(labels[i] == m for i in comp)
    nc, lcc = analytics.largest_component(labels)
    assert nc == nx.number_connected_components(G)
    assert lcc == max(len(c) for c in nx.connected_components(G))


def test_components_with_removal_match_networkx():
    off, cols, G = _graph(seed=4)
    rng = np.random.default_rng(0)
    keep = rng.random(len(G)) > 0.4
    labels = analytics.components(off, cols, keep)
    H = G.subgraph([i for i in range(len(G)) if keep[i]])
    for comp in nx.connected_components(H):
        m = min(comp)
        assert all(labels[i] == m for i in comp)
    assert all(labels[i] == -1 for i in range(len(G)) if not keep[i])


def test_neighbor_degree_matches_networkx():
    off, cols, G = _graph(seed=5)
    knn = analytics.neighbor_degree(off, cols)
    ref = nx.average_neighbor_degree(G)
    assert np.allclose(knn, [ref[i] for i in range(len(G))], rtol=0, atol=1e-12)


def test_lcc_normalisation_definitions():
    n1, n2 = analytics.lcc_normalised(300, 1000, 0.5, 800)
    assert n1 == 300 / 500 and n2 == (300 / 500) / (800 / 1000)
