"""GPU analytics on the device CSR against the CPU oracle (bit-exact labels,
component counts and LCC sizes; neighbour-degree means to 1e-12)."""

import numpy as np
import pytest

import oracle
from oracle import analytics
import paper_2112_06613_b300 as tn
from synthgen import from_strings, generate_config1

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("method,threshold", [("deletion", 1), ("tile", 1), ("tile", 2), ("deletion", 2)])
def test_components_and_removal(method, threshold):
    rep = generate_config1(20_000, seed=81)
    with tn.tcrnet_build_flat(rep.chars, rep.offsets, threshold, method=method) as g:
        off, cols, _ = g.copy_csr()
        off = np.asarray(off, dtype=np.int64)
        labels, nc, lcc = g.components()
        ref = analytics.components(off, cols)
        assert np.array_equal(labels, ref)
        assert (nc, lcc) == analytics.largest_component(ref)
        rng = np.random.default_rng(5)
        for p in (0.1, 0.5, 0.9):
            keep = (rng.random(rep.n) >= p).astype(np.uint8)
            labels, nc, lcc = g.components(keep)
            ref = analytics.components(off, cols, keep)
            assert np.array_equal(labels, ref), p
            assert (nc, lcc) == analytics.largest_component(ref)


def test_components_edge_cases():
    with tn.tcrnet_build(["CASSF"] * 50 + ["W", "Y", "WY"], 1, method="deletion") as g:
        labels, nc, lcc = g.components()
        assert nc == 2 and lcc == 50 and labels[50] == 50 and labels[52] == 50
        labels, nc, lcc = g.components(np.zeros(53, dtype=np.uint8))
        assert nc == 0 and lcc == 0 and (labels == -1).all()
    with tn.tcrnet_build([], 1) as g:
        labels, nc, lcc = g.components()
        assert labels.size == 0 and nc == 0 and lcc == 0


@pytest.mark.parametrize("threshold", [1, 2])
def test_neighbor_degree(threshold):
    rep = generate_config1(20_000, seed=82)
    with tn.tcrnet_build_flat(rep.chars, rep.offsets, threshold) as g:
        off, cols, _ = g.copy_csr()
        knn = g.neighbor_degree()
    ref = analytics.neighbor_degree(np.asarray(off, dtype=np.int64), cols)
    assert np.allclose(knn, ref, rtol=0, atol=1e-12)


@pytest.fixture(scope="module")
def hist_case():
    rep = generate_config1(12_000, seed=83)
    _, _, odeg = oracle.network(rep.chars, rep.offsets, max_dist=1)
    return rep, np.bincount(np.asarray(odeg, dtype=np.int64))


@pytest.mark.parametrize("nbins", [None, 1, 7, 5000, 70_000])
def test_degree_histogram_against_oracle_degrees(hist_case, nbins):
    rep, full = hist_case
    with tn.tcrnet_build_flat(rep.chars, rep.offsets, 1, method="deletion") as g:
        hist = g.degree_histogram(nbins)
    if nbins is None:
        assert np.array_equal(hist, full)
        return
    want = np.zeros(nbins, dtype=np.int64)
    k = min(nbins - 1, full.shape[0])
    want[:k] = full[:k]
    want[nbins - 1] += full[nbins - 1:].sum()
    assert np.array_equal(hist, want)
    assert hist.sum() == rep.n


def test_degree_histogram_empty_and_isolated():
    with tn.tcrnet_build([], 1) as g:
        assert list(g.degree_histogram(3)) == [0, 0, 0]
    with tn.tcrnet_build(["W", "CASSF", "CASSG", "CASSG"], 1) as g:
        assert list(g.degree_histogram()) == [1, 0, 3]
