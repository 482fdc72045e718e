"""GPU analytics on the device CSR against the CPU oracle (bit-exact labels,
component counts and LCC sizes; neighbour-degree means to 1e-12).

The reference analyses run on the oracle's own network (oracle.network), not
on the CSR the library built, so the comparison reaches from the strings to
the analysis (Methods "Computing LCC" and "Overview of network theory
concepts")."""

import functools

import numpy as np
import pytest

import oracle
from oracle import analytics
import paper_2112_06613_b300 as tn
from synthgen import from_strings, generate_config1

from csr_util import assert_csr_equal

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def oracle_case(n, seed, threshold):
    rep = generate_config1(n, seed=seed)
    off, cols, deg = oracle.network(rep.chars, rep.offsets, max_dist=threshold)
    return rep, off, cols


@pytest.mark.parametrize("method,threshold", [("deletion", 1), ("tile", 1), ("tile", 2), ("deletion", 2)])
def test_components_and_removal(method, threshold):
    rep, off, cols = oracle_case(20_000, 81, threshold)
    with tn.tcrnet_build_flat(rep.chars, rep.offsets, threshold, method=method) as g:
        goff, gcols, _ = g.copy_csr()
        assert_csr_equal(goff, gcols, off, cols, f"{method} T={threshold} network")
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


def test_components_on_kept_edges_after_rejected_candidates():
    # the edges between distinct strings that a handle keeps for the analytics
    # are gathered without the join's rejected candidates
    rep, off, cols = oracle_case(20_000, 81, 1)
    with tn.tcrnet_build_flat(rep.chars, rep.offsets, 1, method="deletion", record_hash_bits=3) as g:
        goff, gcols, _ = g.copy_csr()
        assert_csr_equal(goff, gcols, off, cols, "3-bit record hashes")
        assert g.stats()["rejected_candidates"] > 0
        with tn.tcrnet_build_flat(rep.chars, rep.offsets, 1, method="deletion") as full:
            assert g.stats()["unique_edges"] == full.stats()["unique_edges"]
        labels, nc, lcc = g.components()
        ref = analytics.components(off, cols)
        assert np.array_equal(labels, ref)
        assert (nc, lcc) == analytics.largest_component(ref)
        keep = (np.random.default_rng(6).random(rep.n) >= 0.5).astype(np.uint8)
        labels, _, _ = g.components(keep)
        assert np.array_equal(labels, analytics.components(off, cols, keep))


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
    rep, off, cols = oracle_case(20_000, 82, threshold)
    with tn.tcrnet_build_flat(rep.chars, rep.offsets, threshold) as g:
        knn = g.neighbor_degree()
    ref = analytics.neighbor_degree(off, cols)
    assert np.allclose(knn, ref, rtol=0, atol=1e-12)


def _k_clique_tile(n):
    """n identical strings built by the tile method: the complete graph K_n on
    the n-node CSR, where many edges race to link the same roots."""
    return tn.tcrnet_build(["CASSLGQETQYF"] * n, 1, method="tile")


def test_union_find_gives_up_with_etimeout_and_stays_usable():
    """The bounded link loop of the components kernel, with its bound lowered
    to one attempt per edge (options.link_attempts), runs out on a contended
    complete graph: the kernel records it and returns, the call reports
    TCRNET_ETIMEOUT, nothing waits without a bound, and the same handle then
    answers a normal call exactly."""
    n = 2000
    with _k_clique_tile(n) as g:
        assert g.stats()["method"] == tn.METHOD_TILE
        seen = None
        for _ in range(20):
            try:
                labels, nc, lcc = g.components(link_attempts=1)
            except tn.TcrnetError as e:
                seen = e.status
                break
            # an attempt that met no contention is still exact
            assert (nc, lcc) == (1, n) and (labels == 0).all()
        assert seen == tn.ETIMEOUT
        labels, nc, lcc = g.components()
        assert (nc, lcc) == (1, n) and (labels == 0).all()
    # other handles and calls are unaffected
    rep, off, cols = oracle_case(3_000, 84, 1)
    with tn.tcrnet_build_flat(rep.chars, rep.offsets, 1) as g:
        labels, nc, lcc = g.components()
    ref = analytics.components(off, cols)
    assert np.array_equal(labels, ref) and (nc, lcc) == analytics.largest_component(ref)


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
