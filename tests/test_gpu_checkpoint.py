"""Checkpoint / resume: a saved handle restored from its file gives the same
network, the same query answers and accepts inserts (bit-exact)."""

from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2112_06613_b300 as tn
from synthgen import from_strings, generate_batched, generate_config1

from csr_util import assert_csr_equal

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("method,n,threshold", [("deletion", 6000, 1), ("tile", 1500, 1), ("tile", 1200, 2),
                                                ("deletion", 3000, 0), ("deletion", 4000, 2)])
def test_save_load_round_trip(tmp_path, method, n, threshold):
    rep = generate_config1(n, seed=101)
    path = str(tmp_path / "net.tcr")
    q = from_strings(generate_config1(300, seed=102).strings() + rep.strings()[:20])
    add = generate_config1(500, seed=103)
    with tn.tcrnet_build_flat(rep.chars, rep.offsets, threshold, method=method) as g:
        ref = g.copy_csr()
        with g.query_flat(q.chars, q.offsets) as r:
            qref = r.copy_csr()
        keep = (np.random.default_rng(5).random(n) >= 0.3).astype(np.uint8)
        labels, nc, lc = g.components(keep)
        comps = (nc, lc)
        knn = g.neighbor_degree()
        g.save(path)
    with tn.tcrnet_load(path) as h:
        got = h.copy_csr()
        assert_csr_equal(got[0], got[1], ref[0], ref[1], "restored network")
        assert np.array_equal(got[2], ref[2])
        assert h.stats()["method"] == tn.METHODS[method]
        with h.query_flat(q.chars, q.offsets) as r:
            qgot = r.copy_csr()
        assert_csr_equal(qgot[0], qgot[1], qref[0], qref[1], "queries on the restored handle")
        keep = (np.random.default_rng(5).random(n) >= 0.3).astype(np.uint8)
        assert h.components(keep)[1:] == comps
        assert np.array_equal(h.components(keep)[0], labels)
        assert np.array_equal(h.neighbor_degree(), knn)
        h.insert_flat(add.chars, add.offsets)
        full = from_strings(rep.strings() + add.strings())
        fo, fc, _ = h.copy_csr()
        oo, oc, _ = oracle.network(full.chars, full.offsets, max_dist=threshold)
        assert_csr_equal(fo, fc, oo, oc, "insert after restore")


def test_save_load_batched_and_query_result_refused(tmp_path):
    reps = generate_batched(6, seed=104, lo=100, hi=2000)
    strs, bounds = [], [0]
    for r in reps:
        strs += r.strings()
        bounds.append(len(strs))
    flat = from_strings(strs)
    path = str(tmp_path / "b.tcr")
    with tn.tcrnet_build_batched(flat.chars, flat.offsets, np.array(bounds, np.int64), 1) as g:
        ref = g.copy_csr()
        g.save(path)
        with tn.tcrnet_build(["CASSF", "CASSG"], 1) as small:
            with small.query(["CASSF"]) as r:
                with pytest.raises(tn.TcrnetError) as e:
                    r.save(str(tmp_path / "q.tcr"))
                assert e.value.status == tn.ESTATE
    with tn.tcrnet_load(path) as h:
        got = h.copy_csr()
        assert_csr_equal(got[0], got[1], ref[0], ref[1], "restored batched network")
        with pytest.raises(tn.TcrnetError) as e:
            h.query(["CASSF"])
        assert e.value.status == tn.ESTATE
