"""Serving: inserts into a resident network and the continuous-batching engine.

Bar: bit-exact. After inserts the handle equals a fresh build of the
concatenated input; every query result is the same alone and in the mix."""

from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2112_06613_b300 as tn
from paper_2112_06613_b300.serving import ServingEngine, latency_summary
from synthgen import from_strings, generate_config1

from csr_util import assert_csr_equal, check_invariants

pytestmark = pytest.mark.gpu


def csr_of(g):
    off, cols, deg = g.copy_csr()
    return np.asarray(off, dtype=np.int64), cols, deg


def concat(*reps):
    strs = []
    for r in reps:
        strs += r.strings()
    return from_strings(strs)


@pytest.mark.parametrize("method", ["deletion", "tile"])
def test_inserts_equal_fresh_build(method):
    base = generate_config1(6000, seed=31)
    b1 = generate_config1(1500, seed=32)
    b2 = from_strings(base.strings()[:200] + ["A", "W" * 48, "CASSLGQF"] + b1.strings()[:50])
    with tn.tcrnet_build_flat(base.chars, base.offsets, 1, method=method) as g:
        g.insert_flat(b1.chars, b1.offsets)
        g.insert_flat(b2.chars, b2.offsets)
        off, cols, deg = csr_of(g)
        st = g.stats()
        full = concat(base, b1, b2)
        assert st["n"] == full.n
        with tn.tcrnet_build_flat(full.chars, full.offsets, 1, method=method) as f:
            fo, fc, _ = csr_of(f)
        assert_csr_equal(off, cols, fo, fc, f"inserts vs fresh build ({method})")
        ro, rc, _ = oracle.network(full.chars, full.offsets, max_dist=1)
        assert_csr_equal(off, cols, ro, rc, "inserts vs oracle")
        check_invariants(off, cols, deg, full.n)
        # queries see the inserted strings
        q = from_strings(b2.strings()[:60] + ["WWWWWWWWWWWWWWWWWWWWWWWWWWWWWWWWWWWWWWWWWWWWWWWY"])
        with g.query_flat(q.chars, q.offsets) as r:
            qo, qc, _ = csr_of(r)
        ro, rc = oracle.neighbors(full.chars, full.offsets, q.chars, q.offsets, max_dist=1)
        assert_csr_equal(qo, qc, ro, rc, "queries after inserts")


def test_insert_into_empty_and_bad_insert_keeps_network():
    with tn.tcrnet_build([], 1, method="deletion") as g:
        g.insert(["CASSF", "CASSG", "CASF"])
        off, cols, _ = csr_of(g)
        # CASSF-CASSG (substitution), CASSF-CASF (deletion); CASSG-CASF are two edits apart
        assert list(off) == [0, 2, 3, 4] and list(cols) == [1, 2, 0, 0]
        with pytest.raises(tn.TcrnetError) as e:
            g.insert(["CASSW", "CASXF"])
        assert e.value.status == tn.EBADCHAR and e.value.index == 1
        off2, cols2, _ = csr_of(g)
        assert np.array_equal(off, off2) and np.array_equal(cols, cols2)


def _split(strs, sizes):
    out, k = [], 0
    for s in sizes:
        out.append(from_strings(strs[k:k + s]))
        k += s
    return out


@pytest.mark.parametrize("threshold", [1, 2])
def test_engine_results_same_alone_and_in_mix(threshold):
    base = generate_config1(30_000, seed=41)
    pool = generate_config1(40_000, seed=42).strings()
    pool[::20] = base.strings()[: len(pool[::20])]  # queries with many neighbours as well
    rng = np.random.default_rng(3)
    sizes = [int(x) for x in np.exp(rng.uniform(0, np.log(3000), size=40))]
    reqs_in = _split(pool, sizes)
    with tn.tcrnet_build_flat(base.chars, base.offsets, threshold, method="deletion") as g:
        alone = []
        for q in reqs_in:
            with g.query_flat(q.chars, q.offsets) as r:
                alone.append(csr_of(r)[:2])
        with ServingEngine(g, slots=4, max_batch_strings=20_000) as eng:
            reqs = [eng.query(q.chars, q.offsets) for q in reqs_in]
            for r in reqs:
                assert r.done.wait(120)
        for r, (ao, ac) in zip(reqs, alone):
            assert r.error is None
            assert_csr_equal(r.offsets_out, r.cols_out, ao, ac, "engine vs alone")
        # continuous batching merged some requests into shared device calls
        assert len({r.batch_id for r in reqs}) < len(reqs)
        assert latency_summary(reqs, "query")["count"] == len(reqs)


def test_engine_mixed_queries_and_inserts_versions():
    base = generate_config1(2000, seed=51)
    ins = [generate_config1(300, seed=52), generate_config1(250, seed=53)]
    qpool = generate_config1(3000, seed=54).strings() + base.strings()[:100]
    qs = _split(qpool, [40, 7, 120, 1, 60, 33, 300, 2, 90, 15])
    versions = [base]
    for b in ins:
        versions.append(concat(versions[-1], b))
    with tn.tcrnet_build_flat(base.chars, base.offsets, 1, method="deletion") as g:
        with ServingEngine(g, slots=3, max_batch_strings=150) as eng:
            reqs = []
            for k, q in enumerate(qs):
                reqs.append(eng.query(q.chars, q.offsets))
                if k in (2, 6):
                    b = ins[0 if k == 2 else 1]
                    reqs.append(eng.insert(b.chars, b.offsets))
            for r in reqs:
                assert r.done.wait(120)
        assert all(r.error is None for r in reqs)
        inserts = [r for r in reqs if r.kind == "insert"]
        assert [r.version for r in inserts] == [0, 1]
        for r in reqs:
            if r.kind != "query":
                continue
            rep = versions[r.version]
            ro, rc = oracle.neighbors(rep.chars, rep.offsets, r.chars, r.offsets, max_dist=1)
            assert_csr_equal(r.offsets_out, r.cols_out, ro, rc, f"query at version {r.version}")
        off, cols, _ = csr_of(g)
        final = versions[-1]
        ro, rc, _ = oracle.network(final.chars, final.offsets, max_dist=1)
        assert_csr_equal(off, cols, ro, rc, "final network")


def test_extend_is_copy_on_write():
    base = generate_config1(5000, seed=71)
    add = generate_config1(1200, seed=72)
    with tn.tcrnet_build_flat(base.chars, base.offsets, 1, method="deletion") as g:
        before = csr_of(g)
        with g.extend_flat(add.chars, add.offsets) as g2:
            # the original handle is untouched and still answers queries
            after = csr_of(g)
            assert_csr_equal(after[0], after[1], before[0], before[1], "original after extend")
            full = concat(base, add)
            ro, rc, _ = oracle.network(full.chars, full.offsets, max_dist=1)
            eo, ec, _ = csr_of(g2)
            assert_csr_equal(eo, ec, ro, rc, "extended vs oracle")
            q = from_strings(add.strings()[:40])
            with g2.query_flat(q.chars, q.offsets) as r:
                qo, qc, _ = csr_of(r)
            ro, rc = oracle.neighbors(full.chars, full.offsets, q.chars, q.offsets, max_dist=1)
            assert_csr_equal(qo, qc, ro, rc, "queries on the extended handle")
        with g.extend_flat(np.zeros(0, np.uint8), np.zeros(1, np.int64)) as g3:
            co, cc, _ = csr_of(g3)
            assert_csr_equal(co, cc, before[0], before[1], "empty extension is a copy")
