"""Merged inserts: new strings are merged into a deletion build's network and
index (index grown first, closed rows of the new strings' distinct strings from
a query against it, old rows grown at their ends) instead of a rebuild.

Bar: bit-exact. After any sequence of merged inserts the CSR, degrees, query
answers, components and neighbour degrees equal those of a fresh build of the
concatenated input (and the oracle's network); the index statistics (distinct
strings, records, edges between distinct strings) equal the fresh build's."""

from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2112_06613_b300 as tn
from synthgen import from_strings, generate, generate_config1

from csr_util import assert_csr_equal, check_invariants

pytestmark = pytest.mark.gpu


def csr_of(g):
    off, cols, deg = g.copy_csr()
    return np.asarray(off, dtype=np.int64), cols, deg


def fresh(strs, **kw):
    rep = from_strings(strs)
    return tn.tcrnet_build_flat(rep.chars, rep.offsets, 1, method="deletion", **kw)


def assert_same_as_fresh(g, strs, label, oracle_check=True):
    off, cols, deg = csr_of(g)
    check_invariants(off, cols, deg, len(strs))
    with fresh(strs) as f:
        fo, fc, fd = csr_of(f)
        fst = f.stats()
    assert_csr_equal(off, cols, fo, fc, f"{label}: merged vs fresh build")
    assert np.array_equal(deg, fd)
    st = g.stats()
    for k in ("n", "nnz", "n_unique", "n_records", "unique_edges"):
        assert st[k] == fst[k], (label, k, st[k], fst[k])
    if oracle_check:
        rep = from_strings(strs)
        ro, rc, _ = oracle.network(rep.chars, rep.offsets, max_dist=1)
        assert_csr_equal(off, cols, ro, rc, f"{label}: merged vs oracle")


def test_merged_insert_edge_cases():
    base = generate_config1(5000, seed=201).strings()
    # resident duplicates, duplicates inside the batch, strings one edit from
    # resident hubs, the shortest and longest strings, a run-heavy string
    hub = base[0]
    batch = (base[:30] + base[100:105] * 3 + [hub[:-1], hub + "A", "A" + hub, hub[:3] + "W" + hub[4:]] * 2
             + ["A", "C", "AA", "W" * 48, "W" * 47 + "Y", "SSSSSSSSSS", "SSSSSSSSS"])
    with fresh(base) as g:
        assert g.stats()["merged_inserts"] == 0
        b = from_strings(batch)
        g.insert_flat(b.chars, b.offsets, merge=True)
        assert g.stats()["merged_inserts"] == 1
        assert_same_as_fresh(g, base + batch, "edge cases")


def test_many_small_merged_inserts_and_queries():
    base = generate_config1(20_000, seed=202).strings()
    # later draws of the same template model: the new strings join the network
    pool = generate(6000, seed=203, template_seed=202).strings() + base[:500]
    rng = np.random.default_rng(7)
    rng.shuffle(pool)
    strs = list(base)
    k = 0
    with fresh(base) as g:
        for step in range(24):
            size = int(rng.integers(1, 400))
            batch = pool[k:k + size]
            k += size
            b = from_strings(batch)
            g.insert_flat(b.chars, b.offsets, merge=True)
            strs += batch
            assert g.stats()["merged_inserts"] == step + 1
            if step % 8 == 7:
                assert_same_as_fresh(g, strs, f"after insert {step}", oracle_check=(step == 23))
        # queries against the merged index equal the oracle's neighbour lists
        q = from_strings(pool[:300] + generate_config1(300, seed=204).strings() + ["CASSF", "W" * 48])
        full = from_strings(strs)
        with g.query_flat(q.chars, q.offsets) as r:
            qo, qc, _ = csr_of(r)
        ro, rc = oracle.neighbors(full.chars, full.offsets, q.chars, q.offsets, max_dist=1)
        assert_csr_equal(qo, qc, ro, rc, "queries after merged inserts")


def test_merged_insert_analytics_and_checkpoint(tmp_path):
    base = generate_config1(8000, seed=205).strings()
    add = generate(200, seed=206, template_seed=205).strings() + base[:50]
    b = from_strings(add)
    strs = base + add
    keep = (np.random.default_rng(9).random(len(strs)) >= 0.25).astype(np.uint8)
    with fresh(strs) as f:
        ref_comp = f.components(keep)
        ref_all = f.components()
        ref_knn = f.neighbor_degree()
        ref_hist = f.degree_histogram()
    with fresh(base) as g:
        g.insert_flat(b.chars, b.offsets, merge=True)
        assert g.stats()["merged_inserts"] == 1
        comp = g.components(keep)
        assert np.array_equal(comp[0], ref_comp[0]) and comp[1:] == ref_comp[1:]
        allc = g.components()
        assert np.array_equal(allc[0], ref_all[0]) and allc[1:] == ref_all[1:]
        assert np.array_equal(g.neighbor_degree(), ref_knn)
        assert np.array_equal(g.degree_histogram(), ref_hist)
        path = str(tmp_path / "merged.tcr")
        g.save(path)
    with tn.tcrnet_load(path) as h:
        assert h.stats()["merged_inserts"] == 1
        assert_same_as_fresh(h, strs, "restored merged handle", oracle_check=False)
        more = generate(200, seed=207, template_seed=205).strings()
        mb = from_strings(more)
        h.insert_flat(mb.chars, mb.offsets, merge=True)
        assert h.stats()["merged_inserts"] == 2
        assert_same_as_fresh(h, strs + more, "insert after restore")


def test_merged_insert_int64_offsets_and_rebuild_option():
    base = generate_config1(6000, seed=208).strings()
    add = generate(150, seed=209, template_seed=208).strings()
    b = from_strings(add)
    rep = from_strings(base)
    with tn.tcrnet_build_flat(rep.chars, rep.offsets, 1, method="deletion", force_offsets64=True) as g:
        g.insert_flat(b.chars, b.offsets, merge=True)
        assert g.info()[2] == 1 and g.stats()["merged_inserts"] == 1
        assert_same_as_fresh(g, base + add, "int64 offsets", oracle_check=False)
    with fresh(base) as g:
        g.insert_flat(b.chars, b.offsets, rebuild=True)
        assert g.stats()["merged_inserts"] == 0
        merged = None
        with fresh(base) as g2:
            with g2.extend_flat(b.chars, b.offsets, merge=True) as g3:
                assert g3.stats()["merged_inserts"] == 1
                merged = csr_of(g3)
            # copy-on-write: the source handle is unchanged
            assert_same_as_fresh(g2, base, "source of a merged extend", oracle_check=False)
        rb = csr_of(g)
        assert_csr_equal(merged[0], merged[1], rb[0], rb[1], "merged vs rebuilt insert")


def test_large_insert_rebuilds():
    base = generate_config1(3000, seed=210).strings()
    add = generate_config1(4000, seed=211).strings()  # larger than the repertoire: rebuilt
    b = from_strings(add)
    with fresh(base) as g:
        small = from_strings(add[:80])
        g.insert_flat(small.chars, small.offsets, merge=True)
        assert g.stats()["merged_inserts"] == 1
        g.insert_flat(b.chars, b.offsets)  # automatic choice
        assert g.stats()["merged_inserts"] == 0
        assert_same_as_fresh(g, base + add[:80] + add, "rebuild after merge", oracle_check=False)


def test_merged_insert_allocation_failures_keep_the_handle():
    """Every device allocation of a merged insert in turn fails: the call returns
    TCRNET_ENOMEM and the handle keeps its network; then the insert succeeds."""
    import ctypes

    base = generate_config1(3000, seed=212).strings()
    add = generate(60, seed=213, template_seed=212).strings() + base[:5]
    b = from_strings(add)
    lib = tn.load_library()
    with fresh(base) as g:
        before = csr_of(g)
        failures = 0
        for k in range(1, 400):
            opt = tn.make_options(fail_alloc_at=k, insert_rebuild="merge")
            st = lib.tcrnet_insert_ex(g.handle, b.chars.ctypes.data, b.offsets.ctypes.data, b.n, tn.HOST,
                                      ctypes.byref(opt))
            if st == tn.OK:
                break
            assert st == tn.ENOMEM, (k, st)
            failures += 1
            after = csr_of(g)
            assert_csr_equal(after[0], after[1], before[0], before[1], f"merged insert fail_alloc_at={k}")
        assert failures >= 20
        assert g.stats()["merged_inserts"] == 1
        assert_same_as_fresh(g, base + add, "merged insert after failures")


def test_merged_insert_of_resident_strings_only():
    """Every new string equals a resident one: no fresh distinct string, no new
    record; the copies join the member lists and the rows of their strings."""
    base = generate_config1(5000, seed=214).strings()
    add = base[:100] + base[:7] * 5
    b = from_strings(add)
    with fresh(base) as g:
        n_unique = g.stats()["n_unique"]
        g.insert_flat(b.chars, b.offsets, merge=True)
        st = g.stats()
        assert st["merged_inserts"] == 1 and st["n_unique"] == n_unique
        assert_same_as_fresh(g, base + add, "resident strings only")


def test_random_merged_inserts_over_a_tiny_alphabet():
    """Strings of 1..7 letters over three letters: many duplicates, runs and
    hubs. Random sequences of merged inserts, each compared with a fresh build."""
    rng = np.random.default_rng(215)

    def draw(k):
        lens = rng.integers(1, 8, size=k)
        return ["".join(rng.choice(list("ACD"), size=int(L))) for L in lens]

    for trial in range(6):
        base = draw(2400)
        strs = list(base)
        with fresh(base) as g:
            for step in range(5):
                add = draw(int(rng.integers(1, len(strs) // 32 + 1)))
                b = from_strings(add)
                g.insert_flat(b.chars, b.offsets, merge=True)
                strs += add
                assert g.stats()["merged_inserts"] == step + 1
            assert_same_as_fresh(g, strs, f"tiny alphabet trial {trial}", oracle_check=(trial == 0))
            q = from_strings(draw(200))
            with g.query_flat(q.chars, q.offsets) as r:
                qo, qc, _ = csr_of(r)
            full = from_strings(strs)
            ro, rc = oracle.neighbors(full.chars, full.offsets, q.chars, q.offsets, max_dist=1)
            assert_csr_equal(qo, qc, ro, rc, f"queries, trial {trial}")
