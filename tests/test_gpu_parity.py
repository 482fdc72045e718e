"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bar: bit-exact CSR (offsets, cols, degree) — this is integer work.
Full graphs where the oracle finishes in seconds; sampled rows plus global
invariants at the full sizes."""

from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
import paper_2112_06613_b300 as tn
from synthgen import ALPHABET, from_strings, generate, generate_config1

from csr_util import assert_csr_equal, assert_rows_equal, check_invariants, sample_rows

pytestmark = pytest.mark.gpu

METHODS = ["tile", "deletion"]


@pytest.fixture(scope="module", autouse=True)
def _needs_gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    tn.load_library()


def gpu_csr(rep, threshold=1, method="tile", **kw):
    with tn.tcrnet_build_flat(rep.chars, rep.offsets, threshold=threshold, method=method, **kw) as g:
        off, cols, deg = g.copy_csr()
        st = g.stats()
    return np.asarray(off, dtype=np.int64), cols, deg, st


def oracle_csr(rep, threshold=1):
    off, cols, deg = oracle.network(rep.chars, rep.offsets, max_dist=threshold)
    return off, cols, deg


def single_length(n, L, seed=0):
    """n generator strings that all have length L (one bucket)."""
    out = []
    s = seed
    while len(out) < n:
        r = generate(4 * n, seed=s, len_lo=L, len_hi=L)
        out.extend(r.strings())
        s += 1000
    return from_strings(out[:n])


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("threshold", [0, 1])
def test_config1_full_graph(method, threshold):
    rep = generate_config1(10_000, seed=0)
    off, cols, deg, st = gpu_csr(rep, threshold, method)
    ro, rc, rd = oracle_csr(rep, threshold)
    assert_csr_equal(off, cols, ro, rc, f"config1 {method} T={threshold}")
    assert np.array_equal(deg, rd)
    check_invariants(off, cols, deg, rep.n)


@pytest.mark.parametrize("method", METHODS)
def test_one_bucket_several_tiles_ragged(method):
    # 5000 strings of one length: several 2048-row blocks and 512-column
    # chunks, diagonal items and a ragged tail.
    rep = single_length(5003, 14, seed=3)
    off, cols, deg, _ = gpu_csr(rep, 1, method)
    ro, rc, _ = oracle_csr(rep, 1)
    assert_csr_equal(off, cols, ro, rc, f"single bucket {method}")


@pytest.mark.parametrize("method", METHODS)
def test_two_adjacent_buckets_large(method):
    a = single_length(2600, 12, seed=5).strings()
    b = single_length(2300, 13, seed=6).strings()
    # interleave so input order differs from bucket order
    strs = [x for pair in zip(a, b) for x in pair] + a[len(b):]
    rep = from_strings(strs)
    off, cols, _, _ = gpu_csr(rep, 1, method)
    ro, rc, _ = oracle_csr(rep, 1)
    assert_csr_equal(off, cols, ro, rc, f"buckets 12/13 {method}")


def edge_strings():
    rng = np.random.default_rng(17)
    out = []
    for L in (1, 2, 5, 6, 7, 11, 12, 13, 17, 18, 19, 23, 24, 25, 26, 29, 30, 31, 35, 36, 37, 47, 48):
        base = "".join(rng.choice(list(ALPHABET), size=L))
        out.append(base)
        out.append(base)  # duplicate
        p = int(rng.integers(0, L))
        out.append(base[:p] + ("A" if base[p] != "A" else "C") + base[p + 1:])  # substitution
        out.append(base[:p] + base[p + 1:] if L > 1 else "W")  # deletion
        if L < 48:
            out.append(base[:p] + "Y" + base[p:])  # insertion
        out.append(base[::-1])
    # homopolymer runs and their deletion/insertion variants
    out += ["AAAA", "AAA", "AA", "A", "AAC", "AC", "ACC", "CAA", "CAAAF", "CAAF", "CAAAAF"]
    out += ["W" * 48, "W" * 47, "W" * 30, "W" * 29, "W" * 25, "W" * 24, "W" * 13, "W" * 12]
    return out


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("threshold", [0, 1])
def test_edge_cases_lengths_and_runs(method, threshold):
    rep = from_strings(edge_strings())
    off, cols, deg, _ = gpu_csr(rep, threshold, method)
    ro, rc, _ = oracle_csr(rep, threshold)
    assert_csr_equal(off, cols, ro, rc, f"edge strings {method} T={threshold}")


@pytest.mark.parametrize("method", METHODS)
def test_all_identical_is_complete_graph(method):
    rep = from_strings(["CASSLGQETQYF"] * 700)
    off, cols, deg, _ = gpu_csr(rep, 1, method)
    assert (deg == 699).all()
    ro, rc, _ = oracle_csr(rep, 1)
    assert_csr_equal(off, cols, ro, rc, "identical")


@pytest.mark.parametrize("method", METHODS)
def test_degenerate_sizes(method):
    for strs in ([], ["CASSF"], ["CASSF", "CASSF"], ["CASSF", "CASSG"], ["CASSF", "CAS"]):
        rep = from_strings(strs)
        off, cols, deg, _ = gpu_csr(rep, 1, method)
        ro, rc, _ = oracle_csr(rep, 1)
        assert_csr_equal(off, cols, ro, rc, f"{strs}")


@pytest.mark.parametrize("method", METHODS)
def test_empty_neighbour_buckets(method):
    # lengths 10 and 14 only: no (L, L+1) pairs exist
    a = single_length(800, 10, seed=8).strings()
    b = single_length(900, 14, seed=9).strings()
    rep = from_strings(a + b)
    off, cols, _, _ = gpu_csr(rep, 1, method)
    ro, rc, _ = oracle_csr(rep, 1)
    assert_csr_equal(off, cols, ro, rc, "gapped buckets")


@pytest.mark.parametrize("method", METHODS)
def test_deterministic_and_int64_offsets(method):
    rep = generate_config1(20_000, seed=2)
    o1, c1, d1, _ = gpu_csr(rep, 1, method)
    o2, c2, d2, _ = gpu_csr(rep, 1, method, force_offsets64=True)
    assert_csr_equal(o1, c1, o2, c2, "repeat / int64")
    assert np.array_equal(d1, d2)


def _digests():
    import sys

    sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
    import digests

    return digests


def _check_rows_against_stored(off, cols, section, what, rep):
    """Every stored (row, degree, digest) of an oracle section against the
    build's rows; mismatching rows are recomputed by the live oracle so that
    the failure shows what differs."""
    dg = _digests()
    off = np.asarray(off, dtype=np.int64)
    bad = [i for i, d, h in section["rows"]
           if int(off[i + 1] - off[i]) != d or dg.row_digest(cols[off[i]:off[i + 1]]) != h]
    if bad:
        roff, rcols = oracle.rows(rep.chars, rep.offsets, np.array(bad[:5], dtype=np.int64))
        assert_rows_equal(off, cols, bad[:5], roff, rcols, f"{what} (live oracle)")
        raise AssertionError(f"{what}: {len(bad)} rows differ from the stored oracle digests, first {bad[:5]}")


def test_full_1e5_network_equals_oracle():
    """Every row of the N = 100,000 network against the oracle's (stored as
    block digests by tests/golden/make_parity_digests.py, which calls only the
    oracle), by both methods; plus a live oracle comparison of sampled rows."""
    dg = _digests()
    sec = dg.load()["full_1e5"]
    meta = sec["meta"]
    rep = generate_config1(int(meta["n"]), seed=int(meta["seed"]))
    for method in ("auto", "tile"):
        off, cols, deg, st = gpu_csr(rep, 1, method)
        assert st["method"] == (tn.METHOD_DELETION if method == "auto" else tn.METHOD_TILE)
        assert int(off[-1]) == int(meta["nnz"]), f"{method}: nnz"
        check_invariants(off, cols, deg, rep.n)
        bad = [(r0, r1) for r0, r1, h in sec["rows"] if dg.block_digest(off, cols, r0, r1) != h]
        if bad:
            r0, r1 = bad[0]
            ids = np.arange(r0, r1, dtype=np.int64)
            roff, rcols = oracle.rows(rep.chars, rep.offsets, ids)
            assert_rows_equal(off, cols, ids, roff, rcols, f"1e5 {method} block {r0} (live oracle)")
            raise AssertionError(f"1e5 {method}: {len(bad)} blocks differ from the oracle digests")
    rows = sample_rows(deg, 300, seed=1, top=50)
    roff, rcols = oracle.rows(rep.chars, rep.offsets, rows)
    assert_rows_equal(off, cols, rows, roff, rcols, "1e5 sampled rows (live oracle)")


@pytest.mark.parametrize("method", METHODS)
def test_bad_inputs_report_index(method):
    cases = [
        (["CASSF", "CASXF", "CASSB"], tn.EBADCHAR, 1),
        (["CASSF", "cassf"], tn.EBADCHAR, 1),
        (["CASSF", "C" * 49], tn.ETOOLONG, 1),
        (["CASSF", "CASSG", ""], tn.EINVAL, 2),
    ]
    for strs, status, idx in cases:
        with pytest.raises(tn.TcrnetError) as e:
            tn.tcrnet_build(strs, 1, method=method)
        assert e.value.status == status and e.value.index == idx
    # the context is still usable afterwards
    off, cols, deg, _ = gpu_csr(from_strings(["CASSF", "CASSG"]), 1, method)
    assert list(cols) == [1, 0]


def test_string_list_and_device_inputs_agree():
    import torch

    rep = generate_config1(3000, seed=4)
    with tn.tcrnet_build(rep.strings(), 1, method="tile") as g:
        o1, c1, _ = g.copy_csr()
    chars = torch.from_numpy(rep.chars).cuda()
    offs = torch.from_numpy(rep.offsets).cuda()
    with tn.tcrnet_build_flat(chars, offs, 1, method="tile", stream=torch.cuda.current_stream()) as g:
        o2, c2, d2 = g.copy_csr_device()
    assert_csr_equal(o1, c1, o2.cpu().numpy(), c2.cpu().numpy(), "list vs device")


def test_queries_match_oracle():
    rep = generate_config1(20_000, seed=7)
    strs = rep.strings()
    rng = np.random.default_rng(5)
    qs = [strs[i] for i in rng.choice(len(strs), 300, replace=False)]
    qs += [q[:-1] for q in qs[:50]] + [q + "A" for q in qs[50:100]] + ["CASSLGQF", "W", "C" * 48]
    qs += [q[:3] + "W" + q[4:] for q in qs[100:150]]
    q = from_strings(qs)
    with tn.tcrnet_build_flat(rep.chars, rep.offsets, 1, method="tile") as g:
        with g.query_flat(q.chars, q.offsets) as r:
            qo, qc, qd = r.copy_csr()
    ro, rc = oracle.neighbors(rep.chars, rep.offsets, q.chars, q.offsets, max_dist=1)
    assert_csr_equal(qo, qc, ro, rc, "queries")


def test_deletion_exact_fallback_join():
    # a tiny partition capacity sends most partitions to the exact quadratic join
    rep = generate_config1(10_000, seed=11)
    off, cols, deg, st = gpu_csr(rep, 1, "deletion", partition_cap=4)
    assert st["n_fallback"] > 0
    ro, rc, _ = oracle_csr(rep, 1)
    assert_csr_equal(off, cols, ro, rc, "fallback join")


@pytest.mark.parametrize("bits", [1, 6])
def test_deletion_join_rejects_candidates_of_truncated_hashes(bits):
    # with only a few bits of each record's hash kept, variants of different
    # contents in one partition match; the confirmation by content rejects
    # those candidates and the network stays exact
    rep = generate_config1(10_000, seed=13)
    off, cols, deg, st = gpu_csr(rep, 1, "deletion", record_hash_bits=bits)
    ro, rc, rd = oracle_csr(rep, 1)
    assert_csr_equal(off, cols, ro, rc, f"{bits}-bit record hashes")
    assert np.array_equal(deg, rd)
    assert st["rejected_candidates"] > 0  # the truncation did make candidates to reject
    _, _, _, full = gpu_csr(rep, 1, "deletion")
    assert st["unique_edges"] == full["unique_edges"] > 0
    # and with a partition capacity that sends partitions to the quadratic join
    off, cols, _, st = gpu_csr(rep, 1, "deletion", record_hash_bits=bits, partition_cap=4)
    assert st["n_fallback"] > 0
    assert_csr_equal(off, cols, ro, rc, f"{bits}-bit record hashes, quadratic join")


def test_deletion_two_pass_join_with_rejected_candidates():
    # an overflowing candidate list (dense unique graph) whose candidates
    # include rejected ones: the weights come from the second pass only
    letters = list(ALPHABET)
    strs = letters + [a + b for a in letters for b in letters] + ["AA", "C", "CAS"]
    rep = from_strings(strs)
    off, cols, deg, st = gpu_csr(rep, 1, "deletion", record_hash_bits=2)
    assert st["two_pass_join"] == 1 and st["rejected_candidates"] > 0
    ro, rc, _ = oracle_csr(rep, 1)
    assert_csr_equal(off, cols, ro, rc, "dense unique graph, 2-bit record hashes")


@pytest.mark.parametrize("bits", [32, 3])
def test_deletion_two_pass_join_with_multi_tile_scans(bits):
    """Every string of 1..3 letters (8,420 strings, more than one scan tile):
    the one-pass edge buffer overflows, so the second join pass runs and the
    size scans (look-back chains, list cursors, lists of the long sort classes)
    run a second time on the complete weights. bits = 3 adds rejected
    candidates (3-bit record hashes)."""
    letters = list(ALPHABET)
    strs = letters + [a + b for a in letters for b in letters]
    strs += [a + b + c for a in letters for b in letters for c in letters]
    rep = from_strings(strs)
    off, cols, deg, st = gpu_csr(rep, 1, "deletion", record_hash_bits=bits)
    assert st["two_pass_join"] == 1
    if bits < 32:
        assert st["rejected_candidates"] > 0
    ro, rc, _ = oracle_csr(rep, 1)
    assert_csr_equal(off, cols, ro, rc, f"strings of 1..3 letters, {bits}-bit record hashes")
    check_invariants(off, cols, deg, rep.n)


def test_deletion_counts_distinct_strings():
    rep = generate_config1(30_000, seed=12)
    _, _, _, st = gpu_csr(rep, 1, "deletion")
    strs = rep.strings()
    assert st["n_unique"] == len(set(strs))
    assert st["n_records"] == sum(len(s) + 1 for s in set(strs))
    assert st["n_fallback"] == 0


def _device_build(rep, method, **kw):
    import torch

    chars = torch.from_numpy(rep.chars).cuda()
    offs = torch.from_numpy(rep.offsets).cuda()
    g = tn.tcrnet_build_flat(chars, offs, 1, method=method, stream=torch.cuda.current_stream(), **kw)
    return g


def test_full_size_8e5_10000_rows_and_invariants():
    """The configuration bench.py times (N = 800,000, config 2, seed 0, default
    method, device inputs): global invariants in full; 9,900 seeded uniform
    rows against the oracle's lists (stored digests) and the 100 highest-degree
    rows of the build against the live oracle, 10,000 rows in all; 100 of the
    stored rows recomputed live as well; the tile method builds the identical
    network."""
    from synthgen import generate_config2

    dg = _digests()
    sec = dg.load()["rows_8e5"]
    rep = generate_config2(int(sec["meta"]["n"]), seed=int(sec["meta"]["seed"]))
    with _device_build(rep, "auto") as g:
        off, cols, deg = g.copy_csr()
        st = g.stats()
    assert st["method"] == tn.METHOD_DELETION
    off = np.asarray(off, dtype=np.int64)
    check_invariants(off, cols, deg, rep.n)
    assert len(sec["rows"]) == 9_900
    _check_rows_against_stored(off, cols, sec, "8e5 stored oracle rows", rep)
    stored = np.array([i for i, _, _ in sec["rows"]], dtype=np.int64)
    top = np.argsort(-deg, kind="stable")[:100].astype(np.int64)
    live = np.unique(np.concatenate([top, stored[::99]]))
    roff, rcols = oracle.rows(rep.chars, rep.offsets, live)
    assert_rows_equal(off, cols, live, roff, rcols, "8e5 top-degree and stored rows (live oracle)")
    assert len(np.union1d(stored, top)) >= 9_990
    with _device_build(rep, "tile") as g:
        o2, c2, d2 = g.copy_csr()
    assert_csr_equal(off, cols, o2, c2, "tile vs deletion at 8e5")


def test_lmax2_1e6_sampled_rows_and_invariants():
    """l_max = 2 at 1e6 strings (the deletion method's candidates, nnz ~4.4e8):
    global invariants in full, 200 sampled rows plus the 50 highest-degree rows
    against the oracle's full neighbour lists."""
    rep = generate_config1(1_000_000, seed=13)
    with tn.tcrnet_build_flat(rep.chars, rep.offsets, 2) as g:
        assert g.stats()["method"] == tn.METHOD_DELETION
        off, cols, deg = g.copy_csr()
    off = np.asarray(off, dtype=np.int64)
    check_invariants(off, cols, deg, rep.n)
    rows = sample_rows(deg, 200, seed=14, top=50)
    roff, rcols = oracle.rows(rep.chars, rep.offsets, rows, max_dist=2)
    assert_rows_equal(off, cols, rows, roff, rcols, "1e6 l_max=2 sampled rows")


def test_full_size_8e6_1000_rows_int64_offsets():
    """Config 3: N = 8,000,000, insertion 0-9 aa, nnz > 2^31 -> int64 offsets.
    1,000 seeded uniform rows against the oracle (stored digests), the 20
    highest-degree rows and 20 of the stored rows against the live oracle."""
    import torch
    from synthgen import generate_config3

    dg = _digests()
    sec = dg.load()["rows_8e6"]
    rep = generate_config3(int(sec["meta"]["n"]), seed=int(sec["meta"]["seed"]))
    with _device_build(rep, "auto") as g:
        n, nnz, o64 = g.info()
        assert o64 and nnz > 2**31
        off_d, cols_d, deg_d = g.copy_csr_device()
        deg = deg_d.cpu().numpy()
        off_h = off_d.cpu().numpy()
        assert off_h[0] == 0 and off_h[-1] == nnz and np.array_equal(np.diff(off_h), deg)
        assert int(deg.sum()) == nnz and nnz % 2 == 0
        stored = np.array([i for i, _, _ in sec["rows"]], dtype=np.int64)
        top = np.argsort(-deg, kind="stable")[:20].astype(np.int64)
        rows = np.unique(np.concatenate([stored, top]))
        # gather the rows' entries on the device, one copy to the host
        lens = deg[rows].astype(np.int64)
        sub_off = np.zeros(rows.shape[0] + 1, dtype=np.int64)
        np.cumsum(lens, out=sub_off[1:])
        idx = np.repeat(off_h[rows] - sub_off[:-1], lens) + np.arange(sub_off[-1])
        sub_cols = cols_d[torch.from_numpy(idx).to(cols_d.device)].cpu().numpy()
    full_off = np.zeros(rep.n + 1, dtype=np.int64)  # the sampled rows as a sparse CSR over all n
    lens_all = np.zeros(rep.n, dtype=np.int64)
    lens_all[rows] = lens
    np.cumsum(lens_all, out=full_off[1:])
    assert len(sec["rows"]) == 1_000
    _check_rows_against_stored(full_off, sub_cols, sec, "8e6 stored oracle rows", rep)
    live = np.unique(np.concatenate([top, stored[::50]]))
    roff, rcols = oracle.rows(rep.chars, rep.offsets, live)
    assert_rows_equal(full_off, sub_cols, live, roff, rcols, "8e6 top-degree and stored rows (live oracle)")


def test_deletion_dense_unique_graph_takes_two_pass_join():
    # every 1- and 2-letter string: far more edges between distinct strings than
    # records, so the one-pass edge buffer overflows and the exact second pass runs
    letters = list(ALPHABET)
    strs = letters + [a + b for a in letters for b in letters] + ["AA", "C", "CAS"]
    rep = from_strings(strs)
    off, cols, deg, st = gpu_csr(rep, 1, "deletion")
    assert st["two_pass_join"] == 1
    ro, rc, _ = oracle_csr(rep, 1)
    assert_csr_equal(off, cols, ro, rc, "dense unique graph")
    # the generator workload fits in one pass
    _, _, _, st = gpu_csr(generate_config1(5000, seed=3), 1, "deletion")
    assert st["two_pass_join"] == 0


@pytest.mark.parametrize("qmethod", ["auto", "tile", "deletion"])
def test_index_queries_match_oracle(qmethod):
    rep = generate_config1(20_000, seed=17)
    strs = rep.strings()
    rng = np.random.default_rng(8)
    qs = [strs[i] for i in rng.choice(len(strs), 300, replace=False)]
    qs += [q[:-1] for q in qs[:40]] + [q + "A" for q in qs[40:80]] + [q[:2] + q[3:] for q in qs[80:120]]
    qs += [q[:5] + "Y" + q[6:] for q in qs[120:160]] + ["A", "W" * 48, "CASSLGQF", "CAAAF", "CAAF"]
    q = from_strings(qs)
    with tn.tcrnet_build_flat(rep.chars, rep.offsets, 1, method="deletion") as g:
        with g.query_flat(q.chars, q.offsets, method=qmethod) as r:
            qo, qc, _ = r.copy_csr()
            st = r.stats()
    assert st["method"] == (tn.METHOD_TILE if qmethod == "tile" else tn.METHOD_DELETION)
    ro, rc = oracle.neighbors(rep.chars, rep.offsets, q.chars, q.offsets, max_dist=1)
    assert_csr_equal(qo, qc, ro, rc, f"queries via {qmethod}")


def test_index_queries_on_edge_strings():
    strs = edge_strings()
    rep = from_strings(strs)
    qrep = from_strings(strs + ["AAAAA", "AC", "CA", "A" * 47, "Y" * 48])
    with tn.tcrnet_build_flat(rep.chars, rep.offsets, 1, method="deletion") as g:
        with g.query_flat(qrep.chars, qrep.offsets) as r:
            qo, qc, _ = r.copy_csr()
    ro, rc = oracle.neighbors(rep.chars, rep.offsets, qrep.chars, qrep.offsets, max_dist=1)
    assert_csr_equal(qo, qc, ro, rc, "edge-string queries")


def test_query_without_index_rejects_deletion_search():
    rep = generate_config1(1000, seed=1)
    with tn.tcrnet_build_flat(rep.chars, rep.offsets, 1, method="tile") as g:
        with pytest.raises(tn.TcrnetError) as e:
            g.query_flat(rep.chars, rep.offsets, method="deletion")
        assert e.value.status == tn.ENOTSUP


def _all_strings(alphabet, max_len):
    import itertools

    out = []
    for L in range(1, max_len + 1):
        out += ["".join(t) for t in itertools.product(alphabet, repeat=L)]
    return out


@pytest.mark.parametrize("threshold", [2, 3])
def test_larger_threshold_exhaustive_tiny_alphabet(threshold):
    rep = from_strings(_all_strings("AC", 6) + _all_strings("ACD", 3))
    off, cols, deg, st = gpu_csr(rep, threshold, "auto")
    assert st["method"] == tn.METHOD_TILE
    ro, rc, _ = oracle_csr(rep, threshold)
    assert_csr_equal(off, cols, ro, rc, f"tiny alphabet T={threshold}")


@pytest.mark.parametrize("threshold", [2, 3, 6])
def test_larger_threshold_generator_strings(threshold):
    # the paper's analyses use l_max = 2 (assortativity), a sweep, and 6 (LCC drawings)
    rep = generate_config1(3000, seed=60 + threshold)
    off, cols, deg, _ = gpu_csr(rep, threshold, "tile")
    ro, rc, _ = oracle_csr(rep, threshold)
    assert_csr_equal(off, cols, ro, rc, f"generator T={threshold}")
    check_invariants(off, cols, deg, rep.n)


def test_larger_threshold_edge_strings_and_queries():
    rep = from_strings(edge_strings())
    off, cols, _, _ = gpu_csr(rep, 2, "tile")
    ro, rc, _ = oracle_csr(rep, 2)
    assert_csr_equal(off, cols, ro, rc, "edge strings T=2")
    base = generate_config1(4000, seed=71)
    qs = from_strings(base.strings()[:100] + ["CASSF", "A", "W" * 48] + [s[:-2] for s in base.strings()[100:150]])
    with tn.tcrnet_build_flat(base.chars, base.offsets, 2) as g:
        with g.query_flat(qs.chars, qs.offsets) as r:
            qo, qc, _ = r.copy_csr()
    ro, rc = oracle.neighbors(base.chars, base.offsets, qs.chars, qs.offsets, max_dist=2)
    assert_csr_equal(qo, qc, ro, rc, "queries T=2")


@pytest.mark.parametrize("threshold", [2, 3])
def test_larger_threshold_across_the_32_letter_word_boundary(threshold):
    # column strings of <= 32 letters run on 32-bit words, longer ones on 64-bit
    rng = np.random.default_rng(90 + threshold)
    alpha = np.array(list("ACDEFG"))
    strs = []
    for _ in range(300):
        L = int(rng.integers(28, 41))
        s = list(alpha[rng.integers(0, len(alpha), L)])
        strs.append("".join(s))
        for _ in range(3):  # near copies: substitutions, deletions, insertions
            t = list(s)
            for _ in range(int(rng.integers(1, threshold + 2))):
                k = int(rng.integers(0, len(t)))
                op = int(rng.integers(0, 3))
                if op == 0:
                    t[k] = alpha[rng.integers(0, len(alpha))]
                elif op == 1 and len(t) > 1:
                    del t[k]
                elif len(t) < 48:
                    t.insert(k, alpha[rng.integers(0, len(alpha))])
            strs.append("".join(t))
    rep = from_strings(strs)
    lens = np.diff(rep.offsets)
    assert (lens <= 32).any() and (lens > 32).any()
    off, cols, deg, _ = gpu_csr(rep, threshold, "tile")
    ro, rc, _ = oracle_csr(rep, threshold)
    assert_csr_equal(off, cols, ro, rc, f"lengths 26..44, T={threshold}")
    check_invariants(off, cols, deg, rep.n)


@pytest.mark.parametrize("threshold", [1, 2])
def test_tile_write_pass_when_hits_overflow_the_kept_pairs(threshold):
    # 3.1 million adjacent pairs among 2,500 strings: more than the count pass
    # keeps (at least 2^20 pairs, 64 per row), so the write pass runs instead
    strs = ["CASSLGQETQYF"] * 2000 + ["CASSLGQETQYW"] * 300 + ["CASSLGETQYF"] * 200 + ["CASSPGQETQYF"]
    rep = from_strings(strs)
    off, cols, deg, _ = gpu_csr(rep, threshold, "tile")
    ro, rc, _ = oracle_csr(rep, threshold)
    assert_csr_equal(off, cols, ro, rc, f"dense tile build T={threshold}")
    check_invariants(off, cols, deg, rep.n)


@pytest.mark.parametrize("method", ["deletion", "tile"])
def test_repeat_builds_are_bit_identical(method):
    # slots come from atomics in every write, yet rows are sorted: the result
    # may not depend on scheduling
    rep = generate_config1(30_000 if method == "deletion" else 6000, seed=111)
    first = None
    for k in range(4):
        opts = {"partition_target": (12, 24, 40, 0)[k]} if method == "deletion" else {}
        with tn.tcrnet_build_flat(rep.chars, rep.offsets, 1, method=method, **opts) as g:
            off, cols, deg = g.copy_csr()
        if first is None:
            first = (np.asarray(off).copy(), cols.copy(), deg.copy())
        else:
            assert np.array_equal(off, first[0]) and np.array_equal(cols, first[1]) and np.array_equal(deg, first[2])


def test_device_copy_leaves_guard_bytes_untouched():
    import torch

    rep = generate_config1(4000, seed=112)
    with tn.tcrnet_build_flat(rep.chars, rep.offsets, 1, method="deletion") as g:
        n, nnz, o64 = g.info()
        guard = 4096
        sentinel = -123456789
        off = torch.full((guard + n + 1 + guard,), sentinel, dtype=torch.int64 if o64 else torch.int32, device="cuda")
        cols = torch.full((guard + nnz + guard,), sentinel, dtype=torch.int32, device="cuda")
        deg = torch.full((guard + n + guard,), sentinel, dtype=torch.int32, device="cuda")
        st = tn.load_library().tcrnet_copy_csr(g.handle, off[guard:].data_ptr(), cols[guard:].data_ptr(),
                                               deg[guard:].data_ptr(), tn.DEVICE)
        assert st == tn.OK
        torch.cuda.synchronize()
        for t, inner in ((off, n + 1), (cols, nnz), (deg, n)):
            assert (t[:guard] == sentinel).all() and (t[guard + inner:] == sentinel).all()
        ho, hc, hd = g.copy_csr()
        assert np.array_equal(off[guard:guard + n + 1].cpu().numpy(), ho)
        assert np.array_equal(cols[guard:guard + nnz].cpu().numpy(), hc)


@pytest.mark.parametrize("method", ["deletion", "tile"])
def test_flat_offsets_checked_on_the_device(method):
    chars = np.frombuffer(b"XXCASSFCASSGCASF", dtype=np.uint8)
    cases = [
        (np.array([2, 7, 5, 16], np.int64), tn.EINVAL, 1),   # decreasing: negative length
        (np.array([2, 18, 16, 16], np.int64), tn.EINVAL, 0),  # string 0 reaches past offsets[n]
        (np.array([2, 7, 7, 16], np.int64), tn.EINVAL, 1),   # empty string
    ]
    for off, status, idx in cases:
        with pytest.raises(tn.TcrnetError) as e:
            tn.tcrnet_build_flat(chars, off, 1, method=method)
        assert e.value.status == status and e.value.index == idx, (off, e.value.status, e.value.index)
    # a base offset above zero: CASSF, CASSG, CASF
    with tn.tcrnet_build_flat(chars, np.array([2, 7, 12, 16], np.int64), 1, method=method) as g:
        off, cols, _ = g.copy_csr()
    assert list(np.asarray(off)) == [0, 2, 3, 4] and list(cols) == [1, 2, 0, 0]


@pytest.mark.parametrize("method", ["deletion", "tile"])
def test_long_rows_of_every_sort_class(method):
    """Cliques of identical strings joined to their one-substitution neighbours
    give rows of known content in each row-sort class (warp registers, 256-thread
    groups, whole block, chunked merge): row i = every node of the clique and of
    the adjacent clique except i, ascending."""
    sizes = [(300, 250), (1500, 900), (3000, 2500), (9000, 1000), (16000, 1500)]
    strs, groups = [], []
    for g, (a, b) in enumerate(sizes):
        base = "CASS" + ALPHABET[g] * 6 + "QYF"
        other = base[:5] + "W" + base[6:]  # one substitution away
        lo = len(strs)
        strs += [base] * a + [other] * b
        groups.append((lo, lo + a + b))
    rep = from_strings(strs)
    with tn.tcrnet_build_flat(rep.chars, rep.offsets, 1, method=method) as g:
        off, cols, deg = g.copy_csr()
    off = np.asarray(off, dtype=np.int64)
    check_invariants(off, cols, deg, len(strs))
    for lo, hi in groups:
        ids = np.arange(lo, hi, dtype=np.int32)
        for i in (lo, lo + 1, (lo + hi) // 2, hi - 2, hi - 1):
            row = cols[off[i]:off[i + 1]]
            assert np.array_equal(row, ids[ids != i]), (method, lo, hi, i)


def test_lmax2_deletion_method_exact():
    """l_max = 2 through candidates of shared variants with up to two deletions
    and the exact distance check: equal to the oracle and to the all-pairs
    kernels on exhaustive tiny-alphabet sets, generator strings, edge strings
    and strings across the 32-letter word boundary."""
    cases = {
        "tiny alphabet": from_strings(_all_strings("AC", 6) + _all_strings("ACD", 3)),
        "generator": generate_config1(3000, seed=62),
        "edge strings": from_strings(edge_strings()),
    }
    rng = np.random.default_rng(93)
    alpha = np.array(list("ACDEFG"))
    long_strs = []
    for _ in range(200):
        L = int(rng.integers(28, 47))
        s = list(alpha[rng.integers(0, len(alpha), L)])
        long_strs.append("".join(s))
        for _ in range(3):
            t = list(s)
            for _ in range(int(rng.integers(1, 4))):
                k = int(rng.integers(0, len(t)))
                op = int(rng.integers(0, 3))
                if op == 0:
                    t[k] = alpha[rng.integers(0, len(alpha))]
                elif op == 1 and len(t) > 1:
                    del t[k]
                elif len(t) < 48:
                    t.insert(k, alpha[rng.integers(0, len(alpha))])
            long_strs.append("".join(t))
    cases["long strings"] = from_strings(long_strs)
    for name, rep in cases.items():
        off, cols, deg, st = gpu_csr(rep, 2, "deletion")
        assert st["method"] == tn.METHOD_DELETION
        ro, rc, _ = oracle_csr(rep, 2)
        assert_csr_equal(off, cols, ro, rc, f"{name}: deletion l_max=2 vs oracle")
        check_invariants(off, cols, deg, rep.n)
        to, tc, _, _ = gpu_csr(rep, 2, "tile")
        assert_csr_equal(off, cols, to, tc, f"{name}: deletion vs tile l_max=2")


@pytest.mark.parametrize("target", [4, 24, 64, 128])
def test_lmax2_partition_sizes(target):
    """The l_max = 2 candidate pass with partitions of about `target` records:
    partitions of up to 32 records take the one-warp match path, larger ones
    are compared 32 by 32 records. The network is the same for every target."""
    rep = generate_config1(12_000, seed=66)
    off, cols, deg, st = gpu_csr(rep, 2, "deletion", partition_target=target)
    to, tc, _, _ = gpu_csr(rep, 2, "tile")
    assert_csr_equal(off, cols, to, tc, f"deletion (target {target}) vs tile, l_max=2")
    check_invariants(off, cols, deg, rep.n)


def test_lmax2_variant_shared_by_thousands():
    """More than 4,000 distinct strings share one variant (a 10-letter string
    with two letters inserted anywhere): one partition holds them all, with
    over 12 million candidate pairs among its records."""
    rng = np.random.default_rng(71)
    base = "CASSLGQETQ"
    letters = np.array(list(ALPHABET))
    seen = set()
    while len(seen) < 5000:
        t = list(base)
        for _ in range(2):
            t.insert(int(rng.integers(0, len(t) + 1)), str(letters[rng.integers(0, len(letters))]))
        seen.add("".join(t))
    rep = from_strings(sorted(seen) + generate_config1(2000, seed=72).strings())
    off, cols, deg, st = gpu_csr(rep, 2, "deletion")
    to, tc, _, _ = gpu_csr(rep, 2, "tile")
    assert_csr_equal(off, cols, to, tc, "deletion vs tile, l_max=2, one variant shared by 5,000 strings")
    check_invariants(off, cols, deg, rep.n)
    rows = sample_rows(deg, 20, seed=7, top=5)
    roff, rcols = oracle.rows(rep.chars, rep.offsets, rows, max_dist=2)
    assert_rows_equal(off, cols, rows, roff, rcols, "sampled oracle rows")


def _edited_queries(strs, rng, k):
    """k resident strings, each with 0, 1 or 2 random edits (substitution,
    deletion, insertion), plus strings with no neighbour at all."""
    letters = np.array(list(ALPHABET))
    out = []
    for i in rng.choice(len(strs), k, replace=False):
        t = list(strs[i])
        for _ in range(int(rng.integers(0, 3))):
            pos = int(rng.integers(0, len(t)))
            op = int(rng.integers(0, 3))
            if op == 0:
                t[pos] = str(letters[rng.integers(0, len(letters))])
            elif op == 1 and len(t) > 1:
                del t[pos]
            elif len(t) < 48:
                t.insert(pos, str(letters[rng.integers(0, len(letters))]))
        out.append("".join(t))
    return out + ["A", "W" * 48, "CAAAF", "CAAF", "CASSLGQF"]


def test_lmax2_index_queries_match_oracle_and_tile():
    """Queries of an l_max = 2 deletion build go through its variant records
    (method DELETION) and equal the all-pairs query and the oracle."""
    rep = generate_config1(20_000, seed=75)
    rng = np.random.default_rng(76)
    q = from_strings(_edited_queries(rep.strings(), rng, 400))
    with tn.tcrnet_build_flat(rep.chars, rep.offsets, 2) as g:
        assert g.stats()["method"] == tn.METHOD_DELETION
        with g.query_flat(q.chars, q.offsets) as r:
            qo, qc, qd = r.copy_csr()
            assert r.stats()["method"] == tn.METHOD_DELETION
        with g.query_flat(q.chars, q.offsets, method="tile") as r:
            to, tc, _ = r.copy_csr()
    assert_csr_equal(qo, qc, to, tc, "l_max=2 index queries vs all-pairs queries")
    ro, rc = oracle.neighbors(rep.chars, rep.offsets, q.chars, q.offsets, max_dist=2)
    assert_csr_equal(qo, qc, ro, rc, "l_max=2 index queries vs oracle")
    assert np.array_equal(np.asarray(qd), np.diff(np.asarray(qo, dtype=np.int64)))


def test_lmax2_index_after_insert():
    """An insert into an l_max = 2 deletion build rebuilds network and index:
    queries afterwards see the new strings."""
    rep = generate_config1(6000, seed=78)
    add = generate_config1(800, seed=79)
    rng = np.random.default_rng(80)
    full = from_strings(rep.strings() + add.strings())
    q = from_strings(_edited_queries(full.strings(), rng, 200))
    with tn.tcrnet_build_flat(rep.chars, rep.offsets, 2, method="deletion") as g:
        g.insert_flat(add.chars, add.offsets)
        fo, fc, _ = g.copy_csr()
        with g.query_flat(q.chars, q.offsets) as r:
            qo, qc, _ = r.copy_csr()
            assert r.stats()["method"] == tn.METHOD_DELETION
    oo, oc, _ = oracle.network(full.chars, full.offsets, max_dist=2)
    assert_csr_equal(fo, fc, oo, oc, "l_max=2 network after insert")
    ro, rc = oracle.neighbors(full.chars, full.offsets, q.chars, q.offsets, max_dist=2)
    assert_csr_equal(qo, qc, ro, rc, "l_max=2 index queries after insert")


def test_lmax2_index_queries_edge_strings_and_shared_variant():
    """Index queries at l_max = 2 on runs, seams, duplicates and a variant
    shared by thousands of resident strings (rows of thousands of candidates)."""
    rng = np.random.default_rng(77)
    base = "CASSLGQETQ"
    letters = np.array(list(ALPHABET))
    crowd = set()
    while len(crowd) < 3000:
        t = list(base)
        for _ in range(2):
            t.insert(int(rng.integers(0, len(t) + 1)), str(letters[rng.integers(0, len(letters))]))
        crowd.add("".join(t))
    strs = edge_strings() + sorted(crowd) + edge_strings()[:50]
    rep = from_strings(strs)
    qs = from_strings(edge_strings()[:200] + [base, base[:-1], base + "F", "CASSLGQETQYF"] + sorted(crowd)[:30])
    with tn.tcrnet_build_flat(rep.chars, rep.offsets, 2, method="deletion") as g:
        with g.query_flat(qs.chars, qs.offsets) as r:
            qo, qc, _ = r.copy_csr()
            assert r.stats()["method"] == tn.METHOD_DELETION
    ro, rc = oracle.neighbors(rep.chars, rep.offsets, qs.chars, qs.offsets, max_dist=2)
    assert_csr_equal(qo, qc, ro, rc, "l_max=2 index queries, edge strings and a crowded variant")


def test_lmax2_deletion_method_matches_tile_2e4():
    rep = generate_config1(20_000, seed=64)
    off, cols, deg, st = gpu_csr(rep, 2, "auto")
    assert st["method"] == tn.METHOD_DELETION
    to, tc, _, _ = gpu_csr(rep, 2, "tile")
    assert_csr_equal(off, cols, to, tc, "auto (deletion) vs tile, l_max=2, 2e4 strings")
    check_invariants(off, cols, deg, rep.n)
    rows = sample_rows(deg, 40, seed=5, top=10)
    roff, rcols = oracle.rows(rep.chars, rep.offsets, rows, max_dist=2)
    assert_rows_equal(off, cols, rows, roff, rcols, "sampled oracle rows")


def test_auto_takes_tile_method_above_deletion_limit():
    """The deletion method addresses at most TCRNET_DELETION_MAX_N strings; AUTO
    builds larger repertoires with the tile method instead of refusing them.
    options.deletion_max_n lowers the limit so that a small input shows it."""
    import ctypes

    for threshold, n in ((1, 3000), (2, 3000)):
        rep = generate_config1(n, seed=19)
        ro, rc, _ = oracle_csr(rep, threshold)
        with tn.tcrnet_build_flat(rep.chars, rep.offsets, threshold) as g:
            assert g.stats()["method"] == tn.METHOD_DELETION  # above the AUTO cut-over
        with tn.tcrnet_build_flat(rep.chars, rep.offsets, threshold, deletion_max_n=1000) as g:
            assert g.stats()["method"] == tn.METHOD_TILE
            off, cols, _ = g.copy_csr()
        assert_csr_equal(off, cols, ro, rc, f"AUTO above the deletion limit, T={threshold}")
        with pytest.raises(tn.TcrnetError) as e:
            tn.tcrnet_build_flat(rep.chars, rep.offsets, threshold, method="deletion", deletion_max_n=1000)
        assert e.value.status == tn.ENOTSUP
    # an insert that grows a deletion build past the limit is rebuilt by the tile method
    rep = generate_config1(1200, seed=20)
    ro, rc, _ = oracle_csr(rep, 1)
    head = rep.subset(np.arange(900))
    tail = rep.subset(np.arange(900, 1200))
    lib = tn.load_library()
    with tn.tcrnet_build_flat(head.chars, head.offsets, 1, method="deletion", deletion_max_n=1000) as g:
        opt = tn.make_options(deletion_max_n=1000)
        h = ctypes.c_void_p()
        st = lib.tcrnet_extend(g.handle, tail.chars.ctypes.data, tail.offsets.ctypes.data, tail.n, tn.HOST,
                               ctypes.byref(opt), ctypes.byref(h))
        assert st == tn.OK
        with tn.Graph(h.value) as g2:
            assert g2.stats()["method"] == tn.METHOD_TILE
            off, cols, _ = g2.copy_csr()
    assert_csr_equal(off, cols, ro, rc, "insert past the deletion limit")
