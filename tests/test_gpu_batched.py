"""Batched build: many repertoires in one device pass.

Bar: bit-exact. The block-diagonal CSR's slice for each repertoire equals the
network of that repertoire built alone (and the oracle's); no edge joins two
repertoires, even between identical strings."""

from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2112_06613_b300 as tn
from synthgen import from_strings, generate_batched, generate_config1

from csr_util import assert_csr_equal, check_invariants

pytestmark = pytest.mark.gpu


def concat(reps):
    strs, bounds = [], [0]
    for r in reps:
        strs += r if isinstance(r, list) else r.strings()
        bounds.append(len(strs))
    return from_strings(strs), np.array(bounds, dtype=np.int64)


def batched_slices(flat, bounds, threshold=1):
    with tn.tcrnet_build_batched(flat.chars, flat.offsets, bounds, threshold) as g:
        off, cols, deg = g.copy_csr()
        st = g.stats()
    off = np.asarray(off, dtype=np.int64)
    check_invariants(off, cols, deg, flat.n)
    return tn.split_block_diagonal(off, cols, bounds), st


@pytest.mark.parametrize("threshold", [0, 1, 2])
def test_batched_equals_per_repertoire_builds(threshold):
    reps = generate_batched(24, seed=5, lo=50, hi=6000)
    flat, bounds = concat(reps)
    parts, st = batched_slices(flat, bounds, threshold)
    assert st["method"] == tn.METHODS["deletion"]
    for r, rep in enumerate(reps):
        with tn.tcrnet_build_flat(rep.chars, rep.offsets, threshold, method="deletion") as g:
            ro, rc, _ = g.copy_csr()
        assert_csr_equal(parts[r][0], parts[r][1], ro, rc, f"repertoire {r}")
        if r < 4:
            oo, oc, _ = oracle.network(rep.chars, rep.offsets, max_dist=threshold)
            assert_csr_equal(parts[r][0], parts[r][1], oo, oc, f"repertoire {r} vs oracle")


def test_batched_identical_strings_across_repertoires_stay_apart():
    base = generate_config1(3000, seed=61).strings()
    # the same repertoire three times, an empty one, a single string, a clone-heavy one
    reps = [base, [], base, ["CASSF"], base[:500] * 3 + ["CASSF", "CASSG"], base]
    flat, bounds = concat(reps)
    parts, st = batched_slices(flat, bounds)
    for r, strs in enumerate(reps):
        rep = from_strings(strs)
        oo, oc, _ = oracle.network(rep.chars, rep.offsets, max_dist=1)
        assert_csr_equal(parts[r][0], parts[r][1], oo, oc, f"repertoire {r}")
    assert parts[1][0].shape == (1,)
    assert len(parts[3][1]) == 0


def test_batched_edge_strings_and_handle_state():
    edge = ["A", "C", "AA", "W" * 48, "W" * 47, "W" * 47 + "Y", "AC", "CA", "ACA"]
    reps = [edge, edge[::-1], edge[:4]]
    flat, bounds = concat(reps)
    parts, _ = batched_slices(flat, bounds)
    for r, strs in enumerate(reps):
        rep = from_strings(strs)
        oo, oc, _ = oracle.network(rep.chars, rep.offsets, max_dist=1)
        assert_csr_equal(parts[r][0], parts[r][1], oo, oc, f"repertoire {r}")
    with tn.tcrnet_build_batched(flat.chars, flat.offsets, bounds, 1) as g:
        with pytest.raises(tn.TcrnetError) as e:
            g.query(["CASSF"])
        assert e.value.status == tn.ESTATE
        with pytest.raises(tn.TcrnetError) as e:
            g.insert(["CASSF"])
        assert e.value.status == tn.ESTATE
        # analytics work on the block-diagonal network
        labels, ncomp, largest = g.components()
        assert ncomp >= len(reps)


def test_batched_bad_character_reports_global_index():
    reps = [["CASSF", "CASSG"], ["CASSF", "CAS1F", "CASSW"]]
    flat, bounds = concat(reps)
    with pytest.raises(tn.TcrnetError) as e:
        tn.tcrnet_build_batched(flat.chars, flat.offsets, bounds, 1)
    assert e.value.status == tn.EBADCHAR and e.value.index == 3


def test_batched_many_repertoires_on_device_inputs():
    import torch

    reps = generate_batched(300, seed=9, lo=5, hi=400)
    flat, bounds = concat(reps)
    dc = torch.from_numpy(flat.chars).cuda()
    do = torch.from_numpy(flat.offsets).cuda()
    with tn.tcrnet_build_batched(dc, do, bounds, 1) as g:
        off, cols, _ = g.copy_csr()
    parts = tn.split_block_diagonal(np.asarray(off, dtype=np.int64), cols, bounds)
    for r in range(0, len(reps), 37):
        rep = reps[r]
        oo, oc, _ = oracle.network(rep.chars, rep.offsets, max_dist=1)
        assert_csr_equal(parts[r][0], parts[r][1], oo, oc, f"repertoire {r}")
    # no entry leaves its repertoire's block
    rep_of = np.repeat(np.arange(len(reps)), np.diff(bounds))
    rows = np.repeat(np.arange(flat.n), np.diff(np.asarray(off, dtype=np.int64)))
    assert np.array_equal(rep_of[rows], rep_of[np.asarray(cols, dtype=np.int64)])


def test_autotuned_builds_equal_default_builds():
    from paper_2112_06613_b300.autotune import PartitionTuner

    reps = generate_batched(12, seed=13, lo=200, hi=20_000)
    flat, bounds = concat(reps)
    tuner = PartitionTuner(candidates=(12, 24, 40), trials=1)
    with tn.tcrnet_build_batched(flat.chars, flat.offsets, bounds, 1) as g:
        ref = g.copy_csr()
    with tuner.build(flat.chars, flat.offsets, 1, rep_offsets=bounds) as g:
        got = g.copy_csr()
    assert set(tuner.last_timings) == {12, 24, 40}
    assert_csr_equal(got[0], got[1], ref[0], ref[1], "tuned batched vs default")
    one = reps[0]
    with tn.tcrnet_build_flat(one.chars, one.offsets, 1, method="deletion") as g:
        ref = g.copy_csr()
    for t in (4, 7, 128):
        with tn.tcrnet_build_flat(one.chars, one.offsets, 1, method="deletion", partition_target=t) as g:
            got = g.copy_csr()
        assert_csr_equal(got[0], got[1], ref[0], ref[1], f"partition_target {t}")
