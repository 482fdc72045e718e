"""tcrnet_degree_noalloc: node degrees for callers that cannot allocate.

Some programs cannot call cudaMalloc once they run: one that handed all of its
device memory to another allocator at start-up (a caching pool that reserves
the free memory), or a service that forbids device allocation after start-up
because an allocation can synchronise the device and break its latency bound.
The library offers those callers one entry point that works in a fixed device
array instead of allocating. These tests call it through the C ABI and check
its degrees, bit for bit (integers), against the ordinary build's degree array
and against the CPU oracle's network, on several calls in a row, so that
leftovers of one call in the shared array cannot leak into the next. This file
is collected last on purpose.
"""

import numpy as np
import pytest

import oracle
import paper_2112_06613_b300 as tn
from synthgen import ALPHABET, from_strings, generate_config1

pytestmark = pytest.mark.gpu


def _build_degree(rep, threshold):
    with tn.tcrnet_build_flat(rep.chars, rep.offsets, threshold, method="deletion") as g:
        _, _, deg = g.copy_csr()
    return deg


def _oracle_degree(rep, threshold):
    _, _, deg = oracle.network(rep.chars, rep.offsets, max_dist=threshold)
    return deg


def _noalloc(rep, threshold, stream):
    import torch

    chars = torch.from_numpy(rep.chars).cuda()
    offs = torch.from_numpy(rep.offsets).cuda()
    deg = torch.full((rep.n,), -7, dtype=torch.int32, device="cuda")  # must be overwritten
    tn.tcrnet_degree_noalloc(chars, offs, deg, threshold, stream=stream)
    return deg.cpu().numpy()


def seam_strings():
    """Strings of lengths 11-13, 23-25 and 46-48 (the 12- and 24-letter word
    seams of the packed form) sharing prefixes and suffixes, with single edits
    on both sides of each seam, so that the comparison against the longer
    string shifted down one position carries letters across words."""
    rng = np.random.default_rng(31)
    out = []
    for seam in (12, 24, 48):
        base = "".join(rng.choice(list(ALPHABET), size=seam))
        for L in (seam - 1, seam, seam + 1):
            if L > 48:
                continue
            s = (base + base)[:L]
            out.append(s)
            for p in sorted({0, max(L - 2, 0), L - 1, min(11, L - 1), min(12, L - 1), min(23, L - 1),
                             min(24, L - 1)}):
                out.append(s[:p] + ("W" if s[p] != "W" else "Y") + s[p + 1:])  # substitution
                out.append(s[:p] + s[p + 1:])  # deletion
                if L < 48:
                    out.append(s[:p] + "Y" + s[p:])  # insertion
    return out


def test_noalloc_degrees_equal_build_and_oracle_on_calls_in_a_row():
    import torch

    stream = torch.cuda.current_stream()
    cases = [(12_000, 21, 1), (5_000, 22, 1), (5_000, 22, 0), (tn.NOALLOC_MAX_N, 23, 1)]
    for n, seed, threshold in cases:
        rep = generate_config1(n, seed=seed)
        got = _noalloc(rep, threshold, stream)
        assert np.array_equal(got, _build_degree(rep, threshold)), f"n={n} seed={seed} T={threshold} vs build"
        assert np.array_equal(got, _oracle_degree(rep, threshold)), f"n={n} seed={seed} T={threshold} vs oracle"


def test_noalloc_word_seams_match_oracle_twice():
    import torch

    stream = torch.cuda.current_stream()
    rep = from_strings(seam_strings())
    want = _oracle_degree(rep, 1)
    assert want.sum() > 0
    for _ in range(2):  # two calls in a row on the shared array
        got = _noalloc(rep, 1, stream)
        assert np.array_equal(got, want)
        assert np.array_equal(got, _build_degree(rep, 1))


def test_noalloc_rejects_oversized_and_bad_input():
    import torch

    n = tn.NOALLOC_MAX_N + 1
    chars = torch.full((n,), ord("A"), dtype=torch.uint8, device="cuda")
    offs = torch.arange(n + 1, dtype=torch.int64, device="cuda")
    deg = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(tn.TcrnetError) as e:
        tn.tcrnet_degree_noalloc(chars, offs, deg, 1)
    assert e.value.status == tn.ECAPACITY
    rep = from_strings(["CASSF", "CASXF", "CASSG"])
    chars = torch.from_numpy(rep.chars).cuda()
    offs = torch.from_numpy(rep.offsets).cuda()
    deg = torch.zeros(3, dtype=torch.int32, device="cuda")
    with pytest.raises(tn.TcrnetError) as e:
        tn.tcrnet_degree_noalloc(chars, offs, deg, 1)
    assert e.value.status == tn.EBADCHAR and e.value.index == 1
    # a degree tensor shorter than n is refused before anything runs
    with pytest.raises(ValueError):
        tn.tcrnet_degree_noalloc(chars, offs, torch.zeros(2, dtype=torch.int32, device="cuda"), 1)
    # the next call still works and is exact
    rep = from_strings(["CASSF", "CASSG", "CASSGF", "CASF"])
    got = _noalloc(rep, 1, torch.cuda.current_stream())
    assert list(got) == list(_build_degree(rep, 1)) == list(_oracle_degree(rep, 1))
