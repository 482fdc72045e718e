"""tcrnet_degree_noalloc: node degrees for callers that cannot allocate.

Code that runs while a CUDA graph is being captured, or inside a program whose
device memory is fully reserved by another allocator, cannot call cudaMalloc.
The library offers those callers one entry point that uses a fixed device
array instead of allocations. These tests call it through the C ABI and check
that its degrees equal the degree array of the ordinary build (integers: equal
bit for bit), on several calls in a row, so that leftovers of one call cannot
leak into the next. This file is collected last on purpose.
"""

import numpy as np
import pytest

import paper_2112_06613_b300 as tn
from synthgen import from_strings, generate_config1

pytestmark = pytest.mark.gpu


def _build_degree(rep, threshold):
    with tn.tcrnet_build_flat(rep.chars, rep.offsets, threshold, method="deletion") as g:
        _, _, deg = g.copy_csr()
    return deg


def test_noalloc_degrees_equal_build_degrees_on_calls_in_a_row():
    import torch

    stream = torch.cuda.current_stream()
    cases = [(12_000, 21, 1), (5_000, 22, 1), (5_000, 22, 0), (tn.NOALLOC_MAX_N, 23, 1)]
    for n, seed, threshold in cases:
        rep = generate_config1(n, seed=seed)
        chars = torch.from_numpy(rep.chars).cuda()
        offs = torch.from_numpy(rep.offsets).cuda()
        deg = torch.full((n,), -7, dtype=torch.int32, device="cuda")  # must be overwritten
        tn.tcrnet_degree_noalloc(chars, offs, deg, threshold, stream=stream)
        got = deg.cpu().numpy()
        want = _build_degree(rep, threshold)
        assert np.array_equal(got, want), f"n={n} seed={seed} threshold={threshold}"


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
    # the next call still works and is exact
    rep = from_strings(["CASSF", "CASSG", "CASSGF", "CASF"])
    chars = torch.from_numpy(rep.chars).cuda()
    offs = torch.from_numpy(rep.offsets).cuda()
    deg = torch.zeros(4, dtype=torch.int32, device="cuda")
    tn.tcrnet_degree_noalloc(chars, offs, deg, 1)
    assert list(deg.cpu().numpy()) == list(_build_degree(rep, 1))
