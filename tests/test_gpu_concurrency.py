"""Builds from several host threads at once, each on its own stream. One call
at a time holds a device's workspace lease (its arena and side streams); the
others take stream-ordered allocations and run every kernel in order on their
own stream. Bar: every network equals the oracle's, bit for bit."""

from __future__ import annotations

import threading

import numpy as np
import pytest

import oracle
import paper_2112_06613_b300 as tn
from synthgen import generate_config1

from csr_util import assert_csr_equal

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("method", ["deletion", "tile"])
def test_concurrent_builds_from_host_threads(method):
    import torch

    rep = generate_config1(20_000, seed=31)
    ro, rc, _ = oracle.network(rep.chars, rep.offsets, max_dist=1)
    chars = torch.from_numpy(rep.chars).cuda()
    offs = torch.from_numpy(rep.offsets).cuda()
    results, errors = [], []
    lock = threading.Lock()

    def work():
        try:
            s = torch.cuda.Stream()
            for _ in range(3):
                with tn.tcrnet_build_flat(chars, offs, 1, method=method, stream=s) as g:
                    off, cols, _ = g.copy_csr()
                with lock:
                    results.append((np.asarray(off, dtype=np.int64), cols))
        except Exception as exc:  # reported below, on the test's thread
            with lock:
                errors.append(repr(exc))

    threads = [threading.Thread(target=work) for _ in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    assert len(results) == 12
    for off, cols in results:
        assert_csr_equal(off, cols, ro, rc, f"{method} build from one of four host threads")
