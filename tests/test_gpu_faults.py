"""Host-side fault injection: every device allocation of a call in turn is made
to fail (options.fail_alloc_at). Each failing call must return TCRNET_ENOMEM,
release what it held and leave the library usable: the next normal call gives
the exact network, a handle keeps its previous network after a failed insert."""

from __future__ import annotations

import ctypes

import numpy as np
import pytest

import paper_2112_06613_b300 as tn
from synthgen import from_strings, generate_config1

from csr_util import assert_csr_equal

pytestmark = pytest.mark.gpu


def build(rep, method, fail_at=0, threshold=1):
    lib = tn.load_library()
    opt = tn.make_options(method, fail_alloc_at=fail_at)
    h = ctypes.c_void_p()
    st = lib.tcrnet_build_flat(rep.chars.ctypes.data, rep.offsets.ctypes.data, rep.n, tn.HOST, threshold,
                               ctypes.byref(opt), ctypes.byref(h))
    return st, (tn.Graph(h.value) if st == tn.OK else None)


@pytest.mark.parametrize("method,n,threshold", [("deletion", 3000, 1), ("tile", 800, 1), ("tile", 600, 2),
                                                ("deletion", 3000, 2)])
def test_every_build_allocation_failure_is_clean(method, n, threshold):
    rep = generate_config1(n, seed=91)
    st, g = build(rep, method, threshold=threshold)
    assert st == tn.OK
    ref = g.copy_csr()
    g.free()
    failures = 0
    for k in range(1, 200):
        st, g = build(rep, method, fail_at=k, threshold=threshold)
        if st == tn.OK:  # k is past the call's last allocation
            got = g.copy_csr()
            g.free()
            assert_csr_equal(got[0], got[1], ref[0], ref[1], f"build with fail_alloc_at={k}")
            break
        assert st == tn.ENOMEM, (k, st)
        assert g is None
        failures += 1
        st, g = build(rep, method, threshold=threshold)  # the library is still usable
        assert st == tn.OK
        got = g.copy_csr()
        g.free()
        assert_csr_equal(got[0], got[1], ref[0], ref[1], f"normal build after failure {k}")
    assert failures >= 5


@pytest.mark.parametrize("threshold", [1, 2])
def test_query_and_insert_allocation_failures_keep_the_handle(threshold):
    base = generate_config1(3000, seed=92)
    add = generate_config1(400, seed=93)
    q = from_strings(add.strings()[:50])
    lib = tn.load_library()
    with tn.tcrnet_build_flat(base.chars, base.offsets, threshold, method="deletion") as g:
        before = g.copy_csr()
        with g.query_flat(q.chars, q.offsets) as r:
            qref = r.copy_csr()
        for k in range(1, 60):
            opt = tn.make_options("auto", fail_alloc_at=k)
            h = ctypes.c_void_p()
            st = lib.tcrnet_query_ex(g.handle, q.chars.ctypes.data, q.offsets.ctypes.data, q.n, tn.HOST,
                                     ctypes.byref(opt), ctypes.byref(h))
            if st == tn.OK:
                r = tn.Graph(h.value)
                got = r.copy_csr()
                r.free()
                assert_csr_equal(got[0], got[1], qref[0], qref[1], f"query fail_alloc_at={k}")
                break
            assert st == tn.ENOMEM and h.value is None
        for k in range(1, 400):
            opt = tn.make_options(fail_alloc_at=k)
            st = lib.tcrnet_insert_ex(g.handle, add.chars.ctypes.data, add.offsets.ctypes.data, add.n, tn.HOST,
                                      ctypes.byref(opt))
            if st == tn.OK:
                break
            assert st == tn.ENOMEM
            after = g.copy_csr()  # the handle keeps its previous network
            assert_csr_equal(after[0], after[1], before[0], before[1], f"insert fail_alloc_at={k}")
        assert g.info()[0] == base.n + add.n
