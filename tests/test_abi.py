"""The C-ABI library loads and exports every entry point include/tcrnet.h
declares; argument checks that precede any device work answer on the CPU."""

import ctypes
import re

import pytest

import paper_2112_06613_b300 as tn


def declared_functions():
    text = open(tn.HEADER_PATH).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tcrnet_[a-z0-9_]+)\s*\(", text)))


def test_header_declarations_match_binding_list():
    assert declared_functions() == sorted(tn.SYMBOLS)


def test_library_exports_every_declared_symbol():
    lib = tn.load_library()
    for name in declared_functions():
        assert hasattr(lib, name), name
        getattr(lib, name)


def test_status_strings_and_version():
    assert tn.tcrnet_strerror(tn.OK) == "ok"
    assert "amino" in tn.tcrnet_strerror(tn.EBADCHAR)
    assert "sm_103a" in tn.tcrnet_version()


def test_options_init_defaults():
    o = tn.make_options()
    assert o.method == tn.METHOD_AUTO and o.device == -1 and o.stream is None
    assert o.profile == 0 and o.force_offsets64 == 0
    assert ctypes.sizeof(tn.tcrnet_options) == 4 * 3 + 4 + 8 + 4 + 32 + 4  # padded layout of the C struct


@pytest.mark.parametrize("threshold,method,status", [(-1, "auto", tn.EINVAL), (2, "deletion", tn.ENOTSUP),
                                                     (6, "deletion", tn.ENOTSUP)])
def test_threshold_rejected_before_device_work(threshold, method, status):
    # negative l_max, and the deletion join with l_max >= 2, are refused before any device work
    with pytest.raises(tn.TcrnetError) as e:
        tn.tcrnet_build(["CASSF", "CASSG"], threshold=threshold, method=method)
    assert e.value.status == status


def test_null_output_and_negative_n_rejected():
    lib = tn.load_library()
    assert lib.tcrnet_build(None, -1, 1, None, None) == tn.EINVAL
    h = ctypes.c_void_p()
    assert lib.tcrnet_build_flat(None, None, -5, tn.HOST, 1, None, ctypes.byref(h)) == tn.EINVAL
    assert h.value is None
    assert lib.tcrnet_info(None, None, None, None) == tn.EINVAL
    lib.tcrnet_free(None)


def test_bad_method_rejected():
    with pytest.raises(tn.TcrnetError) as e:
        tn.tcrnet_build(["CASSF"], method=7)
    assert e.value.status == tn.EINVAL
