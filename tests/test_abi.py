"""The C-ABI library loads and exports every entry point include/tcrnet.h
declares; argument checks that precede any device work answer on the CPU."""

import ctypes
import re

import numpy as np
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


@pytest.mark.parametrize("threshold,method,status", [(-1, "auto", tn.EINVAL), (3, "deletion", tn.ENOTSUP),
                                                     (6, "deletion", tn.ENOTSUP)])
def test_threshold_rejected_before_device_work(threshold, method, status):
    # negative l_max, and the deletion method with l_max >= 3, are refused before any device work
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


@pytest.mark.parametrize("rep_offsets,threshold,status", [
    ([0, 1], 1, tn.EINVAL),          # does not end at n
    ([1, 2], 1, tn.EINVAL),          # does not start at 0
    ([0, 2, 1, 2], 1, tn.EINVAL),    # decreasing
    ([0, 2], 3, tn.ENOTSUP),         # batched builds use the deletion method: l_max <= 2
    ([0], 1, tn.EINVAL),             # no repertoire
])
def test_batched_bounds_rejected_before_device_work(rep_offsets, threshold, status):
    chars = np.frombuffer(b"CASSFCASSG", dtype=np.uint8)
    offsets = np.array([0, 5, 10], dtype=np.int64)
    with pytest.raises(tn.TcrnetError) as e:
        tn.tcrnet_build_batched(chars, offsets, np.array(rep_offsets, dtype=np.int64), threshold=threshold)
    assert e.value.status == status


def test_batched_repertoire_limit_and_tile_method_rejected():
    lib = tn.load_library()
    chars = np.frombuffer(b"CASSF", dtype=np.uint8)
    offsets = np.array([0, 5], dtype=np.int64)
    too_many = np.zeros(65538, dtype=np.int64)
    too_many[-1] = 1
    h = ctypes.c_void_p()
    assert lib.tcrnet_build_batched(chars.ctypes.data, offsets.ctypes.data, 1, too_many.ctypes.data, 65537,
                                    tn.HOST, 1, None, ctypes.byref(h)) == tn.EINVAL
    ro = np.array([0, 1], dtype=np.int64)
    opt = tn.make_options("tile")
    assert lib.tcrnet_build_batched(chars.ctypes.data, offsets.ctypes.data, 1, ro.ctypes.data, 1,
                                    tn.HOST, 1, ctypes.byref(opt), ctypes.byref(h)) == tn.ENOTSUP
    assert lib.tcrnet_build_batched(chars.ctypes.data, offsets.ctypes.data, 1, None, 1,
                                    tn.HOST, 1, None, ctypes.byref(h)) == tn.EINVAL
    assert h.value is None


@pytest.mark.parametrize("target", [1, 3, 129, -2])
def test_partition_target_out_of_range_rejected(target):
    lib = tn.load_library()
    chars = np.frombuffer(b"CASSF", dtype=np.uint8)
    offsets = np.array([0, 5], dtype=np.int64)
    opt = tn.make_options("deletion", partition_target=target)
    h = ctypes.c_void_p()
    assert lib.tcrnet_build_flat(chars.ctypes.data, offsets.ctypes.data, 1, tn.HOST, 1, ctypes.byref(opt),
                                 ctypes.byref(h)) == tn.EINVAL
    assert h.value is None


def test_load_rejects_bad_files_before_device_work(tmp_path):
    lib = tn.load_library()
    h = ctypes.c_void_p()
    bad = tmp_path / "bad.tcr"
    bad.write_bytes(b"not a checkpoint" * 20)
    assert lib.tcrnet_load(str(bad).encode(), None, ctypes.byref(h)) == tn.EINVAL
    short = tmp_path / "short.tcr"
    short.write_bytes(b"TCRNETCK")
    assert lib.tcrnet_load(str(short).encode(), None, ctypes.byref(h)) == tn.EINVAL
    assert lib.tcrnet_load(str(tmp_path / "missing.tcr").encode(), None, ctypes.byref(h)) == tn.EINVAL
    assert lib.tcrnet_load(None, None, ctypes.byref(h)) == tn.EINVAL
    assert h.value is None
    assert lib.tcrnet_save(None, str(tmp_path / "x.tcr").encode()) == tn.EINVAL


class _FakeCudaTensor:
    """Stands in for a CUDA tensor so that the wrapper's argument checks can be
    exercised without a device: nothing may reach the library."""

    def __init__(self, dtype, numel):
        self.dtype = dtype
        self._numel = numel
        self.is_cuda = True

    def numel(self):
        return self._numel

    def is_contiguous(self):
        return True

    def data_ptr(self):
        raise AssertionError("the library must not be called")


def test_noalloc_short_degree_rejected_before_any_launch():
    import torch

    chars = _FakeCudaTensor(torch.uint8, 50)
    offs = _FakeCudaTensor(torch.int64, 11)  # n = 10
    with pytest.raises(ValueError, match="10 needed"):
        tn.tcrnet_degree_noalloc(chars, offs, _FakeCudaTensor(torch.int32, 9), 1)
    with pytest.raises(ValueError, match="dtypes"):
        tn.tcrnet_degree_noalloc(chars, offs, _FakeCudaTensor(torch.int64, 10), 1)


def test_new_option_knobs_validated():
    lib = tn.load_library()
    chars = np.frombuffer(b"CASSF", dtype=np.uint8)
    offsets = np.array([0, 5], dtype=np.int64)
    h = ctypes.c_void_p()
    for kw in ({"link_attempts": -1}, {"deletion_max_n": -3}):
        opt = tn.make_options(**kw)
        assert lib.tcrnet_build_flat(chars.ctypes.data, offsets.ctypes.data, 1, tn.HOST, 1, ctypes.byref(opt),
                                     ctypes.byref(h)) == tn.EINVAL
    # an explicit deletion build above its (lowered) limit is refused before device work
    opt = tn.make_options("deletion", deletion_max_n=1)
    two = np.array([0, 2, 5], dtype=np.int64)
    assert lib.tcrnet_build_flat(chars.ctypes.data, two.ctypes.data, 2, tn.HOST, 1, ctypes.byref(opt),
                                 ctypes.byref(h)) == tn.ENOTSUP
    assert h.value is None
    nc, lc = ctypes.c_int64(5), ctypes.c_int64(5)
    assert lib.tcrnet_components_ex(None, None, None, tn.HOST, None, ctypes.byref(nc), ctypes.byref(lc)) == tn.EINVAL
    assert nc.value == 0 and lc.value == 0


def test_sort_rows_arguments_checked_before_device_work():
    """tcrnet_sort_rows: a negative row count or missing arrays are rejected, and
    zero rows return at once, all before any CUDA call."""
    lib = tn.load_library()
    assert lib.tcrnet_sort_rows(None, None, -1, None) == tn.EINVAL
    assert lib.tcrnet_sort_rows(None, None, 3, None) == tn.EINVAL
    assert lib.tcrnet_sort_rows(None, None, 0, None) == tn.OK
