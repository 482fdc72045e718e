"""Python binding of tcrnet (B300 builder of the TCR-NET CDR3beta network).

Argument marshalling only: every step of the computation runs in the CUDA
library ``libtcrnet.so`` behind the C ABI of ``include/tcrnet.h``. The
functions keep the C names (``tcrnet_build``, ``tcrnet_build_flat``,
``tcrnet_query`` ...). Device buffers and streams may be given as PyTorch CUDA
tensors / streams; PyTorch is used for nothing else.

There is no CPU fallback: importing the module works without a GPU, but every
call needs the built library and a CUDA device, and fails loudly otherwise.
"""

from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtcrnet.so")
HEADER_PATH = os.path.join(os.path.dirname(_HERE), "include", "tcrnet.h")

MAX_LEN = 48

OK, EINVAL, EBADCHAR, ETOOLONG, ENOTSUP, ENOMEM, EDEVICE, ETIMEOUT, ESTATE, ECAPACITY = range(10)
STATUS_NAMES = ["OK", "EINVAL", "EBADCHAR", "ETOOLONG", "ENOTSUP", "ENOMEM", "EDEVICE", "ETIMEOUT", "ESTATE",
                "ECAPACITY"]
NOALLOC_MAX_N = 16384
DELETION_MAX_N = 1 << 25
METHOD_AUTO, METHOD_TILE, METHOD_DELETION = 0, 1, 2
METHODS = {"auto": METHOD_AUTO, "tile": METHOD_TILE, "deletion": METHOD_DELETION}
HOST, DEVICE = 0, 1


class tcrnet_options(ctypes.Structure):
    _fields_ = [
        ("method", ctypes.c_int32),
        ("device", ctypes.c_int32),
        ("force_offsets64", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
        ("profile", ctypes.c_int32),
        ("partition_cap", ctypes.c_int32),
        ("partition_target", ctypes.c_int32),
        ("fail_alloc_at", ctypes.c_int32),
        ("insert_rebuild", ctypes.c_int32),
        ("link_attempts", ctypes.c_int32),
        ("deletion_max_n", ctypes.c_int32),
        ("record_hash_bits", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 1),
    ]


class tcrnet_stats(ctypes.Structure):
    _fields_ = [
        ("method", ctypes.c_int32),
        ("threshold", ctypes.c_int32),
        ("n", ctypes.c_int64),
        ("nnz", ctypes.c_int64),
        ("candidate_pairs", ctypes.c_int64),
        ("n_unique", ctypes.c_int64),
        ("n_records", ctypes.c_int64),
        ("unique_edges", ctypes.c_int64),
        ("n_fallback", ctypes.c_int64),
        ("kernel_launches", ctypes.c_int64),
        ("closed_total", ctypes.c_int64),
        ("two_pass_join", ctypes.c_int64),
        ("ms_upload", ctypes.c_double),
        ("ms_pack", ctypes.c_double),
        ("ms_count", ctypes.c_double),
        ("ms_scan", ctypes.c_double),
        ("ms_write", ctypes.c_double),
        ("ms_sort", ctypes.c_double),
        ("ms_total", ctypes.c_double),
        ("ms_phase", ctypes.c_double * 8),
        ("merged_inserts", ctypes.c_int64),
        ("rejected_candidates", ctypes.c_int64),
    ]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "ms_phase"}
        d["ms_phase"] = list(self.ms_phase)
        return d


class TcrnetError(RuntimeError):
    def __init__(self, status: int, where: str, index: int = -1, detail: str = ""):
        self.status = status
        self.index = index
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        msg = f"{where}: {name}"
        if index >= 0:
            msg += f" (input index {index})"
        if detail:
            msg += f" [{detail}]"
        super().__init__(msg)


_lib = None
_lock = threading.Lock()

# Exported C-ABI symbols (checked by the CPU test suite against include/tcrnet.h).
SYMBOLS = [
    "tcrnet_options_init", "tcrnet_build", "tcrnet_build_flat", "tcrnet_info", "tcrnet_copy_csr",
    "tcrnet_csr_device", "tcrnet_query_flat", "tcrnet_query", "tcrnet_stats_get", "tcrnet_free",
    "tcrnet_strerror", "tcrnet_last_error_index", "tcrnet_version", "tcrnet_last_cuda_error",
    "tcrnet_degree_noalloc", "tcrnet_query_ex", "tcrnet_insert_flat", "tcrnet_insert_ex", "tcrnet_insert",
    "tcrnet_components", "tcrnet_neighbor_degree", "tcrnet_build_batched",
    "tcrnet_degree_histogram", "tcrnet_extend", "tcrnet_save", "tcrnet_load", "tcrnet_components_ex",
    "tcrnet_probe_int_issue", "tcrnet_sort_rows",
]


def load_library(path: str = LIB_PATH):
    """Load libtcrnet.so and declare its signatures. Raises if it is not built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with `python -m paper_2112_06613_b300.build`")
        lib = ctypes.CDLL(path)
        H = ctypes.c_void_p
        HP = ctypes.POINTER(ctypes.c_void_p)
        i64 = ctypes.c_int64
        i32 = ctypes.c_int32
        vp = ctypes.c_void_p
        optp = ctypes.POINTER(tcrnet_options)
        lib.tcrnet_options_init.argtypes = [optp]
        lib.tcrnet_options_init.restype = None
        lib.tcrnet_build.argtypes = [ctypes.POINTER(ctypes.c_char_p), i64, i32, optp, HP]
        lib.tcrnet_build.restype = ctypes.c_int
        lib.tcrnet_build_flat.argtypes = [vp, vp, i64, i32, i32, optp, HP]
        lib.tcrnet_build_flat.restype = ctypes.c_int
        lib.tcrnet_info.argtypes = [H, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i32)]
        lib.tcrnet_info.restype = ctypes.c_int
        lib.tcrnet_copy_csr.argtypes = [H, vp, vp, vp, i32]
        lib.tcrnet_copy_csr.restype = ctypes.c_int
        lib.tcrnet_csr_device.argtypes = [H, HP, HP, HP]
        lib.tcrnet_csr_device.restype = ctypes.c_int
        lib.tcrnet_query_flat.argtypes = [H, vp, vp, i64, i32, HP]
        lib.tcrnet_query_flat.restype = ctypes.c_int
        lib.tcrnet_save.argtypes = [H, ctypes.c_char_p]
        lib.tcrnet_save.restype = ctypes.c_int
        lib.tcrnet_load.argtypes = [ctypes.c_char_p, optp, HP]
        lib.tcrnet_load.restype = ctypes.c_int
        lib.tcrnet_extend.argtypes = [H, vp, vp, i64, i32, optp, HP]
        lib.tcrnet_extend.restype = ctypes.c_int
        lib.tcrnet_degree_histogram.argtypes = [H, vp, i64, i32, ctypes.POINTER(i64)]
        lib.tcrnet_degree_histogram.restype = ctypes.c_int
        lib.tcrnet_build_batched.argtypes = [vp, vp, i64, vp, i64, i32, i32, optp, HP]
        lib.tcrnet_build_batched.restype = ctypes.c_int
        lib.tcrnet_components.argtypes = [H, vp, vp, i32, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        lib.tcrnet_components.restype = ctypes.c_int
        lib.tcrnet_components_ex.argtypes = [H, vp, vp, i32, optp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        lib.tcrnet_components_ex.restype = ctypes.c_int
        lib.tcrnet_neighbor_degree.argtypes = [H, vp, i32]
        lib.tcrnet_neighbor_degree.restype = ctypes.c_int
        lib.tcrnet_insert_flat.argtypes = [H, vp, vp, i64, i32]
        lib.tcrnet_insert_flat.restype = ctypes.c_int
        lib.tcrnet_insert_ex.argtypes = [H, vp, vp, i64, i32, optp]
        lib.tcrnet_insert_ex.restype = ctypes.c_int
        lib.tcrnet_insert.argtypes = [H, ctypes.POINTER(ctypes.c_char_p), i64]
        lib.tcrnet_insert.restype = ctypes.c_int
        lib.tcrnet_query_ex.argtypes = [H, vp, vp, i64, i32, optp, HP]
        lib.tcrnet_query_ex.restype = ctypes.c_int
        lib.tcrnet_query.argtypes = [H, ctypes.POINTER(ctypes.c_char_p), i64, HP]
        lib.tcrnet_query.restype = ctypes.c_int
        lib.tcrnet_stats_get.argtypes = [H, ctypes.POINTER(tcrnet_stats)]
        lib.tcrnet_stats_get.restype = ctypes.c_int
        lib.tcrnet_free.argtypes = [H]
        lib.tcrnet_free.restype = None
        lib.tcrnet_strerror.argtypes = [ctypes.c_int]
        lib.tcrnet_strerror.restype = ctypes.c_char_p
        lib.tcrnet_last_error_index.argtypes = []
        lib.tcrnet_last_error_index.restype = i64
        lib.tcrnet_version.argtypes = []
        lib.tcrnet_version.restype = ctypes.c_char_p
        lib.tcrnet_last_cuda_error.argtypes = []
        lib.tcrnet_last_cuda_error.restype = ctypes.c_char_p
        lib.tcrnet_degree_noalloc.argtypes = [vp, vp, i64, i32, vp, vp, ctypes.POINTER(i64)]
        lib.tcrnet_degree_noalloc.restype = ctypes.c_int
        lib.tcrnet_probe_int_issue.argtypes = [i32, i32, vp, i64, vp, ctypes.POINTER(i64)]
        lib.tcrnet_probe_int_issue.restype = ctypes.c_int
        lib.tcrnet_sort_rows.argtypes = [vp, vp, i64, vp]
        lib.tcrnet_sort_rows.restype = ctypes.c_int
        _lib = lib
        return lib


def _check(status: int, where: str):
    if status != OK:
        lib = load_library()
        idx = int(lib.tcrnet_last_error_index())
        detail = lib.tcrnet_last_cuda_error().decode() if status in (EDEVICE, ENOMEM) else ""
        raise TcrnetError(status, where, idx, detail)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def make_options(method="auto", device=None, stream=None, profile=False, force_offsets64=False,
                 partition_cap=0, partition_target=0, fail_alloc_at=0, insert_rebuild=False,
                 link_attempts=0, deletion_max_n=0, record_hash_bits=0):
    lib = load_library()
    o = tcrnet_options()
    lib.tcrnet_options_init(ctypes.byref(o))
    o.method = METHODS[method] if isinstance(method, str) else int(method)
    if device is not None:
        o.device = int(device)
    o.stream = _stream_ptr(stream)
    o.profile = 1 if profile else 0
    o.force_offsets64 = 1 if force_offsets64 else 0
    o.partition_cap = int(partition_cap)
    o.partition_target = int(partition_target)
    o.fail_alloc_at = int(fail_alloc_at)
    # False/0: automatic; True/1: rebuild; "merge"/2: merge whenever the index allows
    o.insert_rebuild = 2 if insert_rebuild in ("merge", 2) else (1 if insert_rebuild else 0)
    o.link_attempts = int(link_attempts)
    o.deletion_max_n = int(deletion_max_n)
    o.record_hash_bits = int(record_hash_bits)
    return o


class Graph:
    """Owns one tcrnet handle: a CSR (n rows) in device memory."""

    def __init__(self, handle: int, owned: bool = True):
        self._h = ctypes.c_void_p(handle)
        self._owned = owned

    @classmethod
    def borrowed(cls, handle: int) -> "Graph":
        """A view of a handle owned elsewhere (free() leaves it alone)."""
        return cls(handle, owned=False)

    @property
    def handle(self):
        return self._h

    def release(self) -> int:
        """Give up ownership; returns the raw handle (the caller frees it with tcrnet_free)."""
        h = self._h.value if self._h is not None else None
        self._h = None
        return h

    def adopt(self, handle: int) -> int | None:
        """Take ownership of `handle`; returns the previously held raw handle, not freed."""
        old = self._h.value if (self._h is not None and self._owned) else None
        self._h = ctypes.c_void_p(handle)
        self._owned = True
        return old

    def free(self):
        if self._owned and self._h is not None and self._h.value:
            load_library().tcrnet_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    def info(self):
        n, nnz, o64 = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        _check(load_library().tcrnet_info(self._h, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(o64)),
               "tcrnet_info")
        return n.value, nnz.value, bool(o64.value)

    def copy_csr(self, out=None):
        """Host copies (numpy): offsets (int32 or int64), cols int32, degree int32.
        With `out=(offsets, cols, degree)` preallocated host arrays, fills them."""
        n, nnz, o64 = self.info()
        if out is None:
            off = np.empty(n + 1, dtype=np.int64 if o64 else np.int32)
            cols = np.empty(max(nnz, 1), dtype=np.int32)
            deg = np.empty(max(n, 1), dtype=np.int32)
        else:
            off, cols, deg = out
        _check(load_library().tcrnet_copy_csr(self._h, _ptr(off), _ptr(cols), _ptr(deg), HOST), "tcrnet_copy_csr")
        if out is None:
            return off, cols[:nnz], deg[:n]
        return out

    def copy_csr_device(self, device="cuda"):
        """Device copies as torch tensors (offsets, cols, degree)."""
        import torch

        n, nnz, o64 = self.info()
        off = torch.empty(n + 1, dtype=torch.int64 if o64 else torch.int32, device=device)
        cols = torch.empty(max(nnz, 1), dtype=torch.int32, device=device)
        deg = torch.empty(max(n, 1), dtype=torch.int32, device=device)
        _check(load_library().tcrnet_copy_csr(self._h, off.data_ptr(), cols.data_ptr(), deg.data_ptr(), DEVICE),
               "tcrnet_copy_csr")
        return off, cols[:nnz], deg[:n]

    def stats(self) -> dict:
        st = tcrnet_stats()
        _check(load_library().tcrnet_stats_get(self._h, ctypes.byref(st)), "tcrnet_stats_get")
        return st.as_dict()

    def query(self, queries):
        return tcrnet_query(self, queries)

    def components(self, keep=None, link_attempts=0, stream=None):
        """Connected components (host arrays): (labels int32 [n], n_components, largest).
        keep: optional uint8 mask of the nodes that stay (node removal).
        link_attempts: testing bound of the union-find (0 = default)."""
        n, _, _ = self.info()
        labels = np.empty(max(n, 1), dtype=np.int32)
        kp = None
        if keep is not None:
            keep = np.ascontiguousarray(keep, dtype=np.uint8)
            assert keep.shape[0] == n
            kp = keep.ctypes.data
        nc, lc = ctypes.c_int64(), ctypes.c_int64()
        opt = make_options(stream=stream, link_attempts=link_attempts)
        _check(load_library().tcrnet_components_ex(self._h, kp, labels.ctypes.data, HOST, ctypes.byref(opt),
                                                   ctypes.byref(nc), ctypes.byref(lc)), "tcrnet_components_ex")
        return labels[:n], nc.value, lc.value

    def degree_histogram(self, nbins=None):
        """Nodes per degree (host int64 array); the last bin collects larger degrees.
        nbins=None sizes the bins to the largest degree + 1."""
        lib = load_library()
        mx = ctypes.c_int64()
        if nbins is None:
            one = np.empty(1, dtype=np.int64)
            _check(lib.tcrnet_degree_histogram(self._h, one.ctypes.data, 1, HOST, ctypes.byref(mx)),
                   "tcrnet_degree_histogram")
            nbins = int(mx.value) + 1
        hist = np.empty(int(nbins), dtype=np.int64)
        _check(lib.tcrnet_degree_histogram(self._h, hist.ctypes.data, int(nbins), HOST, ctypes.byref(mx)),
               "tcrnet_degree_histogram")
        return hist

    def neighbor_degree(self):
        """Average neighbour degree per node (host float64 array)."""
        n, _, _ = self.info()
        knn = np.empty(max(n, 1), dtype=np.float64)
        _check(load_library().tcrnet_neighbor_degree(self._h, knn.ctypes.data, HOST), "tcrnet_neighbor_degree")
        return knn[:n]

    def insert(self, seqs):
        """Append host strings as new nodes (tcrnet_insert)."""
        lib = load_library()
        enc = [s.encode("ascii") if isinstance(s, str) else bytes(s) for s in seqs]
        arr = (ctypes.c_char_p * max(len(enc), 1))(*enc)
        _check(lib.tcrnet_insert(self._h, arr, len(enc)), "tcrnet_insert")

    def insert_flat(self, chars, offsets, stream=None, profile=False, rebuild=False, fail_alloc_at=0,
                    merge=False):
        """Append strings in flat layout (numpy or torch, host or device) as new nodes.
        A deletion build at l_max = 1 merges them into its network and index where
        that is faster than a rebuild; rebuild=True always rebuilds the grown
        repertoire, merge=True merges whenever the index can take the strings.
        Every way gives the same network."""
        if rebuild and merge:
            raise ValueError("rebuild and merge exclude each other")
        lib = load_library()
        cp, op, m, mem, keep = _flat_args(chars, offsets)
        opt = make_options(stream=stream, profile=profile, insert_rebuild="merge" if merge else bool(rebuild),
                           fail_alloc_at=fail_alloc_at)
        st = lib.tcrnet_insert_ex(self._h, cp, op, m, mem, ctypes.byref(opt))
        del keep
        _check(st, "tcrnet_insert_ex")

    def save(self, path: str):
        """Checkpoint this handle (network, resident strings, query index) to a file."""
        _check(load_library().tcrnet_save(self._h, os.fsencode(path)), "tcrnet_save")

    def extend_flat(self, chars, offsets, stream=None, profile=False, rebuild=False, fail_alloc_at=0,
                    merge=False) -> "Graph":
        """Copy-on-write insert: a new Graph of this one's strings plus the new ones;
        this Graph is unchanged and may keep serving queries meanwhile. rebuild and
        merge as for insert_flat."""
        if rebuild and merge:
            raise ValueError("rebuild and merge exclude each other")
        lib = load_library()
        cp, op, m, mem, keep = _flat_args(chars, offsets)
        opt = make_options(stream=stream, profile=profile, insert_rebuild="merge" if merge else bool(rebuild),
                           fail_alloc_at=fail_alloc_at)
        h = ctypes.c_void_p()
        st = lib.tcrnet_extend(self._h, cp, op, m, mem, ctypes.byref(opt), ctypes.byref(h))
        del keep
        _check(st, "tcrnet_extend")
        return Graph(h.value)

    def query_flat(self, chars, offsets, method="auto", stream=None):
        if method == "auto" and stream is None:
            return tcrnet_query_flat(self, chars, offsets)
        return tcrnet_query_ex(self, chars, offsets, method=method, stream=stream)


def _ptr(a):
    if a is None:
        return None
    if _is_torch(a):
        return a.data_ptr()
    return a.ctypes.data


def _flat_args(chars, offsets):
    """(chars_ptr, offsets_ptr, n, mem, keepalive) for numpy or torch inputs."""
    if _is_torch(chars):
        import torch

        assert chars.dtype == torch.uint8 and offsets.dtype == torch.int64
        assert chars.is_contiguous() and offsets.is_contiguous()
        assert chars.device == offsets.device
        mem = DEVICE if chars.is_cuda else HOST
        return chars.data_ptr(), offsets.data_ptr(), offsets.numel() - 1, mem, (chars, offsets)
    chars = np.ascontiguousarray(chars, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    if chars.size == 0:
        chars = np.zeros(1, dtype=np.uint8)
    return chars.ctypes.data, offsets.ctypes.data, offsets.shape[0] - 1, HOST, (chars, offsets)


def tcrnet_build(seqs, threshold: int = 1, method="auto", device=None, stream=None, profile=False,
                 force_offsets64=False) -> Graph:
    """Network of a list of strings (host memory)."""
    lib = load_library()
    enc = [s.encode("ascii") if isinstance(s, str) else bytes(s) for s in seqs]
    arr = (ctypes.c_char_p * max(len(enc), 1))(*enc)
    opt = make_options(method, device, stream, profile, force_offsets64)
    h = ctypes.c_void_p()
    _check(lib.tcrnet_build(arr, len(enc), int(threshold), ctypes.byref(opt), ctypes.byref(h)), "tcrnet_build")
    return Graph(h.value)


def tcrnet_build_flat(chars, offsets, threshold: int = 1, method="auto", device=None, stream=None,
                      profile=False, force_offsets64=False, partition_cap=0, partition_target=0,
                      deletion_max_n=0, record_hash_bits=0) -> Graph:
    """Network of strings in flat layout (numpy arrays, or torch tensors on host or device)."""
    lib = load_library()
    cp, op, n, mem, keep = _flat_args(chars, offsets)
    opt = make_options(method, device, stream, profile, force_offsets64, partition_cap, partition_target,
                       deletion_max_n=deletion_max_n, record_hash_bits=record_hash_bits)
    h = ctypes.c_void_p()
    st = lib.tcrnet_build_flat(cp, op, n, mem, int(threshold), ctypes.byref(opt), ctypes.byref(h))
    del keep
    _check(st, "tcrnet_build_flat")
    return Graph(h.value)


def tcrnet_load(path: str, device=None, stream=None) -> Graph:
    """A handle restored from a tcrnet_save checkpoint."""
    lib = load_library()
    opt = make_options("auto", device, stream)
    h = ctypes.c_void_p()
    _check(lib.tcrnet_load(os.fsencode(path), ctypes.byref(opt), ctypes.byref(h)), "tcrnet_load")
    return Graph(h.value)


def tcrnet_build_batched(chars, offsets, rep_offsets, threshold: int = 1, stream=None, profile=False,
                         partition_target=0) -> Graph:
    """Block-diagonal network of several repertoires in one pass (see include/tcrnet.h).
    rep_offsets: host int64 array of nrep + 1 string-index bounds."""
    lib = load_library()
    cp, op, n, mem, keep = _flat_args(chars, offsets)
    ro = np.ascontiguousarray(rep_offsets, dtype=np.int64)
    opt = make_options("deletion", None, stream, profile, partition_target=partition_target)
    h = ctypes.c_void_p()
    st = lib.tcrnet_build_batched(cp, op, n, ro.ctypes.data, ro.shape[0] - 1, mem, int(threshold),
                                  ctypes.byref(opt), ctypes.byref(h))
    del keep
    _check(st, "tcrnet_build_batched")
    return Graph(h.value)


def split_block_diagonal(offsets, cols, rep_offsets):
    """Per-repertoire (offsets, cols) of a batched build's CSR, ids local to the repertoire."""
    off = np.asarray(offsets, dtype=np.int64)
    out = []
    for r in range(len(rep_offsets) - 1):
        a, b = int(rep_offsets[r]), int(rep_offsets[r + 1])
        o = off[a:b + 1]
        out.append((o - o[0], cols[o[0]:o[-1]] - a))
    return out


def tcrnet_query(graph: Graph, queries) -> Graph:
    lib = load_library()
    enc = [s.encode("ascii") if isinstance(s, str) else bytes(s) for s in queries]
    arr = (ctypes.c_char_p * max(len(enc), 1))(*enc)
    h = ctypes.c_void_p()
    _check(lib.tcrnet_query(graph.handle, arr, len(enc), ctypes.byref(h)), "tcrnet_query")
    return Graph(h.value)


def tcrnet_query_flat(graph: Graph, chars, offsets) -> Graph:
    lib = load_library()
    cp, op, m, mem, keep = _flat_args(chars, offsets)
    h = ctypes.c_void_p()
    st = lib.tcrnet_query_flat(graph.handle, cp, op, m, mem, ctypes.byref(h))
    del keep
    _check(st, "tcrnet_query_flat")
    return Graph(h.value)


def tcrnet_query_ex(graph: Graph, chars, offsets, method="auto", stream=None) -> Graph:
    lib = load_library()
    cp, op, m, mem, keep = _flat_args(chars, offsets)
    opt = make_options(method, None, stream)
    h = ctypes.c_void_p()
    st = lib.tcrnet_query_ex(graph.handle, cp, op, m, mem, ctypes.byref(opt), ctypes.byref(h))
    del keep
    _check(st, "tcrnet_query_ex")
    return Graph(h.value)


def tcrnet_strerror(status: int) -> str:
    return load_library().tcrnet_strerror(int(status)).decode()


def tcrnet_version() -> str:
    return load_library().tcrnet_version().decode()


def tcrnet_degree_noalloc(chars, offsets, degree, threshold: int = 1, stream=None) -> None:
    """Node degrees into the preallocated device tensor `degree` (int32, n), for
    callers that cannot allocate device memory: torch CUDA tensors in, nothing
    allocated by the library (see include/tcrnet.h). At most NOALLOC_MAX_N
    strings. The tensors must be contiguous and on the current CUDA device, and
    `degree` must hold at least n entries: the kernels write degree[0..n), so
    these are checked here before anything is launched."""
    import torch

    if not (chars.is_cuda and offsets.is_cuda and degree.is_cuda):
        raise ValueError("tcrnet_degree_noalloc: chars, offsets and degree must be CUDA tensors")
    if not (chars.dtype == torch.uint8 and offsets.dtype == torch.int64 and degree.dtype == torch.int32):
        raise ValueError("tcrnet_degree_noalloc: dtypes must be uint8 chars, int64 offsets, int32 degree")
    if not (chars.is_contiguous() and offsets.is_contiguous() and degree.is_contiguous()):
        raise ValueError("tcrnet_degree_noalloc: tensors must be contiguous")
    n = offsets.numel() - 1
    if n < 0 or degree.numel() < n:
        raise ValueError(f"tcrnet_degree_noalloc: degree holds {degree.numel()} entries, {max(n, 0)} needed")
    dev = torch.cuda.current_device()
    if not (chars.device.index == dev and offsets.device.index == dev and degree.device.index == dev):
        raise ValueError("tcrnet_degree_noalloc: tensors must be on the current CUDA device")
    bad = ctypes.c_int64(-1)
    st = load_library().tcrnet_degree_noalloc(chars.data_ptr(), offsets.data_ptr(), n, int(threshold),
                                              degree.data_ptr(), _stream_ptr(stream), ctypes.byref(bad))
    if st != OK:
        raise TcrnetError(st, "tcrnet_degree_noalloc", int(bad.value))


PROBE_KINDS = {"lop3": 0, "shf": 1, "iadd": 2, "imad": 3, "popc": 4, "mix": 5}


def tcrnet_probe_int_issue(kind: str, iters: int, out, stream=None) -> int:
    """Launch the integer-issue microbenchmark on `stream` (a torch CUDA stream);
    `out` is a contiguous uint32-sized (int32) CUDA tensor with one entry per
    thread (a multiple of 256). Returns the integer instructions each thread
    issues; the caller times the launch with CUDA events on the same stream."""
    ops = ctypes.c_int64()
    st = load_library().tcrnet_probe_int_issue(PROBE_KINDS[kind], int(iters), out.data_ptr(), out.numel(),
                                               _stream_ptr(stream), ctypes.byref(ops))
    _check(st, "tcrnet_probe_int_issue")
    return ops.value


def tcrnet_sort_rows(offsets, cols, stream=None):
    """Sort every row segment cols[offsets[i]:offsets[i+1]] ascending in place on
    the device (the builds' per-row ordering step). offsets: int64 CUDA tensor of
    n + 1 ascending entries ending at cols.numel(); cols: int32 CUDA tensor."""
    import torch

    if offsets.dtype != torch.int64 or cols.dtype != torch.int32:
        raise TypeError("offsets must be int64 and cols int32")
    if not (offsets.is_cuda and cols.is_cuda) or offsets.device != cols.device:
        raise ValueError("offsets and cols must be CUDA tensors on one device")
    if offsets.device.index != torch.cuda.current_device():
        raise ValueError("offsets and cols must be on the current device")
    if not (offsets.is_contiguous() and cols.is_contiguous()) or offsets.dim() != 1 or cols.dim() != 1:
        raise ValueError("offsets and cols must be contiguous 1-D tensors")
    n = offsets.numel() - 1
    if n < 0:
        raise ValueError("offsets needs at least one entry")
    if n > 0:
        ends = offsets[[0, -1]].tolist()
        if ends[0] != 0 or ends[1] != cols.numel() or bool((offsets[1:] < offsets[:-1]).any()):
            raise ValueError("offsets must ascend from 0 to cols.numel()")
    _check(load_library().tcrnet_sort_rows(offsets.data_ptr(), cols.data_ptr(), n, _stream_ptr(stream)),
           "tcrnet_sort_rows")
