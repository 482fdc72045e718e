"""Serving loop over a resident TCR network (host-side scheduler).

A resident build handle answers neighbour queries and absorbs inserts while
requests keep arriving:

- continuous batching: when a worker slot frees up it takes every queued query
  request at the head of the queue (up to `max_batch_strings` strings) and runs
  them as one device call (`tcrnet_query_ex`); the result rows are split back
  per request;
- slots: `slots` worker threads, each with its own CUDA streams (queries on a
  high-priority stream, inserts on a low-priority one), so admitted requests
  overlap on the device (the C library releases the GIL);
- inserts are copy-on-write (`tcrnet_extend`): the grown network (merged
  from the current one for small inserts, else rebuilt) goes into a new handle
  while queries keep running on the current one; the new handle then replaces it (the caller's Graph adopts it) and the old one is
  freed after its last running query. Inserts apply one at a time in arrival
  order; queries that start before an insert's swap see the previous
  repertoire, later ones the grown one; each request records the repertoire
  version it ran on;
- admission by memory: a request starts only when its estimated device memory
  fits in the free HBM reported by the driver minus a reserve (otherwise it
  waits until running requests release theirs);
- answers are copied into per-slot pinned host buffers allocated once, then
  into each request's own arrays (a copy to pageable memory of a long answer
  goes through the driver's small staging buffers); long answers are copied
  out by a few host threads in parallel.

All computation happens in the CUDA library; this module only schedules calls.
"""

from __future__ import annotations

import collections
import concurrent.futures as cf
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import Graph, TcrnetError, load_library


@dataclass
class Request:
    kind: str  # "query" or "insert"
    chars: np.ndarray
    offsets: np.ndarray
    t_arrival: float = 0.0
    t_start: float = 0.0
    t_done: float = 0.0
    version: int = -1  # inserts applied before this request ran
    ticket: int = -1  # arrival order among inserts
    batch_id: int = -1  # device call that served it
    # where a query's time went (seconds): the device call (tcrnet_query_ex with
    # its stream sync), the copy of the batch's answer to the host, the split
    # into per-request arrays; batch_entries = neighbour entries of the whole
    # device call this request shared
    s_call: float = 0.0
    s_copy: float = 0.0
    s_split: float = 0.0
    batch_entries: int = 0
    offsets_out: np.ndarray | None = None
    cols_out: np.ndarray | None = None
    error: BaseException | None = None
    done: threading.Event = field(default_factory=threading.Event)

    @property
    def n_strings(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def latency_s(self) -> float:
        return self.t_done - self.t_arrival

    @property
    def answer_entries(self) -> int:
        return 0 if self.cols_out is None else int(self.cols_out.shape[0])


class ServingEngine:
    def __init__(self, graph: Graph, slots: int = 4, max_batch_strings: int = 200_000,
                 hbm_reserve_bytes: int = 4 << 30, device: int = 0, result_buffer_bytes: int = 64 << 20,
                 copy_threads: int = 4):
        import torch

        self.graph = graph
        self.slots = slots
        self.max_batch_strings = max_batch_strings
        self.reserve = hbm_reserve_bytes
        self.device = device
        self._torch = torch
        # per slot: a high-priority stream for queries, a low-priority one for
        # inserts, so query blocks are scheduled first while a rebuild runs
        lo, hi = torch.cuda.Stream.priority_range()
        self._streams = [torch.cuda.Stream(device=device, priority=hi) for _ in range(slots)]
        self._insert_streams = [torch.cuda.Stream(device=device, priority=lo) for _ in range(slots)]
        self._queue: collections.deque[Request] = collections.deque()
        self._cv = threading.Condition()
        self._cur = graph.handle.value  # raw handle of the current version
        self._refs: collections.Counter = collections.Counter()  # raw handle -> running calls
        self._retired: set = set()  # replaced handles waiting for their last query
        self._tickets = 0  # inserts taken
        self._turn = 0  # next insert to apply
        self._inflight_bytes = 0
        self._inflight = 0
        self._stop = False
        self._version = 0
        self._batches = 0
        # per slot: pinned host buffers for query answers, allocated once (pinned
        # allocations are slow and stall other work); larger answers use pageable
        # arrays of their own
        self._stage = [(torch.empty(max_batch_strings + 1, dtype=torch.int64, pin_memory=True),
                        torch.empty(max(result_buffer_bytes // 4, 1), dtype=torch.int32, pin_memory=True))
                       for _ in range(slots)]
        self._workers = [threading.Thread(target=self._run, args=(k,), daemon=True) for k in range(slots)]
        # host copies of long answers are split over a few threads (numpy
        # releases the GIL for them): one thread writing a fresh multi-MiB
        # array, page faults included, was most of such a request's latency
        self._copy_pool = cf.ThreadPoolExecutor(max_workers=copy_threads)
        self.completed: list[Request] = []

    # ---- lifecycle -----------------------------------------------------
    def start(self):
        for w in self._workers:
            w.start()
        return self

    def shutdown(self, wait: bool = True):
        with self._cv:
            self._stop = True
            self._cv.notify_all()
        if wait:
            for w in self._workers:
                w.join()
            self._copy_pool.shutdown(wait=True)

    def __enter__(self):
        return self.start()

    def __exit__(self, *exc):
        self.shutdown()

    # ---- requests ------------------------------------------------------
    def submit(self, req: Request) -> Request:
        req.t_arrival = time.perf_counter()
        with self._cv:
            self._queue.append(req)
            self._cv.notify_all()
        return req

    def query(self, chars, offsets) -> Request:
        return self.submit(Request("query", np.ascontiguousarray(chars, np.uint8),
                                   np.ascontiguousarray(offsets, np.int64)))

    def insert(self, chars, offsets) -> Request:
        return self.submit(Request("insert", np.ascontiguousarray(chars, np.uint8),
                                   np.ascontiguousarray(offsets, np.int64)))

    # ---- admission -----------------------------------------------------
    def _estimate_bytes(self, kind: str, strings: int) -> int:
        n, nnz, _ = self.graph.info()
        mean_deg = nnz / max(n, 1)
        if kind == "query":
            # packed strings, records, counts, offsets, and the result lists (x4 margin)
            return int(strings * (96 + 4 * 4 * (mean_deg + 1)))
        # an insert builds the grown network into a new handle: at most about
        # 600 B of scratch per string (a rebuild; a merge needs less) plus the
        # new CSR
        return int((n + strings) * 600 + 4 * (nnz * (n + strings) / max(n, 1)))

    def _admissible(self, need: int) -> bool:
        if self._inflight == 0:
            return True  # never starve: one request may always run
        free, _ = self._torch.cuda.mem_get_info(self.device)
        return need + self.reserve <= free

    def _take(self):
        with self._cv:
            while True:
                if self._stop and not self._queue:
                    return None, 0
                if self._queue:
                    head = self._queue[0]
                    if head.kind == "insert":
                        batch = [head]
                        strings = head.n_strings
                    else:
                        batch, strings = [], 0
                        for r in self._queue:
                            if r.kind != "query":
                                break
                            if batch and strings + r.n_strings > self.max_batch_strings:
                                break
                            batch.append(r)
                            strings += r.n_strings
                    need = self._estimate_bytes(head.kind, strings)
                    if self._admissible(need):
                        for _ in batch:
                            self._queue.popleft()
                        if head.kind == "insert":
                            head.ticket = self._tickets
                            self._tickets += 1
                        self._inflight += 1
                        self._inflight_bytes += need
                        return batch, need
                self._cv.wait(timeout=0.05)

    def _release(self, need: int):
        with self._cv:
            self._inflight -= 1
            self._inflight_bytes -= need
            self._cv.notify_all()

    # ---- workers -------------------------------------------------------
    def _run(self, slot: int):
        stream = self._streams[slot]
        insert_stream = self._insert_streams[slot]
        while True:
            batch, need = self._take()
            if batch is None:
                return
            t0 = time.perf_counter()
            for r in batch:
                r.t_start = t0
            try:
                if batch[0].kind == "insert":
                    self._do_insert(batch[0], insert_stream)
                else:
                    self._do_queries(batch, stream, slot)
            except BaseException as e:  # reported per request
                for r in batch:
                    r.error = e
            finally:
                t1 = time.perf_counter()
                for r in batch:
                    r.t_done = t1
                    r.done.set()
                with self._cv:
                    self.completed.extend(batch)
                self._release(need)

    def _acquire(self):
        with self._cv:
            h = self._cur
            self._refs[h] += 1
            return h, self._version

    def _drop(self, h):
        with self._cv:
            self._refs[h] -= 1
            if h in self._retired and self._refs[h] == 0:
                self._retired.discard(h)
                load_library().tcrnet_free(h)

    def _do_insert(self, req: Request, stream):
        with self._cv:
            while self._turn != req.ticket:  # inserts apply in arrival order
                self._cv.wait()
        try:
            h, version = self._acquire()
            try:
                new = Graph.borrowed(h).extend_flat(req.chars, req.offsets, stream=stream)
            finally:
                self._drop(h)
            with self._cv:
                req.version = version
                req.batch_id = self._batches
                self._batches += 1
                old = self.graph.adopt(new.release())
                self._cur = self.graph.handle.value
                self._version += 1
                if old is not None:
                    if self._refs[old] == 0:
                        load_library().tcrnet_free(old)
                    else:
                        self._retired.add(old)
        finally:
            with self._cv:
                self._turn += 1
                self._cv.notify_all()

    def _copy_out(self, src: np.ndarray) -> np.ndarray:
        return _parallel_copy(self._copy_pool, src)

    def _do_queries(self, batch: list[Request], stream, slot: int = 0):
        if len(batch) == 1:
            chars, offsets = batch[0].chars, batch[0].offsets
        else:
            chars = np.concatenate([r.chars[r.offsets[0]:r.offsets[-1]] for r in batch])
            lens = np.concatenate([np.diff(r.offsets) for r in batch])
            offsets = np.zeros(lens.shape[0] + 1, dtype=np.int64)
            np.cumsum(lens, out=offsets[1:])
        h, version = self._acquire()
        try:
            with self._cv:
                bid = self._batches
                self._batches += 1
            t_call = time.perf_counter()
            res = Graph.borrowed(h).query_flat(chars, offsets, method="auto", stream=stream)
            t_copy = time.perf_counter()
            try:
                # into this slot's pinned buffers (a copy to pageable memory goes
                # through the driver's small staging buffers, slowly for long
                # answers), then out into each request's own arrays
                n, nnz, o64 = res.info()
                off_t, cols_t = self._stage[slot]
                if n + 1 <= off_t.numel() and nnz <= cols_t.numel():
                    off_v = off_t.numpy()[:n + 1] if o64 else off_t.numpy().view(np.int32)[:n + 1]
                    cols = cols_t.numpy()[:nnz]
                else:  # larger than the slot's buffers: pageable arrays of its own
                    off_v = np.empty(n + 1, dtype=np.int64 if o64 else np.int32)
                    cols = np.empty(max(nnz, 1), dtype=np.int32)[:nnz]
                st = load_library().tcrnet_copy_csr(res.handle, off_v.ctypes.data, cols.ctypes.data, None, 0)
                if st != 0:
                    raise TcrnetError(st, "tcrnet_copy_csr")
            finally:
                res.free()
        finally:
            self._drop(h)
        t_split = time.perf_counter()
        off = off_v.astype(np.int64)
        row = 0
        for r in batch:
            k = r.n_strings
            o = off[row:row + k + 1]
            r.offsets_out = o - o[0]
            r.cols_out = self._copy_out(cols[o[0]:o[-1]])
            r.version = version
            r.batch_id = bid
            row += k
        t_end = time.perf_counter()
        for r in batch:
            r.s_call = t_copy - t_call
            r.s_copy = t_split - t_copy
            r.s_split = t_end - t_split
            r.batch_entries = int(nnz)


_PARALLEL_COPY_MIN = 1 << 19  # entries (2 MiB of int32)


def _parallel_copy(pool, src: np.ndarray) -> np.ndarray:
    """A fresh copy of `src`, written in equal chunks by the pool's threads
    when it is long."""
    n = src.shape[0]
    if n < _PARALLEL_COPY_MIN:
        return src.copy()
    dst = np.empty_like(src)
    k = pool._max_workers
    step = (n + k - 1) // k
    futs = [pool.submit(np.copyto, dst[i * step:(i + 1) * step], src[i * step:(i + 1) * step]) for i in range(k)]
    for f in futs:
        f.result()
    return dst


def latency_summary(reqs, kind: str):
    lat = [1e3 * r.latency_s for r in reqs if r.kind == kind and r.error is None]
    if not lat:
        return None
    return {"count": len(lat), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(np.mean(lat))}


def latency_by_answer_size(reqs, edges=(0, 1_000, 10_000, 100_000, 1_000_000, 1 << 62)):
    """Query latency binned by the entries of the device call's answer (the
    batch a request shared), with the mean split of each bin's latency into
    queueing, the device call, the host copy of the answer and the split."""
    qs = [r for r in reqs if r.kind == "query" and r.error is None]
    out = []
    for lo, hi in zip(edges[:-1], edges[1:]):
        b = [r for r in qs if lo <= r.batch_entries < hi]
        if not b:
            continue
        lat = np.array([1e3 * r.latency_s for r in b])
        out.append({
            "answer_entries": f"[{lo}, {hi})" if hi < (1 << 62) else f">= {lo}",
            "count": len(b),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()),
            "mean_queue_ms": float(np.mean([1e3 * (r.t_start - r.t_arrival) for r in b])),
            "mean_call_ms": float(np.mean([1e3 * r.s_call for r in b])),
            "mean_copy_ms": float(np.mean([1e3 * r.s_copy for r in b])),
            "mean_split_ms": float(np.mean([1e3 * r.s_split for r in b])),
            "mean_batch_entries": float(np.mean([r.batch_entries for r in b])),
        })
    return out
