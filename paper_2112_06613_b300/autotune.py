"""Autotuner for the deletion join's partition schedule.

The deletion-neighbourhood path splits its records (every string and each of
its one-deletion variants) into P hash partitions of about `partition_target`
records; a warp joins a partition of at most 32 records with one match step,
larger ones with a register sort. Smaller partitions put more of them on the
fast step but spread the record scatter over more counters, so the best target
depends on the number of records (measured on a B300: 20-24 for 1e7 records,
32 for 1.3e8). The network is the same for every target; only the time
changes.

`PartitionTuner.tune` times each candidate target on the caller's own input
(CUDA events on the build stream, best of `trials`) and remembers the winner
per size class (batched or not, log2 of the record count), optionally in a JSON
file. All computation is in the CUDA library; this module only chooses an
option value and times calls.
"""

from __future__ import annotations

import json
import math
import os
import threading

import numpy as np

from . import Graph, tcrnet_build_batched, tcrnet_build_flat

DEFAULT_CANDIDATES = (16, 20, 24, 32, 40, 48)


def records_estimate(offsets) -> int:
    """Records of the deletion join: one per string plus one per character."""
    if hasattr(offsets, "cpu"):
        o = offsets
        n = int(o.numel()) - 1
        total = int(o[-1].item() - o[0].item()) if n > 0 else 0
    else:
        o = np.asarray(offsets)
        n = int(o.shape[0]) - 1
        total = int(o[-1] - o[0]) if n > 0 else 0
    return n + total


def size_class(records: int, batched: bool, device_name: str = "") -> str:
    """Cache key: GPU model, batched or not, log2 of the record count."""
    prefix = f"{device_name}|" if device_name else ""
    return f"{prefix}{'batched' if batched else 'single'}:{int(math.log2(max(records, 1)))}"


class PartitionTuner:
    def __init__(self, candidates=DEFAULT_CANDIDATES, trials: int = 2, cache_path: str | None = None):
        self.candidates = tuple(int(c) for c in candidates)
        self.trials = int(trials)
        self.cache_path = cache_path
        self.cache: dict[str, int] = {}
        self.last_timings: dict[int, float] = {}
        self._lock = threading.Lock()
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.cache = {k: int(v) for k, v in json.load(f).items()}

    def _save(self):
        if self.cache_path:
            tmp = self.cache_path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.cache, f, indent=1, sort_keys=True)
            os.replace(tmp, self.cache_path)

    def choose(self, key: str, timer) -> int:
        """Best candidate for `key`; timer(target) -> milliseconds is called only on a cache miss."""
        with self._lock:
            if key in self.cache:
                return self.cache[key]
        timings = {}
        for t in self.candidates:
            timings[t] = min(timer(t) for _ in range(self.trials))
        best = min(timings, key=timings.get)
        with self._lock:
            self.last_timings = timings
            self.cache[key] = best
            self._save()
        return best

    def tune(self, chars, offsets, rep_offsets=None, threshold: int = 1, stream=None) -> int:
        """Partition target for this input (timed on it once per size class)."""
        import torch

        batched = rep_offsets is not None
        key = size_class(records_estimate(offsets), batched, torch.cuda.get_device_name())
        s = stream if stream is not None else torch.cuda.current_stream()

        def timer(target):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            g = self._build(chars, offsets, rep_offsets, threshold, s, target)
            b.record(s)
            b.synchronize()
            g.free()
            return a.elapsed_time(b)

        with self._lock:
            if key in self.cache:
                return self.cache[key]
        timer(self.candidates[0])  # warm the library's workspace before timing
        return self.choose(key, timer)

    @staticmethod
    def _build(chars, offsets, rep_offsets, threshold, stream, target) -> Graph:
        if rep_offsets is None:
            return tcrnet_build_flat(chars, offsets, threshold, method="deletion", stream=stream,
                                     partition_target=target)
        return tcrnet_build_batched(chars, offsets, rep_offsets, threshold, stream=stream, partition_target=target)

    def build(self, chars, offsets, threshold: int = 1, rep_offsets=None, stream=None) -> Graph:
        """Tuned build (plain or batched)."""
        target = self.tune(chars, offsets, rep_offsets, threshold, stream)
        return self._build(chars, offsets, rep_offsets, threshold, stream, target)


__all__ = ["PartitionTuner", "DEFAULT_CANDIDATES", "records_estimate", "size_class"]
