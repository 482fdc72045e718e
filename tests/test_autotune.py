"""Autotuner host logic (no GPU): size classes, choice, cache file."""

import json

import numpy as np

from paper_2112_06613_b300.autotune import PartitionTuner, records_estimate, size_class


def test_records_estimate_counts_strings_and_characters():
    offsets = np.array([0, 5, 9, 20], dtype=np.int64)
    assert records_estimate(offsets) == 3 + 20
    assert records_estimate(np.array([0], dtype=np.int64)) == 0


def test_size_class_separates_batched_and_scale():
    assert size_class(1 << 20, False) != size_class(1 << 20, True)
    assert size_class(1 << 20, False) == size_class((1 << 21) - 1, False)
    assert size_class(1 << 20, False) != size_class(1 << 21, False)


def test_choice_is_fastest_and_cached(tmp_path):
    path = tmp_path / "tune.json"
    calls = []

    def timer(t):
        calls.append(t)
        return {16: 3.0, 24: 1.0, 32: 2.0}[t]

    tuner = PartitionTuner(candidates=(16, 24, 32), trials=2, cache_path=str(path))
    assert tuner.choose("single:23", timer) == 24
    assert len(calls) == 6 and tuner.last_timings == {16: 3.0, 24: 1.0, 32: 2.0}
    assert tuner.choose("single:23", timer) == 24 and len(calls) == 6  # cache hit
    assert json.loads(path.read_text()) == {"single:23": 24}
    again = PartitionTuner(candidates=(16, 24, 32), cache_path=str(path))
    assert again.choose("single:23", lambda t: 1 / 0) == 24  # loaded from the file


def test_size_class_keys_the_gpu_model():
    assert size_class(1 << 20, False, "GPU A") != size_class(1 << 20, False, "GPU B")
    assert size_class(1 << 20, False, "GPU A").startswith("GPU A|")
