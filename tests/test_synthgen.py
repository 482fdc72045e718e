"""The synthetic repertoire generator: seeded, in-alphabet, lengths in range."""

import numpy as np

from synthgen import ALPHABET, generate_config1, generate_config3, generate_batched


def test_seeded_and_reproducible():
    a = generate_config1(2000, seed=4)
    b = generate_config1(2000, seed=4)
    c = generate_config1(2000, seed=5)
    assert (a.chars == b.chars).all() and (a.offsets == b.offsets).all()
    assert a.strings() != c.strings()


def test_shape_of_config1():
    r = generate_config1(20000, seed=0)
    L = r.lengths()
    assert L.min() >= 10 and L.max() <= 20
    mode = np.bincount(L).argmax()
    assert 12 <= mode <= 15
    assert set(bytes(r.chars).decode()) <= set(ALPHABET)
    # the leading C survives unless the point substitution hits position 0
    assert sum(s[0] == "C" for s in r.strings()[:1000]) > 900
    # repeats exist (shared templates), as in real repertoires
    assert len(set(r.strings())) < r.n


def test_shape_of_config3():
    r = generate_config3(20000, seed=0)
    L = r.lengths()
    assert L.min() >= 8 and L.max() <= 24


def test_batched_sizes():
    reps = generate_batched(count=6, seed=0, lo=1e3, hi=5e3)
    assert len(reps) == 6
    assert all(1000 <= r.n <= 5000 for r in reps)
