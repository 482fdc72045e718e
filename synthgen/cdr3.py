"""Synthetic CDR3beta generator (stand-in for the SONIA / empirical repertoires).

The paper builds its networks from SONIA-generated and empirical naive CD8
CDR3beta sequences (Introduction; Methods "IGoR, OLGA, SONIA"). Neither the
trained generation models nor the data sets are available, so every workload
here is drawn from a seeded V-insertion-J template model with the same
structure: strings start with 'C', carry one of 48 V-like prefixes, a random
N-insertion and one of 13 J-like suffixes ending in 'F', and a point
substitution with probability 0.3. Letters come from the 20 standard amino
acids (Methods "Combination of amino acids") with a Zipf(1) background over a
seeded permutation of the alphabet.

Output format: ``chars`` (uint8, ASCII letters, all strings concatenated) and
``offsets`` (int64, n+1 entries, string i is chars[offsets[i]:offsets[i+1]]).
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# The 20 standard amino acids in the order the paper lists them (Methods,
# "Combination of amino acids").
ALPHABET = "ARNDCQEGHILKMFPSTWYV"
_ALPHA_BYTES = np.frombuffer(ALPHABET.encode("ascii"), dtype=np.uint8)
_C = ord("C")
_F = ord("F")


@dataclass
class Repertoire:
    chars: np.ndarray  # uint8 [total]
    offsets: np.ndarray  # int64 [n+1]

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0] - 1)

    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)

    def strings(self) -> list[str]:
        return to_strings(self.chars, self.offsets)

    def subset(self, idx) -> "Repertoire":
        idx = np.asarray(idx, dtype=np.int64)
        strs = self.strings()
        return from_strings([strs[i] for i in idx])


def to_strings(chars: np.ndarray, offsets: np.ndarray) -> list[str]:
    raw = bytes(np.asarray(chars, dtype=np.uint8))
    off = np.asarray(offsets, dtype=np.int64)
    return [raw[off[i]:off[i + 1]].decode("ascii") for i in range(off.shape[0] - 1)]


def from_strings(strs) -> Repertoire:
    enc = [s.encode("ascii") for s in strs]
    lens = np.fromiter((len(e) for e in enc), dtype=np.int64, count=len(enc))
    offsets = np.zeros(len(enc) + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    chars = np.frombuffer(b"".join(enc), dtype=np.uint8).copy()
    return Repertoire(chars, offsets)


def _background(rng: np.random.Generator) -> np.ndarray:
    """Zipf(1) letter probabilities over a seeded permutation of the alphabet."""
    perm = rng.permutation(20)
    p = np.empty(20, dtype=np.float64)
    p[perm] = 1.0 / np.arange(1, 21, dtype=np.float64)
    return p / p.sum()


def _templates(rng, probs, count, lo, hi, suffix=None):
    """`count` templates of lo..hi background letters (+ optional suffix byte)."""
    width = hi + (1 if suffix is not None else 0)
    out = np.zeros((count, width), dtype=np.uint8)
    lens = rng.integers(lo, hi + 1, size=count)
    for t in range(count):
        letters = _ALPHA_BYTES[rng.choice(20, size=lens[t], p=probs)]
        out[t, : lens[t]] = letters
        if suffix is not None:
            out[t, lens[t]] = suffix
    if suffix is not None:
        lens = lens + 1
    return out, lens.astype(np.int64)


def generate(
    n: int,
    seed: int = 0,
    ins_max: int = 6,
    len_lo: int = 10,
    len_hi: int = 20,
    n_v: int = 48,
    n_j: int = 13,
    p_sub: float = 0.3,
    template_seed: int | None = None,
    n_v_use: int | None = None,
    n_j_use: int | None = None,
) -> Repertoire:
    """Draw `n` CDR3-like strings.

    string = 'C' + V (3-5 aa) + U{0..ins_max} background aa + J (3-5 aa + 'F');
    with probability p_sub one uniformly chosen position is replaced by a
    background draw (which may equal the old letter); strings whose length falls
    outside [len_lo, len_hi] are redrawn.

    `template_seed` (default: `seed`) fixes the template set; `n_v_use` /
    `n_j_use` restrict a repertoire to a seeded subset of the templates (the
    batched workload's per-repertoire template subsets).
    """
    trng = np.random.default_rng(seed if template_seed is None else template_seed)
    probs = _background(trng)
    vt, vl = _templates(trng, probs, n_v, 3, 5)
    jt, jl = _templates(trng, probs, n_j, 3, 5, suffix=_F)
    rng = np.random.default_rng([seed, 0x5EED])
    v_pool = np.arange(n_v)
    j_pool = np.arange(n_j)
    if n_v_use is not None:
        v_pool = rng.choice(n_v, size=n_v_use, replace=False)
    if n_j_use is not None:
        j_pool = rng.choice(n_j, size=n_j_use, replace=False)

    width = 1 + vt.shape[1] + ins_max + jt.shape[1]
    rows = np.zeros((0, width), dtype=np.uint8)
    lens = np.zeros(0, dtype=np.int64)
    need = n
    while need > 0:
        m = max(16, int(need * 1.3))
        vi = v_pool[rng.integers(0, v_pool.shape[0], size=m)]
        ji = j_pool[rng.integers(0, j_pool.shape[0], size=m)]
        li = rng.integers(0, ins_max + 1, size=m)
        ins = _ALPHA_BYTES[rng.choice(20, size=(m, max(ins_max, 1)), p=probs)]
        lv = vl[vi]
        lj = jl[ji]
        L = 1 + lv + li + lj
        col = np.arange(width)[None, :]
        lvc = lv[:, None]
        lic = li[:, None]
        Lc = L[:, None]
        M = np.zeros((m, width), dtype=np.uint8)
        M[:, 0] = _C
        in_v = (col >= 1) & (col < 1 + lvc)
        vcol = np.clip(col - 1, 0, vt.shape[1] - 1)
        M = np.where(in_v, vt[vi[:, None], vcol], M)
        in_i = (col >= 1 + lvc) & (col < 1 + lvc + lic)
        icol = np.clip(col - 1 - lvc, 0, ins.shape[1] - 1)
        M = np.where(in_i, ins[np.arange(m)[:, None], icol], M)
        in_j = (col >= 1 + lvc + lic) & (col < Lc)
        jcol = np.clip(col - 1 - lvc - lic, 0, jt.shape[1] - 1)
        M = np.where(in_j, jt[ji[:, None], jcol], M)
        # one point substitution with probability p_sub
        sub = rng.random(m) < p_sub
        pos = (rng.random(m) * L).astype(np.int64)
        letter = _ALPHA_BYTES[rng.choice(20, size=m, p=probs)]
        r = np.nonzero(sub)[0]
        M[r, pos[r]] = letter[r]
        keep = (L >= len_lo) & (L <= len_hi)
        M = M[keep]
        L = L[keep]
        take = min(need, M.shape[0])
        rows = np.concatenate([rows, M[:take]])
        lens = np.concatenate([lens, L[:take]])
        need -= take

    offsets = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    mask = np.arange(width)[None, :] < lens[:, None]
    chars = rows[mask]
    return Repertoire(np.ascontiguousarray(chars, dtype=np.uint8), offsets)


def generate_config1(n: int = 10_000, seed: int = 0) -> Repertoire:
    """Single repertoire, insertion 0-6 aa, lengths 10-20 (N = 1e4 and 8e5)."""
    return generate(n, seed=seed, ins_max=6, len_lo=10, len_hi=20)


def generate_config2(n: int = 800_000, seed: int = 0) -> Repertoire:
    """The paper's largest size, same generator as config 1."""
    return generate(n, seed=seed, ins_max=6, len_lo=10, len_hi=20)


def generate_config3(n: int = 8_000_000, seed: int = 0) -> Repertoire:
    """Ten-times N, insertion 0-9 aa, lengths 8-24 (realised 8-21)."""
    return generate(n, seed=seed, ins_max=9, len_lo=8, len_hi=24)


def generate_batched(count: int = 256, seed: int = 0, lo: float = 1e3, hi: float = 2e5):
    """`count` repertoires, sizes log-uniform in [lo, hi], per-repertoire template subsets."""
    rng = np.random.default_rng([seed, 0xBA7C])
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), size=count)).astype(np.int64)
    reps = []
    for k in range(count):
        reps.append(
            generate(int(sizes[k]), seed=seed * 100003 + k + 1, template_seed=seed,
                     n_v_use=24, n_j_use=7)
        )
    return reps
