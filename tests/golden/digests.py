"""Row digests of the oracle's network, and the parser of `parity_digests.txt`.

A stored digest stands for an oracle neighbour list that is too long to keep
in the repository: the digest of a row is the 8-byte BLAKE2b of its ascending
neighbour ids as little-endian int32, and the digest of a block of rows is the
BLAKE2b of the block's degrees followed by its entries. Two lists with equal
digests are equal (up to a 2^-64 chance per row), so comparing digests is an
exact comparison of the complete lists (Methods "TCR network": row i lists
every j with lev(s_i, s_j) <= l_max). This module holds no distance or network
arithmetic; it only hashes integer arrays and reads the text file.
"""

from __future__ import annotations

import hashlib
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DIGEST_FILE = os.path.join(HERE, "parity_digests.txt")


def row_digest(cols) -> str:
    """8-byte BLAKE2b (hex) of one ascending neighbour list."""
    b = np.ascontiguousarray(cols, dtype="<i4").tobytes()
    return hashlib.blake2b(b, digest_size=8).hexdigest()


def block_digest(off, cols, r0: int, r1: int) -> str:
    """BLAKE2b (hex) of rows r0..r1-1 of a CSR: their degrees, then their entries."""
    off = np.asarray(off, dtype=np.int64)
    deg = np.diff(off[r0:r1 + 1]).astype("<i4")
    h = hashlib.blake2b(digest_size=8)
    h.update(np.ascontiguousarray(deg).tobytes())
    h.update(np.ascontiguousarray(cols[off[r0]:off[r1]], dtype="<i4").tobytes())
    return h.hexdigest()


def load(path: str = DIGEST_FILE) -> dict:
    """Sections of the digest file: {name: {"meta": {...}, "rows": [(a, b, digest), ...]}}.

    A section starts with `[name] key=value ...`; its lines are three fields
    (`block r0 digest` lines of a full network hold the block's first row; `row
    degree digest` lines of a sample hold a row id and its degree).
    """
    out: dict = {}
    cur = None
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                name, _, rest = line[1:].partition("]")
                meta = dict(kv.split("=", 1) for kv in rest.split())
                cur = out.setdefault(name, {"meta": meta, "rows": []})
                continue
            a, b, d = line.split()
            cur["rows"].append((int(a), int(b), d))
    return out
