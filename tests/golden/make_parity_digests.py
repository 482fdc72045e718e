"""Write tests/golden/parity_digests.txt from the CPU oracle alone.

The GPU parity tests compare the library's networks with the oracle at sizes
where running the oracle live in the test would take many minutes:

  full_1e5   every row of the N = 100,000 network (config-1 generator, seed 0,
             l_max = 1): 10^10 Wagner-Fischer evaluations;
  rows_8e5   9,900 seeded uniform rows of the N = 800,000 network (config-2
             generator, seed 0, l_max = 1), the size the bench times;
  rows_8e6   1,000 seeded uniform rows of the N = 8,000,000 network (config-3
             generator, seed 0, l_max = 1).

The tests add the highest-degree rows of the build under test and a live
oracle run over part of each sample, so the stored values are checked against
the oracle on the GPU host too. Every expected value here comes from
`oracle.network` / `oracle.rows` (Methods "Levenshtein distance", "TCR
network"); nothing reads the CUDA library. Run from the repository root:

    python tests/golden/make_parity_digests.py [--only NAME]

It takes about 15 minutes on 8 cores.
"""

from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import oracle  # noqa: E402
from synthgen import generate_config1, generate_config2, generate_config3  # noqa: E402

from digests import DIGEST_FILE, block_digest, row_digest  # noqa: E402

BLOCK = 1000
SAMPLE_SEED = 20211213  # arXiv 2112.06613


def sample_ids(n: int, count: int, seed: int) -> np.ndarray:
    """Seeded uniform sample of row ids, ascending (independent of any build)."""
    rng = np.random.default_rng([seed, n])
    return np.sort(rng.choice(n, size=count, replace=False)).astype(np.int64)


def full_section(name, gen, n, seed):
    rep = gen(n, seed=seed)
    t = time.time()
    off, cols, _ = oracle.network(rep.chars, rep.offsets, max_dist=1)
    dt = time.time() - t
    lines = [f"[{name}] generator={gen.__name__} n={n} seed={seed} l_max=1 block={BLOCK} "
             f"nnz={int(off[-1])} oracle_s={dt:.0f}"]
    for r0 in range(0, n, BLOCK):
        lines.append(f"{r0} {min(r0 + BLOCK, n)} {block_digest(off, cols, r0, min(r0 + BLOCK, n))}")
    return lines


def rows_section(name, gen, n, seed, count):
    rep = gen(n, seed=seed)
    ids = sample_ids(n, count, SAMPLE_SEED)
    t = time.time()
    roff, rcols = oracle.rows(rep.chars, rep.offsets, ids, max_dist=1)
    dt = time.time() - t
    lines = [f"[{name}] generator={gen.__name__} n={n} seed={seed} l_max=1 count={count} "
             f"sample_seed={SAMPLE_SEED} entries={int(roff[-1])} oracle_s={dt:.0f}"]
    for k, i in enumerate(ids):
        lines.append(f"{int(i)} {int(roff[k + 1] - roff[k])} {row_digest(rcols[roff[k]:roff[k + 1]])}")
    return lines


SECTIONS = {
    "full_1e5": lambda: full_section("full_1e5", generate_config1, 100_000, 0),
    "rows_8e5": lambda: rows_section("rows_8e5", generate_config2, 800_000, 0, 9_900),
    "rows_8e6": lambda: rows_section("rows_8e6", generate_config3, 8_000_000, 0, 1_000),
}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", default=None, help="recompute one section, keep the others")
    ap.add_argument("--out", default=DIGEST_FILE)
    args = ap.parse_args()
    keep = {}
    if args.only and os.path.exists(args.out):
        cur = None
        with open(args.out) as f:
            for line in f:
                if line.startswith("["):
                    cur = line[1:].split("]")[0]
                    keep.setdefault(cur, [])
                if cur:
                    keep[cur].append(line.rstrip("\n"))
    out = [
        "# Oracle digests for the GPU parity tests (written by make_parity_digests.py;",
        "# every value comes from the CPU oracle). Row lines: row degree digest;",
        "# block lines: first_row end_row digest (BLAKE2b-64, see digests.py).",
    ]
    for name, fn in SECTIONS.items():
        if args.only and name != args.only:
            out += keep.get(name, [])
            continue
        t = time.time()
        out += fn()
        print(f"{name}: {time.time() - t:.0f} s", flush=True)
    with open(args.out, "w") as f:
        f.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()
