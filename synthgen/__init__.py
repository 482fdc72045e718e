"""Seeded synthetic CDR3beta repertoires shared by the tests, the bench and the oracle.

This module only draws strings. It holds none of the network-construction
arithmetic (no distances, no packing, no adjacency), so that the CUDA path and
the CPU oracle can both consume its output without sharing any of the method.
"""

from .cdr3 import (  # noqa: F401
    ALPHABET,
    Repertoire,
    generate,
    generate_config1,
    generate_config2,
    generate_config3,
    generate_batched,
    to_strings,
    from_strings,
)
