"""CPU oracle for chordless-cycle enumeration (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import this package.  It shares no code with the CUDA path; see ``cc_oracle.c``.
"""
from .oracle import (  # noqa: F401
    Result, build, bruteforce, cycle_hash, degree_labeling, enumerate_cycles,
    enumerate_parallel, niche_overlap, splitmix64_next, triplet_count, vertex_hash,
)
