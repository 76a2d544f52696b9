"""Plain FP64 CPU oracle for BSGD-TV (Gao & Blumensath, arXiv 1812.01307).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline legs of ``bench.py`` may import this package.  The GPU
library never calls it, and it shares no code with the GPU library: the two
meet only in the seeded input generator ``paper_1812_01307_gb300.synth``,
which makes problem instances and holds none of the method's arithmetic.

Every function follows the paper's steps in its order and notation, in
float64, without blocking, fusion or reordering beyond what the passage
states.  Pins (tests that tie each function to something other than itself)
live in ``tests/test_oracle_*.py``.
"""
from .bsgdtv_oracle import *  # noqa: F401,F403
