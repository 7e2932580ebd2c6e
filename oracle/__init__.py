"""CPU FP64 oracle for batched RKCK / RKC integration.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline and reference legs may import this package.  It
shares no code with the CUDA library (``paper_1611_02274_gb300``); the two
meet only through the seeded generators in
``paper_1611_02274_gb300.workloads``, which hold none of the method's
arithmetic.
"""
from .oracle import *  # noqa: F401,F403
