"""CPU FP64 oracle for the cascade of Beylkin, "Fast convolution algorithm for
state space models" (arXiv 2411.17729).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` call it.  It shares no code with the CUDA library; its only
dependency inside the repository is the seeded input generator package
``workloads``.
"""
from .cascade import *  # noqa: F401,F403
