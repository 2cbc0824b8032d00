"""CPU oracle for the transform in the Lin-Chung-Han basis and the RS erasure code.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``.  The product library never imports it.
"""
from .oracle import *  # noqa: F401,F403
