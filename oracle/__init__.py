"""CPU oracle for the transform in the Lin-Chung-Han basis and the RS erasure code.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``.  The product library never imports it.
``oracle.fastcpu`` (not imported here) is a CPU restatement of the paper's fast
algorithms, pinned to the oracle by the tests and used only for comparison
timings on a CPU core.
"""
from .oracle import *  # noqa: F401,F403
