"""FP64 CPU oracle of the Levy LIBOR Monte Carlo.

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only code that may import it.  It
shares no code with the CUDA library (``paper_1006_3340_gb300``); both read
the same seeded inputs from ``paper_1006_3340_gb300.workloads``.

Parity status: every function here is pinned by a test against something
other than itself (see tests/test_oracle_*.py).  The Philox generator is
pinned bit for bit against cuRAND's Philox4_32_10 on all four counter words:
words 0-2 by the host generator (``-m "not gpu"``), word 3 by cuRAND's device
API (tests/test_gpu_philox.py, which needs a GPU).
"""
