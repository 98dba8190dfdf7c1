"""FP64 CPU oracle of the Levy LIBOR Monte Carlo.

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only code that may import it.  It
shares no code with the CUDA library (``paper_1006_3340_gb300``); both read
the same seeded inputs from ``paper_1006_3340_gb300.workloads``.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against something other than itself (see tests/test_oracle_*.py), except the
Philox counter words 1 and 3, which the external cuRAND comparison does not
exercise ("parity unpinned" for those two words beyond structural tests).
"""
