"""FP64 CPU oracle for HHL state-vector simulation -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct reference implementation of what the CUDA library computes:
``core`` (C, compiled with gcc) applies each gate of an *unfused* gate list by the textbook
rule and computes the readout sums with compensated FP64 summation; ``hhl`` builds the HHL
gate list from (A, b, m, t, C) with numpy's Hermitian eigensolver and reads the solution out,
following the paper's Sec. III-A procedure step by step.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  It shares no code with ``paper_2402_08136_gb300`` and neither imports the other;
both take their inputs from ``synth``.

Pins (tests that tie the oracle to something other than itself) are in
``tests/test_oracle_pins.py``.  Every oracle function is pinned; none is marked unpinned.
"""
from . import core, hhl  # noqa: F401
