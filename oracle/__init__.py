"""FP64 CPU oracle for exact higher-order U-statistics (arXiv 2508.12627).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference leg may import, call, link or execute anything in this
package.  It shares no code with the CUDA library and neither imports the other;
the only module both sides use is the seeded input module ``synth``.

Two independent evaluators:
  * ``brute``: enumerates index tuples (C, OpenMP) -- the definitions of the
    U-statistic, the V-set / restricted V-statistic and the U-set / restricted
    U-statistic, written out.
  * ``ustat_oracle``: the paper's method (Algorithm 4) in float64 numpy: partitions,
    Moebius coefficients, induced notation, and the Einsum by one-index-at-a-time
    elimination.

Parity status: the per-workload values of U and V_pi are pinned through the
closed forms, identities and brute force listed in tests/test_oracle_pins.py;
nothing in this package is "parity unpinned".
"""
from . import ustat_oracle  # noqa: F401
