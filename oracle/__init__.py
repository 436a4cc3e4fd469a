"""FP64 CPU oracle of the rational-program method (KLARAPTOR, arXiv 1911.02373).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
statement of what the library computes.  It is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``; the
library itself never imports, links or calls it, and the oracle shares no code
with the CUDA path (only the seeded input generators in ``workloads`` serve
both).

Modules, each citing the paper passage it follows:

* ``configs``   -- the configuration set F of thread-block shapes (Section IV,
  step 4 and its footnote; Section V).
* ``rational``  -- monomial bases and the linearised least-squares fit of a
  rational function p/q by SVD (Section V-E; Section IV, step 2).
* ``occupancy`` -- the occupancy rational program of Fig. 1 and Eq. 1
  (Example 1).
* ``mwpcwp``    -- the MWP-CWP execution-time model cited by Example 2.
* ``program``   -- the whole rational program: fitted metrics -> occupancy ->
  MWP-CWP -> constrained argmin (Section IV, steps 4 and 5).
* ``mlp``       -- the learned proposer's network, loss, gradients and AdamW
  (this project's addition; the paper has no learned component).

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against
closed forms, brute force, hand-worked cases or library routines, except
the fidelity of the MWP-CWP formula to the paper's own generated code, which the
paper does not print (parity unpinned; see ``mwpcwp``).
"""
from . import configs, rational, occupancy, mwpcwp, program, mlp  # noqa: F401
