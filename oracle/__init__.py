"""FP64 CPU oracle for the greedy CS decoders with CG-based weighted least squares.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plainly written reference that the CUDA
path is checked against.  Only the test suite, the smoke check and the benchmark's CPU-baseline
leg may import it; the library's product path never does.  It shares no code with the CUDA
library: it has its own random-number definition, its own DCT, and closed-form least squares.

Contents (each module cites the passage it follows):
  rng       -- SplitMix64 definitions of the operator's random draws (Omega, d)
  dct       -- orthonormal DCT-II/III: O(N^2) definition and Makhoul FFT form
  operator  -- A = P_Omega C_N R (Eq. 7), R signs or permutation, optional basis Psi (DCT, 2-D DCT),
               A^T, closed-form columns
  ls        -- LS(S) by QR / Cholesky, and Algorithm 1's CG
  greedy    -- OMP (Sec. II, Algorithm 1), SP, OMPR, OMPR(l) and CoSaMP (readings stated in the module),
               with selection margins and selection policies (replay)
  replay    -- selection-by-selection comparison with a GPU recovery's trace, and pool workers
  adjoint   -- dL/dy of the fixed-support LS step

Parity status: every function is pinned by the not-gpu tests in tests/test_oracle_*.py against
library routines, closed forms, invariants of the theorems, brute force and ground truth; the
selection margins by hand-built vectors and closed forms (tests/test_oracle_margins.py); the
replay harness by traces written from oracle runs (tests/test_replay_harness.py).  The paper
does not define SP's and OMPR's stopping rules: beyond brute force at N = 16, exact recovery
and OMPR's no-improving-swap final state they are pinned only by their stated readings
(parity unpinned by the paper for those two rules).
"""
from . import rng, dct, operator, ls, greedy, adjoint, replay  # noqa: F401
from .operator import Operator  # noqa: F401
