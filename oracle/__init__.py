"""FP64 CPU oracle for the local ETKF control law (arXiv:1310.5954).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of what the control law computes, written from the paper: the
state-space model and Eq. 1 (Sect. 2.1), the ensemble transform Kalman filter
(Sect. 2.2), the local ETKF by domain decomposition (Sect. 2.3) and the
classical Kalman filter with a Riccati-solved gain (Sect. 2.1) as the
comparison system.  Only the test suite, the smoke check of the build entry
point and the CPU-baseline leg of the benchmark may import it; the CUDA path
never does, and this package imports nothing from the CUDA path.  It shares
only the seeded input generators (package `synth`) with it.

Pinning: every function here is pinned by a CPU test against something other
than itself (the paper's printed counts, closed forms, algebraic identities, a
textbook library routine, or brute force).  No function is left unpinned.
"""


