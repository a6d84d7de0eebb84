"""CPU oracle of the FP64 GEMM C <- alpha*A*B + beta*C (Section 4.2).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import anything here.  The oracle
shares no code with the CUDA library and never calls it; the two meet only in
the seeded input generators of the separate ``synth`` package.

Modules:
  cgemm  - plain C triple-loop DGEMM (the definition), a row-sampled form, an
           OpenMP form with identical bits, and a double-double reference.
  exact  - exact rational DGEMM, the FP64 error bound, exact residuals.
  ozaki  - step-by-step CPU model of the split-precision path (e1..e4).
"""
