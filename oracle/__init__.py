"""CPU oracle for the integer-determinant path (test infrastructure only).

This package is the plain, slow, obviously correct reference that the CUDA
path is compared against. Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import it; the product library never does.

Contents (each function cites the passage of Dumas & Urbanska, "An
introspective algorithm for the integer determinant", that it follows):

  exact     -- fraction-free Bareiss determinant over Python integers, exact
               rational solve, lcm of denominators (Sections 1, 2.2),
               Hadamard bound (Lemma 2.1).
  modular   -- plain Gaussian elimination over Z/p in C (det mod p, LU with
               first-nonzero pivoting, rank, inverse) (Section 2.1, Alg. 2.1).
  cra       -- symmetric-range Chinese remaindering and the early-terminated
               CRA loop of Alg. 2.1 with the stopping rules of Lemma 2.1.
  dixon     -- Dixon p-adic lifting digits (Section 2.2) written as the
               textbook iteration over Python integers.
  params    -- parameter formulas: Lemma 2.1(iv) k, Alg. 4.1's S.

Nothing here shares code with the CUDA path.
"""
from . import exact, modular, cra, dixon, params  # noqa: F401
