"""The extended bonus of Section 3.2 (oracle; test-only).

With X = A^{-1} B for an n x k right-hand side B, s~ the common denominator
of the entries of X (the lcm of their denominators, Section 2.2) and
N = s~ X the integer matrix of numerators, Lemma 3.5 and the subsection of
Section 3.2 on taking out the unwanted factors give the factor

    pi~_k = s~^k / gcd(det(R N), s~^k)

of pi_k, the product of the k largest invariant factors of A, for a k x n
matrix R. Every quantity is computed here from its definition with exact
rational arithmetic: the solve by exact.solve_rational, the k x k
determinant by exact.bareiss_det.
"""
from __future__ import annotations

import math
from fractions import Fraction

from . import exact


def solutions(A, B):
    """X = A^{-1} B column by column (B given as a list of k vectors)."""
    return [exact.solve_rational(A, list(b)) for b in B]


def extended_bonus(A, B, R):
    """(pi~_k, s~) for the right-hand sides B (k vectors of length n) and the
    k x n matrix R (Section 3.2)."""
    X = solutions(A, B)
    k = len(X)
    s = 1
    for col in X:
        s = s * exact.lcm_denominators(col) // math.gcd(s, exact.lcm_denominators(col))
    N = [[int(Fraction(v) * s) for v in col] for col in X]      # N[l][j] = s x_lj
    RN = [[sum(int(R[r][j]) * N[l][j] for j in range(len(N[l]))) for l in range(k)]
          for r in range(k)]
    d = exact.bareiss_det(RN)
    sk = s ** k
    return sk // math.gcd(d, sk), s
