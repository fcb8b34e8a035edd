"""Exact integer and rational reference computations (oracle; test-only).

* bareiss_det -- the determinant by fraction-free Bareiss elimination over
  arbitrary-precision integers. The paper's problem statement is "compute
  det(A) for an integer matrix A" (Abstract, Section 1); this is the plain
  definition of that value.
* solve_rational -- x = A^{-1} b over Q (Section 2.2, "rational solution of
  the linear systems Ax = b"), by Bareiss forward elimination on [A | b]
  followed by back substitution in exact fractions.
* lcm_denominators -- the LargestInvariantFactor output s~_n: the lcm of the
  denominators of the entries of x (Section 2.2).
* hadamard_* -- Hadamard's bound |det A| <= (sqrt(n) ||A||)^n (Lemma 2.1) and
  the row-norm form prod_i ||row_i||_2 it is derived from.
"""
from __future__ import annotations

import math
from fractions import Fraction


def _as_int_rows(A) -> list[list[int]]:
    return [[int(v) for v in row] for row in A]


def bareiss_det(A) -> int:
    """det(A) by Bareiss' fraction-free elimination.

    For k = 0 .. n-2: take the first row i >= k with a nonzero entry in column
    k as pivot row (swap, flip the sign; none -> det = 0); then for all
    i, j > k set a_ij <- (a_ij * a_kk - a_ik * a_kj) / prev, an exact
    division, and prev <- a_kk. det = sign * a_{n-1,n-1}.
    """
    M = _as_int_rows(A)
    n = len(M)
    if n == 0:
        return 1
    sign = 1
    prev = 1
    for k in range(n - 1):
        if M[k][k] == 0:
            for i in range(k + 1, n):
                if M[i][k] != 0:
                    M[k], M[i] = M[i], M[k]
                    sign = -sign
                    break
            else:
                return 0
        akk = M[k][k]
        rowk = M[k]
        for i in range(k + 1, n):
            rowi = M[i]
            aik = rowi[k]
            for j in range(k + 1, n):
                rowi[j] = (rowi[j] * akk - aik * rowk[j]) // prev
            rowi[k] = 0
        prev = akk
    return sign * M[n - 1][n - 1]


class SingularMatrix(ValueError):
    pass


def solve_rational(A, b) -> list[Fraction]:
    """Exact x with A x = b over Q.

    Bareiss forward elimination is applied to the augmented matrix [A | b]
    (every Bareiss step replaces row i by a nonzero multiple of itself plus a
    multiple of the pivot row, so the solution set is unchanged); the
    resulting upper-triangular system is solved by back substitution with
    exact fractions.
    """
    M = _as_int_rows(A)
    n = len(M)
    for i in range(n):
        M[i].append(int(b[i]))
    prev = 1
    for k in range(n):
        if M[k][k] == 0:
            for i in range(k + 1, n):
                if M[i][k] != 0:
                    M[k], M[i] = M[i], M[k]
                    break
            else:
                raise SingularMatrix("matrix is singular")
        akk = M[k][k]
        rowk = M[k]
        for i in range(k + 1, n):
            rowi = M[i]
            aik = rowi[k]
            for j in range(k + 1, n + 1):
                rowi[j] = (rowi[j] * akk - aik * rowk[j]) // prev
            rowi[k] = 0
        prev = akk
    x = [Fraction(0)] * n
    for i in range(n - 1, -1, -1):
        acc = Fraction(M[i][n])
        row = M[i]
        for j in range(i + 1, n):
            if row[j]:
                acc -= row[j] * x[j]
        x[i] = acc / row[i]
    return x


def check_solution(A, b, x) -> bool:
    """A x == b exactly (independent check of a rational solution)."""
    A = _as_int_rows(A)
    for i, row in enumerate(A):
        s = sum((a * xj for a, xj in zip(row, x)), Fraction(0))
        if s != int(b[i]):
            return False
    return True


def lcm_denominators(x) -> int:
    """lcm of the denominators of the (reduced) entries of x (Section 2.2)."""
    s = 1
    for v in x:
        d = Fraction(v).denominator
        s = s * d // math.gcd(s, d)
    return s


def largest_invariant_factor(A, b) -> int:
    """s~_n for right-hand side b: lcm of the denominators of A^{-1} b."""
    x = solve_rational(A, b)
    assert check_solution(A, b, x)
    return lcm_denominators(x)


def projection_denominator(A, b, u) -> int:
    """Denominator of the reduced fraction u . (A^{-1} b)."""
    x = solve_rational(A, b)
    s = sum((int(ui) * xi for ui, xi in zip(u, x)), Fraction(0))
    return s.denominator


def hadamard_rows_sq(A) -> int:
    """prod_i ||row_i||_2^2 as an exact integer; |det A|^2 <= this."""
    A = _as_int_rows(A)
    p = 1
    for row in A:
        p *= sum(v * v for v in row)
    return p


def hadamard_lemma_log2(A) -> float:
    """log2 of the bound (sqrt(n) ||A||)^n of Lemma 2.1."""
    A = _as_int_rows(A)
    n = len(A)
    amax = max((abs(v) for row in A for v in row), default=0)
    if amax == 0:
        return float("-inf")
    return n * (0.5 * math.log2(n) + math.log2(amax))


def matmul(A, B) -> list[list[int]]:
    A = _as_int_rows(A)
    B = _as_int_rows(B)
    n, m, p = len(A), len(B), len(B[0]) if B else 0
    return [[sum(A[i][k] * B[k][j] for k in range(m)) for j in range(p)]
            for i in range(n)]
