"""Dixon p-adic lifting and rational reconstruction (oracle; test-only).

Section 2.2 solves A x = b "using Dixon p-adic lifting" (cited, not spelled
out). The textbook iteration, with the digit convention used by the CUDA
path stated explicitly:

    C = A^{-1} mod p,   r_0 = b,
    x_i = C r_i mod p   taken in the balanced range [-(p-1)/2, (p-1)/2],
    r_{i+1} = (r_i - A x_i) / p     (exact division).

After m steps X = sum_{i<m} x_i p^i satisfies A X = b - p^m r_m, hence
A X = b mod p^m. The rational solution is recovered from X mod p^m by
rational reconstruction: the textbook extended Euclidean algorithm run on
(p^m, X) stopped at the first remainder <= N, giving the unique N/D with
|N| <= N_bound, 0 < D <= D_bound when 2 N_bound D_bound < p^m.
"""
from __future__ import annotations

import math

import numpy as np

from . import modular


def balanced(v: int, p: int) -> int:
    v %= p
    return v - p if v > (p - 1) // 2 else v


def inverse_balanced(A, p: int) -> list[list[int]]:
    inv = modular.inverse_mod_p(A, p)
    if inv is None:
        raise ValueError("A is singular mod p")
    return [[balanced(int(v), p) for v in row] for row in inv]


def dixon_digits(A, b, p: int, m: int):
    """Return (digits[m][n], r_m, projections) following the iteration above."""
    A = [[int(v) for v in row] for row in np.asarray(A)]
    n = len(A)
    C = inverse_balanced(np.asarray(A, dtype=np.int64), p)
    r = [int(v) for v in b]
    digits = []
    for _ in range(m):
        rm = [balanced(v, p) for v in r]
        x = [balanced(sum(C[i][j] * rm[j] for j in range(n)), p)
             for i in range(n)]
        digits.append(x)
        nr = []
        for i in range(n):
            s = r[i] - sum(A[i][j] * x[j] for j in range(n))
            assert s % p == 0
            nr.append(s // p)
        r = nr
    return digits, r


def padic_value(digits, p: int, j: int) -> int:
    """X_j = sum_i x_{i,j} p^i."""
    X = 0
    for i in range(len(digits) - 1, -1, -1):
        X = X * p + int(digits[i][j])
    return X


def rational_reconstruct(X: int, Q: int, N_bound: int, D_bound: int):
    """(num, den) with num = den * X mod Q, |num| <= N_bound,
    0 < den <= D_bound, by the extended Euclidean algorithm on (Q, X mod Q)
    stopped at the first remainder <= N_bound. Returns None if no such
    fraction exists."""
    r0, r1 = Q, X % Q
    t0, t1 = 0, 1
    while r1 > N_bound:
        q = r0 // r1
        r0, r1 = r1, r0 - q * r1
        t0, t1 = t1, t0 - q * t1
    if t1 == 0 or abs(t1) > D_bound:
        return None
    num, den = r1, t1
    if den < 0:
        num, den = -num, -den
    if math.gcd(num, den) != 1:
        return None
    return num, den


def hadamard_log2_rows(A) -> float:
    A = np.asarray(A, dtype=np.float64)
    return float(0.5 * np.sum(np.log2(np.maximum(np.sum(A * A, axis=1), 1.0))))
