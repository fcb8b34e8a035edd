"""Parameter formulas of the paper (oracle; test-only).

* k_default -- Lemma 2.1(iv): k >= ceil(log(1/eps) / (log P' - log(log_l H)))
  with P' = |P| - ceil(log_l H). Alg. 4.1 line 1 prints the same quantity
  with the ceiling misplaced; the lemma's form is used.
* rhs_range -- Alg. 4.1's S = 13 E(#factors)^3 ceil(log H)^4, with
  E(#factors) = ceil(sqrt(2 log2 n)) + 3 (Section 4.1) and log = log2,
  clamped to 2^62 so that the right-hand side fits in 64 bits.
"""
from __future__ import annotations

import math


def k_default(eps_log2: float, pool_size: int, log2_H: float, l: int) -> int | None:
    """Lemma 2.1(iv) number of agreeing steps; None when the pool is too
    small for the lemma (P' <= log_l H)."""
    logl_H = log2_H / math.log2(l)
    if logl_H <= 0:
        return 1
    Pp = pool_size - math.ceil(logl_H)
    if Pp <= logl_H:
        return None
    return max(1, math.ceil(-eps_log2 / (math.log2(Pp) - math.log2(logl_H))))


def expected_factors(n: int) -> int:
    return math.ceil(math.sqrt(2.0 * math.log2(max(n, 2)))) + 3


def rhs_range(n: int, log2_H: float) -> int:
    e = expected_factors(n)
    lh = math.ceil(max(log2_H, 1.0))
    log2_S = math.log2(13) + 3 * math.log2(e) + 4 * math.log2(lh)
    if log2_S >= 62:
        return 1 << 62
    return 13 * e ** 3 * lh ** 4
