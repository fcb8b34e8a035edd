"""Parameter formulas of the paper (oracle; test-only).

* k_default -- Lemma 2.1(iv): k >= ceil(log(1/eps) / (log P' - log(log_l H)))
  with P' = |P| - ceil(log_l H). Alg. 4.1 line 1 prints the same quantity
  with the ceiling misplaced; the lemma's form is used.
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
