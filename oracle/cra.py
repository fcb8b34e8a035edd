"""Chinese remaindering with early termination (oracle; test-only).

Follows Section 2.1 of the paper:
* crt_symmetric -- the value modulo p_0...p_t, taken in the symmetric range
  -floor(M/2) <= r < ceil(M/2) (proof of Lemma 2.1(i)), computed by the
  textbook CRT formula r = sum_k d_k M_k (M_k^{-1} mod p_k) mod M.
* et_cra -- Algorithm 2.1 (Early Terminated CRA): add one modular
  determinant at a time, reconstruct r_i by the two-modulus CRT step,
  track k = max{t : r_{i-t} = ... = r_i} and stop when the on-the-fly bound
  of Lemma 2.1(iii) drops below epsilon or when prod p_i >= 2H.
"""
from __future__ import annotations

import math


def symmetric(r: int, M: int) -> int:
    """Representative of r mod M in -floor(M/2) <= r < ceil(M/2)."""
    r %= M
    if r >= (M + 1) // 2:
        r -= M
    return r


def crt_symmetric(residues, primes) -> int:
    M = 1
    for p in primes:
        M *= int(p)
    r = 0
    for d, p in zip(residues, primes):
        p = int(p)
        Mk = M // p
        r += int(d) * Mk * pow(Mk % p, -1, p)
    return symmetric(r, M)


def crt_step(r: int, M: int, d: int, p: int) -> tuple[int, int]:
    """Combine r mod M with d mod p (gcd(M, p) = 1): the unique value mod Mp
    congruent to r mod M and to d mod p, in the symmetric range."""
    t = ((d - r) * pow(M % p, -1, p)) % p
    Mp = M * p
    return symmetric(r + M * t, Mp), Mp


def log_l(x: float | int, l: int) -> float:
    if isinstance(x, int):
        if x <= 0:
            return float("-inf")
        return (math.log2(x)) / math.log2(l)
    return math.log(x) / math.log(l)


def log2_int(x: int) -> float:
    """log2 of a positive Python int without float overflow."""
    if x <= 0:
        return float("-inf")
    b = x.bit_length()
    if b <= 1000:
        return math.log2(x)
    return math.log2(x >> (b - 900)) + (b - 900)


def R_prime(log2_H: float, r: int, log2_M: float, l: int) -> int:
    """R' = ceil(log_l((H + |r|) / (p_0 ... p_{i-k}))) of Lemma 2.1(iii)
    (clamped at 0: a count of primes)."""
    lr = log2_int(abs(r)) if r else float("-inf")
    hi, lo = max(log2_H, lr), min(log2_H, lr)
    log2_num = hi + math.log2(1.0 + 2.0 ** (lo - hi)) if lo > float("-inf") else hi
    v = (log2_num - log2_M) / math.log2(l)
    return max(0, math.ceil(v - 1e-12))


def on_the_fly_bound(Rp: int, k: int, P: int, i: int) -> float:
    """R'(R'-1)...(R'-k+1) / ((|P|-i+k-1)...(|P|-i)) (Alg. 2.1 until-test)."""
    num = 1.0
    den = 1.0
    for j in range(k):
        num *= max(0, Rp - j)
        den *= (P - i + k - 1 - j)
    if den <= 0:
        return float("inf")
    return num / den


def et_cra(residues, primes, log2_H: float, eps_log2: float, l: int,
           pool_size: int, certify: bool = False):
    """Run Alg. 2.1 over the given stream of (p_i, det mod p_i).

    Returns (r, primes_used, reason) where reason is "et" (early
    termination), "bound" (prod p >= 2H) or "exhausted" (stream ended).
    With certify=True only the bound stops the loop.
    """
    r, M = 0, 1
    hist = []  # r_i values
    logM_hist = []
    eps = 2.0 ** eps_log2
    for idx, (d, p) in enumerate(zip(residues, primes)):
        r, M = crt_step(r, M, int(d), int(p))
        hist.append(r)
        logM_hist.append(log2_int(M))
        i = idx  # index of the prime just added
        k = 0
        while k < i and hist[i - k - 1] == r:
            k += 1
        i_used = i + 1
        if log2_int(M) >= 1.0 + log2_H:
            return r, i_used, "bound"
        if certify:
            continue
        Rp = R_prime(log2_H, r, logM_hist[i - k], l)
        if k > 0 and on_the_fly_bound(Rp, k, pool_size, i_used) < eps:
            return r, i_used, "et"
    return r, len(hist), "exhausted"
