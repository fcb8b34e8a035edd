"""Residue streams on which Alg. 2.1 can stop early on a wrong value, for the
statistical pin of Lemma 2.1(iii) (test input only: it draws primes and
values, it does no reconstruction)."""
import math
import random

from oracle import cra, modular


def adversarial_streams(trials, seed=1, R=500, extra=12):
    """The pool P is every prime in (2^20, 2^20 + 2^14) and l = 2^20, so each
    prime adds just over one unit of log_l and Lemma 2.1(iii)'s R' is tight.
    A fixed prefix of three primes p0 p1 p2 is followed by the rest of the
    pool in a random order (sampling without replacement). The determinant is
    D = r* + K p0 p1 p2 with K the product of a random set S of R pool primes:
    after the prefix the reconstruction is r* != D, and it stays r* exactly
    while the primes drawn divide K, so a run of k primes from S makes k
    false agreements (Lemma 2.1(ii)). Each stream is cut after `extra` random
    primes (a false stop needs the first few of them; later ones can only
    stop on other wrong values with negligible probability). Returns
    (D, log2 H, pool size, [(residues, primes)])."""
    pool = modular.primes_in(1 << 20, (1 << 20) + (1 << 14))
    rng = random.Random(seed)
    prefix = rng.sample(pool, 3)
    rest = [q for q in pool if q not in prefix]
    K = math.prod(rng.sample(rest, R))
    Mt = math.prod(prefix)
    D = Mt // 3 + 12345 + K * Mt
    log2H = cra.log2_int(D) + 1e-9
    streams = []
    for t in range(trials):
        order = rest[:]
        random.Random(1000 + t).shuffle(order)
        primes = prefix + order[:extra]
        streams.append(([D % q for q in primes], primes))
    return D, log2H, len(pool), streams
