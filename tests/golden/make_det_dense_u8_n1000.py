"""Writes det_dense_u8_n1000_seed0.txt: the exact determinant of the
n = 1000 workload (entries uniform in [0, 255], numpy PCG64 seed 0), computed
by the CPU oracle alone.

Method (Section 2.1, Lemma 2.1(i)): det(A) mod p by the oracle's plain
elimination for the primes above 2^20 in increasing order, until their
product M satisfies M^2 > 4 H^2 with H^2 = prod_i ||row_i||^2 computed
exactly (Hadamard's bound); then det is the symmetric-range Chinese
remainder of the residues. Nothing from the CUDA path is used.

Usage: python tests/golden/make_det_dense_u8_n1000.py  (about 650 primes;
a few minutes on 8 cores)
"""
import hashlib
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402
from oracle import cra, exact, modular  # noqa: E402

OUT = os.path.join(HERE, "det_dense_u8_n1000_seed0.txt")


def main():
    A = workloads.dense_u8(1000, seed=0)
    H2 = exact.hadamard_rows_sq(A.tolist())
    pool = modular.primes_in(1 << 20, 1 << 22)
    primes, M = [], 1
    for q in pool:
        if M * M > 4 * H2:
            break
        primes.append(q)
        M *= q
    t0 = time.time()
    res = modular.det_mod_primes(A, primes, threads=os.cpu_count() or 1)
    det = cra.crt_symmetric([int(r) for r in res], primes)
    assert det * det <= H2
    digest = hashlib.sha256(A.astype("<i8").tobytes()).hexdigest()
    with open(OUT, "w") as f:
        f.write("# det of workloads.dense_u8(1000, seed=0): oracle elimination mod the\n")
        f.write("# first primes above 2^20 past twice Hadamard's bound, then CRT\n")
        f.write("# (tests/golden/make_det_dense_u8_n1000.py)\n")
        f.write(f"workload dense_u8 n=1000 seed=0\n")
        f.write(f"sha256_int64le {digest}\n")
        f.write(f"primes {len(primes)} first {primes[0]} last {primes[-1]}\n")
        f.write(f"bits {abs(det).bit_length()}\n")
        f.write(f"det {'-' if det < 0 else ''}{abs(det):x}\n")
    print(f"{len(primes)} primes in {time.time() - t0:.1f} s; det has {abs(det).bit_length()} bits")


if __name__ == "__main__":
    main()
