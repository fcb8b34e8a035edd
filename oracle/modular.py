"""ctypes wrapper of oracle/modular.c: plain elimination over Z/p (test-only).

See modular.c for the algorithm (Section 2.1 / Alg. 2.1: det(A) mod p_i by LU
with the first nonzero pivot). Also provides small prime utilities written
from their textbook definitions (trial division, deterministic Miller-Rabin).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "modular.c")
_LIB = os.path.join(_HERE, "_modular.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile modular.c into _modular.so (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or \
            os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i64, u32, i32 = ctypes.c_int64, ctypes.c_uint32, ctypes.c_int32
        P = ctypes.c_void_p
        lib.orc_det_mod_p.argtypes = [P, i64, i64, u32]
        lib.orc_det_mod_p.restype = u32
        lib.orc_det_mod_primes.argtypes = [P, i64, i64, P, i32, P, i32]
        lib.orc_det_mod_primes.restype = None
        lib.orc_lu_mod_p.argtypes = [P, i64, i64, u32, P, P, P]
        lib.orc_lu_mod_p.restype = u32
        lib.orc_rank_mod_p.argtypes = [P, i64, i64, i64, u32]
        lib.orc_rank_mod_p.restype = i64
        lib.orc_inverse_mod_p.argtypes = [P, i64, i64, u32, P]
        lib.orc_inverse_mod_p.restype = i32
        _lib = lib
    return _lib


def _mat(A) -> np.ndarray:
    A = np.ascontiguousarray(np.asarray(A, dtype=np.int64))
    if A.ndim != 2:
        raise ValueError("matrix expected")
    return A


def det_mod_p(A, p: int) -> int:
    A = _mat(A)
    return int(_load().orc_det_mod_p(A.ctypes.data, A.shape[0], A.shape[1], p))


def det_mod_primes(A, primes, threads: int = 0) -> np.ndarray:
    A = _mat(A)
    pr = np.ascontiguousarray(np.asarray(primes, dtype=np.uint32))
    out = np.zeros(len(pr), dtype=np.uint32)
    _load().orc_det_mod_primes(A.ctypes.data, A.shape[0], A.shape[1],
                               pr.ctypes.data, len(pr), out.ctypes.data,
                               threads)
    return out


def lu_mod_p(A, p: int):
    """(LU residues [0,p), perm, det mod p, stopped_at)."""
    A = _mat(A)
    n = A.shape[0]
    LU = np.zeros((n, n), dtype=np.uint32)
    perm = np.zeros(n, dtype=np.int32)
    stop = ctypes.c_int64(0)
    d = _load().orc_lu_mod_p(A.ctypes.data, n, A.shape[1], p, LU.ctypes.data,
                             perm.ctypes.data, ctypes.byref(stop))
    return LU, perm, int(d), int(stop.value)


def rank_mod_p(A, p: int) -> int:
    A = _mat(A)
    return int(_load().orc_rank_mod_p(A.ctypes.data, A.shape[0], A.shape[1],
                                      A.shape[1], p))


def inverse_mod_p(A, p: int) -> np.ndarray | None:
    A = _mat(A)
    n = A.shape[0]
    inv = np.zeros((n, n), dtype=np.uint32)
    rc = _load().orc_inverse_mod_p(A.ctypes.data, n, A.shape[1], p,
                                   inv.ctypes.data)
    return None if rc else inv


# Prime utilities (textbook definitions) ---------------------------------------

def is_prime(m: int) -> bool:
    """Deterministic Miller-Rabin for m < 3.3e24 (bases: first 12 primes)."""
    if m < 2:
        return False
    small = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)
    for q in small:
        if m % q == 0:
            return m == q
    d, s = m - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in small:
        x = pow(a, d, m)
        if x in (1, m - 1):
            continue
        for _ in range(s - 1):
            x = x * x % m
            if x == m - 1:
                break
        else:
            return False
    return True


def primes_in(lo: int, hi: int) -> list[int]:
    """All primes in (lo, hi) by a sieve of Eratosthenes on the interval."""
    import math
    seg = np.ones(hi - lo - 1, dtype=bool)  # lo+1 .. hi-1
    r = int(math.isqrt(hi)) + 1
    base = np.ones(r + 1, dtype=bool)
    base[:2] = False
    for i in range(2, int(math.isqrt(r)) + 1):
        if base[i]:
            base[i * i::i] = False
    for q in np.nonzero(base)[0]:
        q = int(q)
        start = max(q * q, ((lo + 1 + q - 1) // q) * q)
        seg[start - lo - 1::q] = False
    out = [lo + 1 + int(i) for i in np.nonzero(seg)[0]]
    return [v for v in out if v >= 2]
