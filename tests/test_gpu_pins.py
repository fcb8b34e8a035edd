"""Pins of the CUDA path at the headline sizes, at the worst cases of its
arithmetic, and of its stopping and failure-detection rules, against the CPU
oracle or against facts that hold by construction.

Every call goes through the C ABI (the ctypes binding marshals arguments
only). Integer results are compared bit for bit.
"""
import hashlib
import math
import os
import random

import numpy as np
import pytest

import et_streams
import workloads
from oracle import cra, dixon, exact, modular

pytestmark = pytest.mark.gpu

idet = pytest.importorskip("paper_cs_0511066_b300")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
P21 = modular.primes_in(1 << 20, 1 << 21)
CORES = os.cpu_count() or 1


def p31(k, seed):
    r = random.Random(seed)
    out = []
    while len(out) < k:
        c = r.randrange(1 << 30, 1 << 31) | 1
        if modular.is_prime(c) and c not in out:
            out.append(c)
    return out


# --- early termination: the device rule against the oracle's Alg. 2.1 --------------

def test_et_stop_index_and_value_match_oracle():
    """The device reconstruction with the host stopping rule (the one
    idet_int_det applies) stops at the same prime as the oracle's Alg. 2.1 and
    returns the same value, on the adversarial streams of the statistical pin
    (false stops included) with eps = 0.05."""
    D, log2H, P, streams = et_streams.adversarial_streams(400)
    eps_log2 = math.log2(0.05)
    false_stops = 0
    for res, primes in streams:
        v, used, why = cra.et_cra(res, primes, log2H, eps_log2, 1 << 20, P)
        dv, stop, dwhy = idet.cra_early_termination(res, primes, log2H, eps_log2, 20.0, P)
        if why == "et":
            assert (dwhy, stop, dv) == (1, used - 1, v)
            false_stops += v != D
        else:
            assert why == "exhausted" and dwhy == 0 and stop == -1
            assert dv == cra.crt_symmetric(res, primes)
    assert false_stops >= 5


def test_et_small_determinant_and_certified_bound():
    """A small determinant stops early at the oracle's prime; with certify the
    device runs 40 bits past 2H (the oracle stops at 2H) and both return det;
    a wrong residue before the bound is reported as inconsistent (reason 3)."""
    primes = random.Random(5).sample(P21, 80)
    d = -123456789012345
    res = [d % q for q in primes]
    v, used, why = cra.et_cra(res, primes, 600.0, -64, 1 << 20, len(P21))
    dv, stop, dwhy = idet.cra_early_termination(res, primes, 600.0, -64.0, 20.0, len(P21))
    assert why == "et" and (dwhy, stop, dv) == (1, used - 1, v) and v == d
    big = random.Random(6).randint(1 << 400, 1 << 401)
    res = [big % q for q in primes]
    v, used, why = cra.et_cra(res, primes, 402.0, -64, 1 << 20, len(P21), certify=True)
    dv, stop, dwhy = idet.cra_early_termination(res, primes, 402.0, -64.0, 20.0, len(P21),
                                                certify=True)
    assert why == "bound" and v == big and dwhy == 2 and dv == big
    M = math.prod(primes[:stop + 1])
    assert stop >= used - 1 and M >= (1 << (403 + 40)) and M // primes[stop] < (1 << (403 + 40))
    res[7] = (res[7] + 1) % primes[7]
    dv, stop, dwhy = idet.cra_early_termination(res, primes, 402.0, -64.0, 20.0, len(P21),
                                                certify=True)
    assert dwhy == 3


# --- the headline workloads, in full --------------------------------------------------

def _golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split(" ", 1)
        out[k] = v.strip()
    return out


def test_int_det_dense_u8_n1000_full_value():
    """n = 1000, entries in [0, 255]: the whole determinant (about 12,900
    bits) equals the value the oracle's elimination and CRT past twice the
    Hadamard bound produced offline (tests/golden)."""
    torch = pytest.importorskip("torch")
    g = _golden("det_dense_u8_n1000_seed0.txt")
    A = workloads.dense_u8(1000, seed=0)
    assert hashlib.sha256(A.astype("<i8").tobytes()).hexdigest() == g["sha256_int64le"]
    want = int(g["det"], 16)
    assert want.bit_length() == int(g["bits"])
    d, st = idet.int_det(torch.from_numpy(A).cuda(), return_stats=True)
    assert d == want
    assert st["lift_iters"] > 0 and st["et_stop"] == 1, st


def test_int_det_dense_pm2p20_n4000_spot_check_and_lif():
    """n = 4000, entries in [-2^20, 2^20], in the launch configuration the
    benchmark times: the determinant agrees with the oracle's elimination
    modulo eight 31-bit primes drawn independently of the path's, and the
    largest invariant factor for another right-hand side divides it, with a
    cofactor of at most a few bits (random dense matrices have s_n close to
    det)."""
    torch = pytest.importorskip("torch")
    A = workloads.dense_pm2p20(4000, seed=0)
    Ad = torch.from_numpy(A).cuda()
    d, st = idet.int_det(Ad, return_stats=True)
    qs = p31(8, seed=77)
    ref = modular.det_mod_primes(A, qs, threads=CORES)
    assert [d % q for q in qs] == [int(r) for r in ref]
    b = workloads.random_rhs(4000, 1 << 40, seed=9)
    s = idet.largest_invariant_factor(Ad, b)
    assert d % s == 0 and abs(d // s).bit_length() <= 64


def test_int_det_batch_full_512_matches_oracle():
    """The whole batched workload (512 matrices, n log-uniform in [32, 512],
    entries in [-2^10, 2^10]) in one batched call: every determinant agrees
    with the oracle's elimination modulo eight fresh 31-bit primes, and the
    small ones (n <= 40) equal the exact Bareiss determinant."""
    mats = workloads.batch_mix(count=512, nmin=32, nmax=512, bits=10, seed=0)
    got = idet.int_det_batch(mats)
    qs = p31(8, seed=4321)
    for A, d in zip(mats, got):
        ref = modular.det_mod_primes(A, qs, threads=CORES)
        assert [d % q for q in qs] == [int(r) for r in ref], A.shape
        if A.shape[0] <= 40:
            assert d == exact.bareiss_det(A.tolist())


# --- worst cases of the tensor-core accumulations -----------------------------------

def _limbs7(x, L):
    out = []
    for _ in range(L):
        l0 = ((x + 64) & 127) - 64
        out.append(l0)
        x = (x - l0) >> 7
    return out, x


def _worst_lu_matrix(n, p, x):
    """A = L U mod p with L unit lower triangular, every entry below the
    diagonal x, and U upper triangular with unit diagonal, every entry above
    it x: a_ij = min(i, j) x^2 + (1 if i == j else x) mod p. Its LU with the
    first-nonzero pivot needs no exchange and every trailing update
    multiplies blocks whose entries are all x."""
    i = np.arange(n, dtype=object)[:, None]
    j = np.arange(n, dtype=object)[None, :]
    A = (np.minimum(i, j) * (x * x) + np.where(i == j, 1, x)) % p
    LU = np.where(np.arange(n)[:, None] == np.arange(n)[None, :], 1, x % p).astype(np.uint32)
    return A.astype(np.int64), LU


PATHS21 = {"int64": 1, "i8": 2, "f64": 3, "bf16": 4, "tc05": 5}


@pytest.mark.parametrize("path", sorted(PATHS21))
def test_trailing_update_worst_case_21bit(path):
    """Every limb at the edge of its range: x = 1040319 has the 7-bit limbs
    (63, 63, 63), so each limb product group of the rank-128 update sums 128
    terms of the same sign (3 * 128 * 63^2, the largest group); for FP64 every
    entry is (p - 1)/2, the largest balanced residue (128 * 2^40 < 2^53). The
    LU factors must come out exactly as constructed."""
    p = max(q for q in P21 if q < (1 << 21))
    if path == "f64":
        x = (p - 1) // 2
    else:
        x = 1040319
        assert _limbs7(x, 3) == ([63, 63, 63], 0) and 2 * x < p
    A, want = _worst_lu_matrix(300, p, x)
    lu, perm, sing = idet.lu_mod_prime(A, p, update_path=PATHS21[path])
    assert not sing and (perm == np.arange(300)).all()
    assert (lu == want).all()
    assert list(idet.det_mod_primes(A, [p], update_path=PATHS21[path])) == [1]


@pytest.mark.parametrize("path", ["int64", "tc05"])
def test_trailing_update_worst_case_31bit(path):
    """31-bit primes, five 7-bit limbs: x has the limbs (63, 63, 63, 63, 3),
    the largest the balanced range allows, so the middle groups sum 4 * 128 *
    63^2 same-sign products."""
    x = 63 * (1 + (1 << 7) + (1 << 14) + (1 << 21)) + 3 * (1 << 28)
    assert _limbs7(x, 5) == ([63, 63, 63, 63, 3], 0)
    p = next(q for q in range((1 << 31) - 1, 2 * x, -2) if modular.is_prime(q))
    A, want = _worst_lu_matrix(300, p, x)
    lu, perm, sing = idet.lu_mod_prime(A, p, update_path=PATHS21[path])
    assert not sing and (perm == np.arange(300)).all()
    assert (lu == want).all()


# --- the whole int32 range of entries ------------------------------------------------

def _int32_edges(n, seed):
    g = np.random.default_rng(seed)
    A = g.integers(-(1 << 31), (1 << 31) - 1, size=(n, n), endpoint=True, dtype=np.int64)
    A[g.random((n, n)) < 0.2] = -(1 << 31)
    A[g.random((n, n)) < 0.1] = (1 << 31) - 1
    return A


def test_int32_range_entries_every_entry_point():
    """Entries equal to -2^31 (and 2^31 - 1), as 32-bit served jobs contain:
    int_det, the batch, the server and the lifting digits agree with the
    oracle; 2^31 itself is refused."""
    A = _int32_edges(24, 1)
    want = exact.bareiss_det(A.tolist())
    assert idet.int_det(A) == want
    assert idet.int_det(A, certify=True) == want
    B = _int32_edges(260, 2)
    qs = p31(3, seed=8)
    dB = idet.int_det(B)
    assert [dB % q for q in qs] == [int(r) for r in modular.det_mod_primes(B, qs)]
    assert idet.int_det_batch([A, B, A[:5, :5]]) == [want, dB, exact.bareiss_det(A[:5, :5].tolist())]
    with idet.Server(slots=2) as srv:
        t1, t2 = srv.submit(A), srv.submit(B)
        assert srv.poll(t1)[0] == want and srv.poll(t2)[0] == dB
    b = workloads.random_rhs(24, 1 << 40, seed=3)
    p = p31(1, 11)[0]
    dg, r = idet.dixon_digits(A, b, p, 4)
    odg, orr = dixon.dixon_digits(A, b, p, 4)
    assert dg.tolist() == odg and r.tolist() == orr
    C = A.copy()
    C[3, 4] = 1 << 31
    with pytest.raises(idet.IdetError) as e:
        idet.int_det(C)
    assert e.value.code == 1


# --- failure detection (a wrong modular determinant, made on the host) -------------

def test_wrong_residue_is_caught_at_the_bound():
    """A modular determinant made wrong on the host: the reconstruction never
    stabilises (no early termination), and at the bound the check |r| <= H
    fails, so the call reports IDET_ERR_INTERNAL instead of a wrong value, in
    certified and in early-terminated mode; the next call is unaffected."""
    A = workloads.dense_pm100(60, seed=4)
    want = exact.bareiss_det(A.tolist())
    for kw in ({"certify": True, "inject_fault": 3}, {"inject_fault": 2},
               {"lif": False, "inject_fault": 1}):
        with pytest.raises(idet.IdetError) as e:
            idet.int_det(A, **kw)
        assert e.value.code == 7, kw
    assert idet.int_det(A, certify=True) == want
    assert idet.int_det(A) == want


# --- the lift: one-product kernel, block lift, bounded waits -----------------------

@pytest.mark.parametrize("n,lo,hi,m", [(5, -100, 100, 4), (67, -100, 100, 5), (300, 0, 255, 3),
                                       (1100, -(1 << 20), 1 << 20, 2)])
def test_block_lift_two_rhs_matches_oracle(n, lo, hi, m):
    """Two right-hand sides lifted in one pass (the block lift): both digit
    sequences and both residuals equal the oracle's Dixon iteration run on
    each right-hand side alone; the stepping kernel reads the lifting matrix
    once per step for both (the same algorithmic bytes as one vector)."""
    A = workloads.dense_uniform(n, lo, hi, seed=n + 3)
    B = np.stack([workloads.random_rhs(n, 1 << 61, seed=n + 4),
                  workloads.random_rhs(n, 1 << 30, seed=n + 5)])
    p = p31(1, n + 6)[0]
    dg, r, st = idet.dixon_digits_block(A, B, p, m, return_stats=True)
    for k in range(2):
        odg, orr = dixon.dixon_digits(A, B[k], p, m)
        assert dg[k].tolist() == odg and r[k].tolist() == orr
    _, _, st1 = idet.dixon_digits_block(A, B[:1], p, m, return_stats=True)
    assert st["lift_path"] == 1 and st["lift_bytes"] == st1["lift_bytes"] == (m - 1) * 4 * n * n


def test_lift_one_product_and_two_product_kernels_agree(monkeypatch):
    """The one-product kernel (E = (C A - I)/p) and the two-product kernel (C
    and A every step) produce the same digits; entries of 32 bits make n
    max|a| exceed 2^32, where only the two-product kernel applies."""
    n, m = 700, 4
    A = workloads.dense_pm2p20(n, seed=31)
    B = np.stack([workloads.random_rhs(n, 1 << 50, seed=32), workloads.random_rhs(n, 9, seed=33)])
    p = p31(1, 34)[0]
    d1, r1, s1 = idet.dixon_digits_block(A, B, p, m, return_stats=True)
    monkeypatch.setenv("IDET_LIFT_PATH", "classic")
    d0, r0, s0 = idet.dixon_digits_block(A, B, p, m, return_stats=True)
    monkeypatch.delenv("IDET_LIFT_PATH")
    assert (s1["lift_path"], s0["lift_path"]) == (1, 0)
    assert (d1 == d0).all() and (r1 == r0).all()
    W = _int32_edges(40, 35)
    b = workloads.random_rhs(40, 1 << 40, seed=36)
    dg, r, st = idet.dixon_digits_block(W, b[None, :], p, 3, return_stats=True)
    odg, orr = dixon.dixon_digits(W, b, p, 3)
    assert st["lift_path"] == 0 and dg[0].tolist() == odg and r[0].tolist() == orr


def test_lift_wait_limit_runs_out_and_recovers():
    """A bounded wait that runs out (the limit lowered to one cycle) ends the
    lifting kernel cleanly: the call returns IDET_ERR_TIMEOUT with
    lift_timed_out set, and the next call with the default limit succeeds."""
    torch = pytest.importorskip("torch")
    A = torch.from_numpy(workloads.dense_pm2p20(4000, seed=2)).cuda()
    b = workloads.random_rhs(4000, 1 << 40, seed=3)
    p = 2147483629
    try:
        idet.set_wait_limit(1)
        with pytest.raises(idet.IdetError) as e:
            idet.dixon_digits(A, b, p, 8)
        assert e.value.code == 5
        with pytest.raises(idet.IdetError) as e:
            idet.int_det(A)
        assert e.value.code == 5 and e.value.stats["lift_timed_out"] != 0
    finally:
        idet.set_wait_limit(0)
    dg, r = idet.dixon_digits(A, b, p, 3)
    X = np.zeros(4000, dtype=object)
    for i in range(2, -1, -1):
        X = X * p + dg[i].astype(object)
    An = workloads.dense_pm2p20(4000, seed=2).astype(object)
    assert (An.dot(X) + (p ** 3) * r.astype(object) == b.astype(object)).all()


def test_lif_completion_with_long_denominators_matches_oracle():
    """Entry-by-entry completion of the denominator when the numbers span many
    radix-p digits: entries near 2^20 and scaled columns (a factor 2^k that a
    random projection misses about half of the time), so that lcm(D, d_j) is
    formed by the extended Euclidean algorithm on numbers of a hundred digits
    whose leading digits differ widely."""
    for seed in range(3):
        A = workloads.dense_pm2p20(120, seed=300 + seed)
        A[:, 0] *= 8
        A[:, 1] *= 2
        b = workloads.random_rhs(120, 1 << 30, seed=seed)
        assert idet.largest_invariant_factor(A, b) == exact.largest_invariant_factor(
            A.tolist(), b.tolist())


# --- the extended bonus (Section 3.2) --------------------------------------------------

def _engineered(d, seed):
    """U diag(d) V with random unimodular U, V (2n elementary operations of
    multiplier +-1 each), entries kept in the int32 range."""
    n = len(d)
    r = random.Random(seed)

    def unimodular():
        U = [[int(i == j) for j in range(n)] for i in range(n)]
        for _ in range(2 * n):
            i, j = r.sample(range(n), 2)
            c = r.choice([-1, 1])
            U[i] = [x + c * y for x, y in zip(U[i], U[j])]
        return U

    D = [[d[i] if i == j else 0 for j in range(n)] for i in range(n)]
    A = exact.matmul(exact.matmul(unimodular(), D), unimodular())
    assert max(abs(v) for row in A for v in row) < (1 << 31)
    return np.array(A, dtype=np.int64)


def test_extended_bonus_closed_form_and_oracle():
    """pi~_2 = s~^2 / gcd(det(R N), s~^2) through the C ABI equals the
    oracle's exact-rational value: on diag(1, .., 1, a, b) with a | b and
    B, R selecting the last two coordinates (pi~_2 = a b), on engineered
    Smith forms with large-prime invariant factors and on random dense
    matrices with random B and R (|b|, |r| up to 2^40)."""
    from oracle import bonus
    n = 6
    A = np.diag([1, 1, 1, 1, 6, 60]).astype(np.int64)
    E = np.zeros((2, n), dtype=np.int64)
    E[0, 4] = E[1, 5] = 1
    assert idet.extended_bonus(A, E, E) == (360, 60)
    g = np.random.default_rng(5)
    cases = [_engineered([1, 1, 1, 1, 101, 101 * 103, 101 * 103 * 107], 7)]
    cases += [workloads.dense_pm100(k, seed=k) for k in (12, 40, 90)]
    for A in cases:
        n = A.shape[0]
        B = g.integers(-(1 << 40), 1 << 40, size=(2, n), dtype=np.int64)
        R = g.integers(-(1 << 40), 1 << 40, size=(2, n), dtype=np.int64)
        want = bonus.extended_bonus(A.tolist(), B.tolist(), R.tolist())
        assert idet.extended_bonus(A, B, R) == want, n


def test_int_det_i_max_2_exact_and_larger_K():
    """Alg. 4.1 with i_max = 2 (two solves in one block lift, then the
    extended bonus): exact determinants on Table 1's engineered matrices
    (det = n!) and on random dense ones; on the engineered ones (about n/2
    invariant factors) K = lcm(s~_n, pi~_2) has more bits than s~_n alone, so
    the CRA of det/K needs no more primes."""
    for n in (60, 150):
        A = workloads.engineered_smith(n, seed=n)
        d1, s1 = idet.int_det(A, return_stats=True)
        d2, s2 = idet.int_det(A, i_max=2, return_stats=True)
        assert d1 == d2 == math.factorial(n)
        assert s2["log2_K"] > s1["log2_K"] + 10 and s2["primes_in_cra"] <= s1["primes_in_cra"], (s1, s2)
    for n, seed in ((40, 1), (120, 2)):
        A = workloads.dense_pm100(n, seed=seed)
        assert idet.int_det(A, i_max=2) == exact.bareiss_det(A.tolist())
    S = workloads.dense_pm100(30, seed=3)
    S[4] = S[9] + S[11]
    assert idet.int_det(S, i_max=2) == 0


def test_prime_bits_31_lift_reuses_a_cra_lu():
    """With CRA primes of the lifting class (31 bits) the lift takes one of
    them, whose LU the first wave kept: only the triangular solves run
    (n^3/6 forward, L^{-1} being lower triangular, plus n^3/2 backward:
    2/3 n^3 MACs instead of 4/3 n^3 with the LU), and the determinant is
    exact."""
    for n, seed in ((90, 1), (300, 2)):
        A = workloads.dense_pm2p20(n, seed=seed)
        d, st = idet.int_det(A, prime_bits=31, return_stats=True)
        if n <= 90:
            assert d == exact.bareiss_det(A.tolist())
        else:
            qs = p31(4, seed=n)
            assert [d % q for q in qs] == [int(r) for r in modular.det_mod_primes(A, qs)]
        assert st["inverse_macs"] == pytest.approx(2.0 / 3.0 * n ** 3), st
        d21, st21 = idet.int_det(A, return_stats=True)
        assert d21 == d and st21["inverse_macs"] == pytest.approx(4.0 / 3.0 * n ** 3)


# --- order of the steps: speculative solve beside the first wave (n >= 500) ------------

def _unimodular_np(n, ops, seed):
    r = np.random.default_rng(seed)
    U = np.eye(n, dtype=np.int64)
    for _ in range(ops):
        i, j = r.choice(n, 2, replace=False)
        U[i] += int(r.choice([-1, 1])) * U[j]
    return U


def test_speculative_order_matches_wave_first(monkeypatch):
    """From n = 500 the inverse and the lift run first and the first CRA wave
    is factored beside the reconstruction. The determinant, the primes used
    and the stopping point are those of the wave-first order (IDET_ET_FIRST),
    for a dense matrix and for det = 7 (K = 7 from the solve, det/K = 1); a
    singular matrix, whose lifting prime's LU is singular, falls back to the
    wave-first order and returns 0."""
    A = workloads.dense_pm100(600, seed=11)
    d_spec, st_spec = idet.int_det(A, return_stats=True)
    monkeypatch.setenv("IDET_ET_FIRST", "1")
    d_first, st_first = idet.int_det(A, return_stats=True)
    monkeypatch.delenv("IDET_ET_FIRST")
    assert d_spec == d_first
    assert st_spec["primes_used"] == st_first["primes_used"]
    assert st_spec["primes_in_cra"] == st_first["primes_in_cra"]
    qs = P21[-5:]
    assert [d_spec % q for q in qs] == [int(x) for x in modular.det_mod_primes(A, qs)]
    # det = 7: U diag(1, ..., 1, 7) V with U, V products of elementary operations
    n = 520
    U, V = _unimodular_np(n, n, 1), _unimodular_np(n, n, 2)
    D = np.eye(n, dtype=np.int64)
    D[-1, -1] = 7
    B = U @ D @ V
    assert np.abs(B).max() < (1 << 31)
    d7, st7 = idet.int_det(B, return_stats=True)
    monkeypatch.setenv("IDET_ET_FIRST", "1")
    d7f, st7f = idet.int_det(B, return_stats=True)
    monkeypatch.delenv("IDET_ET_FIRST")
    assert d7 == d7f == 7
    for key in ("primes_used", "primes_in_cra", "et_stop", "log2_K"):
        assert st7[key] == st7f[key], key
    # two equal rows: det = 0
    S = workloads.dense_pm100(510, seed=12)
    S[17] = S[400]
    assert idet.int_det(S) == 0
