"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

None of these tests re-types the oracle's formula: each checks it against an
independent fact (brute force, a closed form, an invariant, a value stated in
the paper) chosen so that a dropped term, a wrong sign or index, or a
transposed operand in the oracle fails at least one of them.
"""
import itertools
import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest

import et_streams
import workloads
from oracle import cra, dixon, exact, modular, params

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def leibniz(A):
    n = len(A)
    total = 0
    for perm in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if perm[i] > perm[j])
        prod = 1
        for i in range(n):
            prod *= int(A[i][perm[i]])
        total += -prod if inv % 2 else prod
    return total


def rand_mat(n, lo, hi, seed):
    r = random.Random(seed)
    return [[r.randint(lo, hi) for _ in range(n)] for _ in range(n)]


# --- Bareiss determinant --------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_bareiss_vs_leibniz_random(n):
    for seed in range(25):
        A = rand_mat(n, -9, 9, 1000 * n + seed)
        assert exact.bareiss_det(A) == leibniz(A)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_bareiss_vs_leibniz_adversarial(n):
    r = random.Random(n)
    cases = []
    A = rand_mat(n, -3, 3, n)
    A[0][0] = 0                        # zero leading pivot: needs a swap
    cases.append(A)
    B = rand_mat(n, -3, 3, n + 1)
    B[n - 1] = list(B[0])              # repeated row: det 0
    cases.append(B)
    C = rand_mat(n, -3, 3, n + 2)
    for i in range(n):
        C[i][n // 2] = 0               # zero column
    cases.append(C)
    D = [[0] * n for _ in range(n)]    # anti-diagonal: sign of a permutation
    for i in range(n):
        D[i][n - 1 - i] = r.randint(1, 5)
    cases.append(D)
    E = rand_mat(n, 0, 1, n + 3)       # 0/1 entries, frequent zero pivots
    cases.append(E)
    for M in cases:
        assert exact.bareiss_det(M) == leibniz(M)


def test_vandermonde_closed_form():
    for seed in range(5):
        r = random.Random(seed)
        n = 7 + seed
        xs = r.sample(range(-40, 40), n)
        V = [[x ** j for j in range(n)] for x in xs]
        want = 1
        for i in range(n):
            for j in range(i + 1, n):
                want *= xs[j] - xs[i]
        assert exact.bareiss_det(V) == want


def test_triangular_product_of_diagonal():
    for seed in range(5):
        n = 12
        A = rand_mat(n, -50, 50, seed)
        U = [[A[i][j] if j >= i else 0 for j in range(n)] for i in range(n)]
        L = [[A[i][j] if j <= i else 0 for j in range(n)] for i in range(n)]
        d = math.prod(A[i][i] for i in range(n))
        assert exact.bareiss_det(U) == d
        assert exact.bareiss_det(L) == d
        # reversing the row order of U multiplies det by the sign of the
        # reversal permutation, (-1)^(n(n-1)/2)
        R = U[::-1]
        assert exact.bareiss_det(R) == d * (-1) ** (n * (n - 1) // 2)


def test_multiplicativity():
    for seed in range(6):
        n = 9
        A = rand_mat(n, -20, 20, seed)
        B = rand_mat(n, -20, 20, seed + 100)
        AB = exact.matmul(A, B)
        assert exact.bareiss_det(AB) == exact.bareiss_det(A) * exact.bareiss_det(B)


def test_unimodular_invariance_and_swap_sign():
    r = random.Random(3)
    n = 10
    A = rand_mat(n, -30, 30, 77)
    d = exact.bareiss_det(A)
    M = [row[:] for row in A]
    for _ in range(40):          # row_i += c * row_j keeps the determinant
        i, j = r.sample(range(n), 2)
        c = r.choice([-3, -2, -1, 1, 2, 3])
        M[i] = [a + c * b for a, b in zip(M[i], M[j])]
    assert exact.bareiss_det(M) == d
    M[0], M[5] = M[5], M[0]      # one swap flips the sign
    assert exact.bareiss_det(M) == -d
    T = [list(col) for col in zip(*A)]   # transpose keeps det
    assert exact.bareiss_det(T) == d


def test_hadamard_bound_holds_and_is_tight_for_orthogonal_rows():
    for seed in range(6):
        A = rand_mat(12, -100, 100, seed)
        d = exact.bareiss_det(A)
        assert d * d <= exact.hadamard_rows_sq(A)
        amax = max(abs(v) for row in A for v in row)
        assert d * d <= (12 * amax * amax) ** 12
    # Sylvester Hadamard matrix of order 8: |det| = 8^(8/2) attains the bound
    H = [[1]]
    for _ in range(3):
        H = [r + r for r in H] + [r + [-v for v in r] for r in H]
    d = exact.bareiss_det(H)
    assert d * d == exact.hadamard_rows_sq(H) == 8 ** 8


# --- rational solve and largest invariant factor ----------------------------------

def test_solve_rational_matches_cramer():
    for seed in range(4):
        n = 6
        A = rand_mat(n, -9, 9, seed + 50)
        b = [random.Random(seed).randint(-20, 20) for _ in range(n)]
        d = exact.bareiss_det(A)
        if d == 0:
            continue
        x = exact.solve_rational(A, b)
        for j in range(n):
            Aj = [row[:] for row in A]
            for i in range(n):
                Aj[i][j] = b[i]
            assert x[j] == Fraction(leibniz(Aj), leibniz(A))


def test_lif_divides_det():
    for seed in range(5):
        A = rand_mat(15, -50, 50, seed)
        b = [random.Random(seed + 9).randint(-1000, 1000) for _ in range(15)]
        d = exact.bareiss_det(A)
        s = exact.largest_invariant_factor(A, b)
        assert d % s == 0


def _unimodular(n, nops, seed):
    r = random.Random(seed)
    U = [[int(i == j) for j in range(n)] for i in range(n)]
    for _ in range(nops):
        i, j = r.sample(range(n), 2)
        c = r.choice([-1, 1])
        U[i] = [a + c * b for a, b in zip(U[i], U[j])]
    return U


@pytest.mark.parametrize("n", [6, 10, 16])
def test_engineered_smith_diag_1_to_n(n):
    """Table 1 matrices: Smith form of diag(1..n), so det = n! and, for the
    right-hand side b = U * (1,...,1), A^{-1} b = V^{-1} (1, 1/2, ..., 1/n)
    whose lcm of denominators is lcm(1..n) = s_n."""
    U = _unimodular(n, 3 * n, n)
    V = _unimodular(n, 3 * n, n + 1)
    D = [[(i + 1) if i == j else 0 for j in range(n)] for i in range(n)]
    A = exact.matmul(exact.matmul(U, D), V)
    assert exact.bareiss_det(A) == math.factorial(n)
    b = [sum(row) for row in U]
    lcm = 1
    for k in range(1, n + 1):
        lcm = lcm * k // math.gcd(lcm, k)
    assert exact.largest_invariant_factor(A, b) == lcm


def test_workload_engineered_smith_det():
    A = workloads.engineered_smith(20, seed=1)
    assert exact.bareiss_det(A.tolist()) == math.factorial(20)


# --- modular elimination ------------------------------------------------------------

PRIMES21 = [1048583, 1048589, 1048601, 1048609, 2097143, 2097091]


def test_det_mod_p_matches_exact_det():
    A = workloads.dense_pm100(40, seed=4)
    d = exact.bareiss_det(A.tolist())
    for p in PRIMES21 + [2, 3, 65537, 2147483647]:
        assert modular.det_mod_p(A, p) == d % p


def test_det_mod_p_when_p_divides_det():
    p = 1048583
    A = workloads.dense_pm100(12, seed=1)
    A[:, 0] *= p      # every term of det now has a factor p
    assert modular.det_mod_p(A, p) == 0
    assert modular.det_mod_p(A, 1048589) == exact.bareiss_det(A.tolist()) % 1048589


def test_rank_count_nx2_01_matches_paper():
    rows = []
    with open(os.path.join(GOLDEN, "rank1_nx2_01.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(tuple(int(v) for v in line.split()))
    for n, want, total in rows:
        cnt = 0
        for bits in range(1 << (2 * n)):
            M = np.array([[(bits >> (2 * i + j)) & 1 for j in range(2)]
                          for i in range(n)], dtype=np.int64)
            if modular.rank_mod_p(M, 2) == 1:
                cnt += 1
        assert total == 1 << (2 * n)
        assert cnt == want == 3 * (2 ** n - 1)


def test_lu_factors_and_first_nonzero_pivot():
    p = 1048583
    A = workloads.dense_pm100(9, seed=2)
    A[0, 0] = 0
    A[1, 0] = p          # also zero mod p: the first nonzero is row 2
    LU, perm, d, stop = modular.lu_mod_p(A, p)
    assert stop == 9
    assert perm[0] == 2
    n = 9
    L = np.eye(n, dtype=object)
    U = np.zeros((n, n), dtype=object)
    for i in range(n):
        for j in range(n):
            if j < i:
                L[i, j] = int(LU[i, j])
            else:
                U[i, j] = int(LU[i, j])
    PA = np.array([[int(A[perm[i], j]) for j in range(n)] for i in range(n)], dtype=object)
    assert ((L.dot(U) - PA) % p == 0).all()
    assert d == exact.bareiss_det(A.tolist()) % p


def test_inverse_mod_p():
    p = 2147483647
    A = workloads.dense_pm100(17, seed=3)
    inv = modular.inverse_mod_p(A, p)
    prod = (A.astype(object).dot(inv.astype(object))) % p
    assert (prod == np.eye(17, dtype=object)).all()


def test_prime_utilities():
    pr = modular.primes_in(1 << 20, 1 << 21)
    assert len(pr) == 73586            # pi(2^21) - pi(2^20) = 155611 - 82025
    assert all(modular.is_prime(q) for q in pr[:50] + pr[-50:])
    assert not modular.is_prime(1048583 * 3)


# --- Chinese remaindering -----------------------------------------------------------

def test_crt_symmetric_recovers_integers():
    r = random.Random(11)
    primes = PRIMES21[:4]
    M = math.prod(primes)
    for N in [0, 1, -1, 12345, -987654321, M // 2, -(M // 2)] + \
             [r.randint(-(M // 2), M // 2) for _ in range(50)]:
        res = [N % p for p in primes]
        assert cra.crt_symmetric(res, primes) == N
    # symmetric range: -floor(M/2) <= r < ceil(M/2) (M odd here)
    assert cra.crt_symmetric([(M // 2 + 1) % p for p in primes], primes) == M // 2 + 1 - M


def test_et_cra_terminates_on_small_det_and_certifies_large():
    pool = modular.primes_in(1 << 20, 1 << 21)
    r = random.Random(5)
    primes = r.sample(pool, 60)
    d = -123456789012345
    res = [d % p for p in primes]
    v, used, why = cra.et_cra(res, primes, log2_H=600.0, eps_log2=-64,
                              l=1 << 20, pool_size=len(pool))
    assert why == "et" and v == d and used < 20
    big = r.randint(1 << 400, 1 << 401)
    res = [big % p for p in primes]
    v, used, why = cra.et_cra(res, primes, log2_H=402.0, eps_log2=-64,
                              l=1 << 20, pool_size=len(pool), certify=True)
    assert why == "bound" and v == big


def test_k_default_is_minimal_solution_of_lemma_inequality():
    """Lemma 2.1(iv) proof: (log_l H / P')^k < eps; k is the least such."""
    for log2_H, pool in [(997.0, 73586), (12977.0, 73586), (103932.0, 73586)]:
        l = 1 << 20
        k = params.k_default(-64, pool, log2_H, l)
        ratio = (log2_H / 20) / (pool - math.ceil(log2_H / 20))
        assert ratio ** k < 2.0 ** -64
        assert ratio ** (k - 1) >= 2.0 ** -64


# --- Dixon lifting -------------------------------------------------------------------

def test_dixon_invariants_and_reconstruction():
    n = 8
    A = workloads.dense_pm100(n, seed=8)
    b = workloads.random_rhs(n, 1000, seed=8)
    p = 2147483629
    d = exact.bareiss_det(A.tolist())
    assert d % p != 0
    m = 6
    digits, rm = dixon.dixon_digits(A, b, p, m)
    for j in range(n):
        assert all(abs(digits[i][j]) <= (p - 1) // 2 for i in range(m))
    X = [dixon.padic_value(digits, p, j) for j in range(n)]
    Q = p ** m
    for i in range(n):          # A X + p^m r_m == b exactly
        s = sum(int(A[i, j]) * X[j] for j in range(n))
        assert s + Q * rm[i] == int(b[i])
    x = exact.solve_rational(A.tolist(), b.tolist())
    Nb = max(abs(v.numerator) for v in x)
    Db = abs(d)
    assert 2 * Nb * Db < Q
    for j in range(n):
        num, den = dixon.rational_reconstruct(X[j], Q, Nb, Db)
        assert Fraction(num, den) == x[j]


# --- helpers the parity tests rely on -------------------------------------------

def _sylvester_hadamard(k):
    """Order 2^k matrix with entries +-1 and mutually orthogonal rows."""
    H = [[1]]
    for _ in range(k):
        H = [r + r for r in H] + [r + [-v for v in r] for r in H]
    return H


@pytest.mark.parametrize("threads", [1, 3])
def test_det_mod_primes_batch_agrees_with_exact_det(threads):
    """The multi-prime oracle (one elimination per prime, threads over the
    primes) gives det mod p for every prime of the list, in list order,
    including a prime that divides det (a zero residue)."""
    A = rand_mat(9, -50, 50, seed=41)
    d = exact.bareiss_det(A)
    primes = [1048583, 1048589, 2147483629, 1048601, 2147483587, 1048609, 1048613]
    got = modular.det_mod_primes(np.array(A, dtype=np.int64), primes, threads=threads)
    assert [int(v) for v in got] == [d % p for p in primes]
    p = 1048627
    B = [[p, 0, 0], [3, 1, 0], [5, 7, 2]]          # det = 2 p
    U = [[1, 2, 0], [0, 1, 3], [0, 0, 1]]          # unimodular
    BU = exact.matmul(B, U)
    got = modular.det_mod_primes(np.array(BU, dtype=np.int64), [p, 1048633], threads=threads)
    assert [int(v) for v in got] == [0, (2 * p) % 1048633]


def test_check_solution_accepts_the_solution_and_rejects_a_perturbed_one():
    A = rand_mat(6, -9, 9, seed=42)
    while exact.bareiss_det(A) == 0:
        A[0][0] += 1
    b = [3, -1, 4, 1, -5, 9]
    x = exact.solve_rational(A, b)
    assert exact.check_solution(A, b, x)
    y = list(x)
    y[2] += Fraction(1, 7)
    assert not exact.check_solution(A, b, y)


def test_lcm_denominators_closed_forms():
    assert exact.lcm_denominators([]) == 1
    assert exact.lcm_denominators([3, -4, 0]) == 1
    assert exact.lcm_denominators([Fraction(1, 2), Fraction(1, 3), Fraction(5, 6)]) == 6
    assert exact.lcm_denominators([Fraction(4, 8), Fraction(-9, 12)]) == 4   # 1/2, -3/4
    assert exact.lcm_denominators([Fraction(1, 2 ** 40), Fraction(1, 3 ** 25)]) == 2 ** 40 * 3 ** 25


def test_projection_denominator_diagonal_and_divisibility():
    """For a diagonal A and b = 1 the solution is x_i = 1/d_i, so u . x is an
    explicit fraction; in general the denominator of u . x divides the lcm of
    the denominators of x (the largest invariant factor for b)."""
    D = [[2, 0, 0, 0], [0, 3, 0, 0], [0, 0, 5, 0], [0, 0, 0, 7]]
    one = [1, 1, 1, 1]
    assert exact.projection_denominator(D, one, [1, 1, 1, 1]) == 210   # 247/210
    assert exact.projection_denominator(D, one, [2, 0, 0, 0]) == 1
    assert exact.projection_denominator(D, one, [0, 3, 5, 0]) == 1     # 3/3 + 5/5 = 2
    assert exact.projection_denominator(D, one, [0, 1, 5, 0]) == 3     # 1/3 + 1 = 4/3
    r = random.Random(43)
    for n in (3, 5, 7):
        A = rand_mat(n, -6, 6, seed=n + 100)
        if exact.bareiss_det(A) == 0:
            continue
        b = [r.randint(-20, 20) for _ in range(n)]
        u = [r.randint(0, 1 << 16) for _ in range(n)]
        s = exact.largest_invariant_factor(A, b)
        assert s % exact.projection_denominator(A, b, u) == 0


def test_hadamard_log2_forms_meet_at_orthogonal_rows():
    """Rows of +-1 that are mutually orthogonal reach both bounds:
    |det| = prod ||row_i|| = (sqrt(n) max|a|)^n = n^(n/2)."""
    for k in (1, 2, 3):
        H = _sylvester_hadamard(k)
        n = len(H)
        want = 0.5 * n * math.log2(n)
        assert math.log2(abs(exact.bareiss_det(H))) == pytest.approx(want, abs=1e-12)
        assert exact.hadamard_lemma_log2(H) == pytest.approx(want, abs=1e-12)
        assert dixon.hadamard_log2_rows(H) == pytest.approx(want, abs=1e-12)
    assert exact.hadamard_lemma_log2([[0, 0], [0, 0]]) == float("-inf")


def test_hadamard_row_bound_float_and_exact_forms_agree():
    for seed in range(4):
        A = rand_mat(7, -1000, 1000, seed=seed + 200)
        exact_log2 = 0.5 * math.log2(exact.hadamard_rows_sq(A))
        assert dixon.hadamard_log2_rows(A) == pytest.approx(exact_log2, rel=1e-12)
        assert exact.hadamard_lemma_log2(A) >= dixon.hadamard_log2_rows(A) - 1e-9


def test_dixon_inverse_is_an_inverse_mod_p():
    p = 2147483629
    A = rand_mat(8, -100, 100, seed=44)
    C = dixon.inverse_balanced(np.array(A, dtype=np.int64), p)
    for i in range(8):
        for j in range(8):
            v = sum(int(C[i][k]) * A[k][j] for k in range(8)) % p
            assert v == (1 if i == j else 0)
        assert all(abs(int(c)) <= (p - 1) // 2 for c in C[i])


# --- Early termination: the false-stop probability of Lemma 2.1(iii) --------------

def _false_stop_rate(eps, trials=4000):
    D, log2H, P, streams = et_streams.adversarial_streams(trials)
    wrong = 0
    for res, primes in streams:
        v, used, why = cra.et_cra(res, primes, log2H, math.log2(eps), 1 << 20, P)
        if why == "et" and v != D:
            wrong += 1
    return wrong / trials


def test_et_false_stop_rate_within_lemma_bound():
    """Lemma 2.1(iii): stopping when the on-the-fly bound is below eps keeps
    the probability of a wrong result below eps. With eps = 0.05 and about
    43 % of the remaining pool dividing K, the wrong-stop rate over 4000
    random prime orders must stay below eps (the exact hypergeometric rate
    of four consecutive primes from S is 0.035, a binomial sigma 0.003)."""
    rate = _false_stop_rate(0.05)
    assert 0.0 < rate <= 0.05, rate


def test_et_stopping_one_prime_early_exceeds_the_bound(monkeypatch):
    """A stop rule that fires one agreement early (the bound evaluated as if
    k + 1 values had agreed) is caught by the same experiment: its wrong-stop
    rate (about 0.08) exceeds eps."""
    real = cra.on_the_fly_bound
    monkeypatch.setattr(cra, "on_the_fly_bound", lambda Rp, k, P, i: real(Rp, k + 1, P, i + 1))
    assert _false_stop_rate(0.05) > 0.05


# --- Extended bonus (Section 3.2): pi~_k = s~^k / gcd(det(R N), s~^k) --------------

def test_extended_bonus_closed_form_diagonal():
    """A = diag(1, .., 1, a, b) with a | b has Smith form A itself, so the two
    largest invariant factors are a and b. With B = [e_{n-2}, e_{n-1}] and R
    selecting the same two rows, X = [e_{n-2}/a, e_{n-1}/b], s~ = b,
    N = s~ X, R N = diag(b/a, 1): pi~_2 = b^2 / gcd(b/a, b^2) = a b exactly."""
    from oracle import bonus
    n, a, b = 6, 6, 60
    A = [[(a if i == n - 2 else b if i == n - 1 else 1) if i == j else 0 for j in range(n)]
         for i in range(n)]
    e = lambda i: [int(j == i) for j in range(n)]
    pi, s = bonus.extended_bonus(A, [e(n - 2), e(n - 1)], [e(n - 2), e(n - 1)])
    assert (pi, s) == (a * b, b)
    pi1, s1 = bonus.extended_bonus(A, [e(n - 1)], [e(n - 1)])
    assert (pi1, s1) == (b, b)


def _smith_engineered(d, seed):
    """U diag(d) V with random unimodular U, V: Smith form diag(d) when d is a
    divisibility chain."""
    n = len(d)
    r = random.Random(seed)

    def unimodular():
        U = [[int(i == j) for j in range(n)] for i in range(n)]
        for _ in range(3 * n):
            i, j = r.sample(range(n), 2)
            c = r.choice([-2, -1, 1, 2])
            U[i] = [x + c * y for x, y in zip(U[i], U[j])]
        return U

    D = [[d[i] if i == j else 0 for j in range(n)] for i in range(n)]
    return exact.matmul(exact.matmul(unimodular(), D), unimodular())


def test_extended_bonus_divides_and_usually_equals_pi_k():
    """Lemmas 3.5 and 3.6: pi~_k always divides pi_k, the product of the k
    largest invariant factors (checked on a chain with the small primes 2, 3,
    5, which random determinants often share); when the invariant factors are
    products of large primes, random B and R give pi~_k = pi_k except with
    probability about k / 1000 per prime (Lemma 3.7's under-estimation comes
    from primes dividing det(R N) by chance)."""
    from oracle import bonus
    for d, need in (([1, 1, 1, 1, 2, 6, 12, 60], 0),
                    ([1, 1, 1, 1009, 1009 * 1013, 1009 * 1013 * 1019], 10)):
        n = len(d)
        hits = {1: 0, 2: 0, 3: 0}
        trials = 12
        for t in range(trials):
            A = _smith_engineered(d, 100 + t)
            r = random.Random(200 + t)
            for k in (1, 2, 3):
                B = [[r.randint(-(1 << 20), 1 << 20) for _ in range(n)] for _ in range(k)]
                R = [[r.randint(-(1 << 20), 1 << 20) for _ in range(n)] for _ in range(k)]
                pi, s = bonus.extended_bonus(A, B, R)
                pik = math.prod(d[n - k:])
                assert pik % pi == 0 and d[-1] % s == 0
                hits[k] += pi == pik
        assert min(hits.values()) >= need, (d, hits)
