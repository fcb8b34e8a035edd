"""The seeded input generators (no method arithmetic): the fast limb-form
lift-heavy generator must produce exactly the matrix of the Python-int
construction U diag(1, ..., 1, d) V from the same random stream."""
import workloads
from oracle import exact


def test_lift_heavy_limbs_matches_python_sandwich():
    for n, bits in [(5, 64), (17, 100), (33, 300)]:
        mag, sgn, d = workloads.lift_heavy_limbs(n, dbits=bits, seed=n)
        A = workloads.from_limbs(mag, sgn)
        g = workloads.rng(n)
        M = [[0] * n for _ in range(n)]
        for i in range(n):
            M[i][i] = 1
        M[n - 1][n - 1] = d
        workloads._row_ops(M, 4 * n, g, 3)
        workloads._col_ops(M, 4 * n, g, 3)
        assert A == M
        assert d.bit_length() == bits and d % 2 == 1


def test_lift_heavy_limbs_det_is_d():
    mag, sgn, d = workloads.lift_heavy_limbs(9, dbits=80, seed=3)
    assert exact.bareiss_det(workloads.from_limbs(mag, sgn)) == d
