/* Plain Gaussian elimination over Z/p (oracle; test infrastructure only).
 *
 * Section 2.1 of Dumas & Urbanska computes det(A) mod p_i "using the LU
 * factorization modulo p_i" inside the CRA loop (Alg. 2.1). This file is the
 * textbook O(n^3) elimination that defines those values, with no blocking,
 * no delayed reduction and no tensor arithmetic:
 *
 *   for each column k: take as pivot the FIRST row i >= k (lowest index) whose
 *   entry in column k is nonzero mod p; swap it into row k (flipping the
 *   sign); eliminate below with l_ik = a_ik / a_kk.
 *   det(A) mod p = sign * prod_k a_kk.
 *
 * Residues are kept in [0, p); p < 2^32. OpenMP runs independent primes in
 * parallel. Nothing here is shared with the CUDA path.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static uint32_t red64(int64_t a, uint32_t p) {
    int64_t r = a % (int64_t)p;
    if (r < 0) r += p;
    return (uint32_t)r;
}

static uint32_t mulmod(uint32_t a, uint32_t b, uint32_t p) {
    return (uint32_t)(((uint64_t)a * b) % p);
}

static uint32_t submod(uint32_t a, uint32_t b, uint32_t p) {
    return a >= b ? a - b : a + p - b;
}

/* Inverse of a in Z/p by the extended Euclidean algorithm; a != 0. */
static uint32_t invmod(uint32_t a, uint32_t p) {
    int64_t t = 0, newt = 1, r = p, newr = a;
    while (newr != 0) {
        int64_t q = r / newr, tmp;
        tmp = t - q * newt; t = newt; newt = tmp;
        tmp = r - q * newr; r = newr; newr = tmp;
    }
    if (t < 0) t += p;
    return (uint32_t)t;
}

/* Reduce the rows x cols block of A (leading dimension lda) mod p into W. */
static void load_mod(const int64_t *A, int64_t rows, int64_t cols, int64_t lda,
                     uint32_t p, uint32_t *W) {
    for (int64_t i = 0; i < rows; ++i)
        for (int64_t j = 0; j < cols; ++j)
            W[i * cols + j] = red64(A[i * lda + j], p);
}

/* In-place LU of the n x n residue matrix W (row-major): on return the
 * strict lower part holds L (unit diagonal implied), the upper part U, and
 * perm[i] is the original row now at position i. Returns det mod p, which is
 * 0 as soon as a column has no nonzero pivot (the factorisation stops
 * there and *stopped_at receives that column, else n). */
static uint32_t lu_inplace(uint32_t *W, int64_t n, uint32_t p, int32_t *perm,
                           int64_t *stopped_at) {
    uint32_t det = 1 % p;
    int neg = 0;
    if (perm)
        for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int64_t k = 0; k < n; ++k) {
        int64_t piv = -1;
        for (int64_t i = k; i < n; ++i)
            if (W[i * n + k] != 0) { piv = i; break; }
        if (piv < 0) {
            if (stopped_at) *stopped_at = k;
            return 0;
        }
        if (piv != k) {
            for (int64_t j = 0; j < n; ++j) {
                uint32_t t = W[k * n + j];
                W[k * n + j] = W[piv * n + j];
                W[piv * n + j] = t;
            }
            if (perm) { int32_t t = perm[k]; perm[k] = perm[piv]; perm[piv] = t; }
            neg ^= 1;
        }
        uint32_t akk = W[k * n + k];
        det = mulmod(det, akk, p);
        uint32_t inv = invmod(akk, p);
        for (int64_t i = k + 1; i < n; ++i) {
            uint32_t l = mulmod(W[i * n + k], inv, p);
            W[i * n + k] = l;
            if (l == 0) continue;
            for (int64_t j = k + 1; j < n; ++j)
                W[i * n + j] = submod(W[i * n + j], mulmod(l, W[k * n + j], p), p);
        }
    }
    if (stopped_at) *stopped_at = n;
    return neg ? (det == 0 ? 0 : p - det) : det;
}

uint32_t orc_det_mod_p(const int64_t *A, int64_t n, int64_t lda, uint32_t p) {
    if (n == 0) return 1 % p;
    uint32_t *W = (uint32_t *)malloc(sizeof(uint32_t) * n * n);
    if (!W) return 0xffffffffu;
    load_mod(A, n, n, lda, p, W);
    uint32_t d = lu_inplace(W, n, p, NULL, NULL);
    free(W);
    return d;
}

void orc_det_mod_primes(const int64_t *A, int64_t n, int64_t lda,
                        const uint32_t *primes, int32_t np, uint32_t *out,
                        int32_t nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int32_t k = 0; k < np; ++k)
        out[k] = orc_det_mod_p(A, n, lda, primes[k]);
    (void)nthreads;
}

/* LU with first-nonzero pivoting; LU receives n*n residues, perm n entries.
 * Returns det mod p; *stopped_at = n when the matrix is invertible mod p. */
uint32_t orc_lu_mod_p(const int64_t *A, int64_t n, int64_t lda, uint32_t p,
                      uint32_t *LU, int32_t *perm, int64_t *stopped_at) {
    load_mod(A, n, n, lda, p, LU);
    return lu_inplace(LU, n, p, perm, stopped_at);
}

/* Rank of a rows x cols matrix over Z/p by row echelon elimination (a column
 * without a pivot is skipped). */
int64_t orc_rank_mod_p(const int64_t *A, int64_t rows, int64_t cols,
                       int64_t lda, uint32_t p) {
    uint32_t *W = (uint32_t *)malloc(sizeof(uint32_t) * (rows * cols + 1));
    load_mod(A, rows, cols, lda, p, W);
    int64_t r = 0;
    for (int64_t k = 0; k < cols && r < rows; ++k) {
        int64_t piv = -1;
        for (int64_t i = r; i < rows; ++i)
            if (W[i * cols + k]) { piv = i; break; }
        if (piv < 0) continue;
        if (piv != r)
            for (int64_t j = 0; j < cols; ++j) {
                uint32_t t = W[r * cols + j];
                W[r * cols + j] = W[piv * cols + j];
                W[piv * cols + j] = t;
            }
        uint32_t inv = invmod(W[r * cols + k], p);
        for (int64_t i = r + 1; i < rows; ++i) {
            uint32_t l = mulmod(W[i * cols + k], inv, p);
            if (!l) continue;
            for (int64_t j = k; j < cols; ++j)
                W[i * cols + j] = submod(W[i * cols + j], mulmod(l, W[r * cols + j], p), p);
        }
        ++r;
    }
    free(W);
    return r;
}

/* A^{-1} mod p by Gauss-Jordan elimination on [A | I]; returns 0 on
 * success, 1 if A is singular mod p. inv receives n*n residues in [0, p). */
int32_t orc_inverse_mod_p(const int64_t *A, int64_t n, int64_t lda, uint32_t p,
                          uint32_t *inv) {
    int64_t w = 2 * n;
    uint32_t *W = (uint32_t *)malloc(sizeof(uint32_t) * n * w);
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < n; ++j) W[i * w + j] = red64(A[i * lda + j], p);
        for (int64_t j = 0; j < n; ++j) W[i * w + n + j] = (i == j) ? 1u % p : 0u;
    }
    for (int64_t k = 0; k < n; ++k) {
        int64_t piv = -1;
        for (int64_t i = k; i < n; ++i)
            if (W[i * w + k]) { piv = i; break; }
        if (piv < 0) { free(W); return 1; }
        if (piv != k)
            for (int64_t j = 0; j < w; ++j) {
                uint32_t t = W[k * w + j];
                W[k * w + j] = W[piv * w + j];
                W[piv * w + j] = t;
            }
        uint32_t ik = invmod(W[k * w + k], p);
        for (int64_t j = 0; j < w; ++j) W[k * w + j] = mulmod(W[k * w + j], ik, p);
        for (int64_t i = 0; i < n; ++i) {
            if (i == k) continue;
            uint32_t l = W[i * w + k];
            if (!l) continue;
            for (int64_t j = 0; j < w; ++j)
                W[i * w + j] = submod(W[i * w + j], mulmod(l, W[k * w + j], p), p);
        }
    }
    for (int64_t i = 0; i < n; ++i)
        memcpy(inv + i * n, W + i * w + n, sizeof(uint32_t) * n);
    free(W);
    return 0;
}
