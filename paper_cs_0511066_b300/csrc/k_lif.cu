// Exact lcm of the denominators of x = A^{-1} b (Section 2.2: s~_n is the
// lcm of the denominators of the rational solution).
//
// The lift gives X_j = x_j mod p^m for every entry j (base-p digits, balanced).
// A candidate common denominator D (from the reconstruction of a random
// projection u . x) divides the lcm. D is the lcm exactly when every D x_j is
// an integer, i.e. when y_j = D X_j mod p^m is a small number (|y_j| below the
// numerator bound p^h): by uniqueness of rational reconstruction, the
// unique fraction with numerator < p^h and denominator <= D that is congruent
// to X_j must then be y_j / D. k_lif_check computes y_j for all entries at
// once (one CTA per entry: base-p convolution of D's digits with X_j's
// digits, truncated at m, then carry normalisation) and flags the entries
// whose y_j is not small. For a flagged entry the host reconstructs x_j
// itself (denominator d_j) and replaces D by lcm(D, d_j) = d_j (D / g),
// D / g being the cofactor that the extended Euclidean algorithm on (D, d_j)
// produces at its zero remainder (k_ratrecon with a given first operand);
// k_mul_radix forms the product.
#include "idet_internal.cuh"

namespace idet {

namespace {

constexpr int kLT = 256;

__device__ __forceinline__ int64_t floor_div(int64_t v, int64_t p) {
    int64_t q = v / p;
    if ((v % p) < 0) --q;
    return q;
}

// One CTA per entry j. digits: m x n balanced int32 (row i = digit vector
// x_i). D: dlen base-p digits in [0, p). Writes flag[j] = 1 when
// y_j = D X_j mod p^m has a digit >= h that is neither all-zero (a small
// positive y_j) nor all (p-1) (a small negative y_j). When yout is not null
// (and j == only), the normalised digits of y_j are written there.
__global__ void __launch_bounds__(kLT)
k_lif_check(const int32_t *__restrict__ digits, int64_t n, int m, const uint32_t *__restrict__ D,
            int dlen, uint32_t p, int h, int32_t *__restrict__ flag, int64_t only,
            int64_t *__restrict__ yout) {
    extern __shared__ int64_t lsm[];
    const int64_t j = only >= 0 ? only : (int64_t)blockIdx.x;
    int32_t *x = (int32_t *)lsm;                     // m digits of X_j
    int32_t *dh = x + m, *dl = dh + dlen;            // D digits split in 16-bit halves
    int64_t *sh = (int64_t *)(((uintptr_t)(dl + dlen) + 15) & ~(uintptr_t)15);
    int64_t *sl = sh + kLT;
    __shared__ int64_t s_carry;
    __shared__ int s_zero, s_max;
    for (int i = threadIdx.x; i < m; i += kLT) x[i] = digits[(int64_t)i * n + j];
    for (int i = threadIdx.x; i < dlen; i += kLT) {
        dh[i] = (int32_t)(D[i] >> 16);
        dl[i] = (int32_t)(D[i] & 0xffff);
    }
    if (threadIdx.x == 0) {
        s_carry = 0;
        s_zero = 1;
        s_max = 1;
    }
    __syncthreads();
    for (int c0 = 0; c0 < m; c0 += kLT) {
        const int c = c0 + threadIdx.x;
        int64_t ah = 0, al = 0;
        if (c < m) {
            const int alo = c - (m - 1) > 0 ? c - (m - 1) : 0;
            const int ahi = c < dlen - 1 ? c : dlen - 1;
            for (int a = alo; a <= ahi; ++a) {
                const int64_t xv = x[c - a];
                ah += (int64_t)dh[a] * xv;
                al += (int64_t)dl[a] * xv;
            }
        }
        sh[threadIdx.x] = ah;
        sl[threadIdx.x] = al;
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t carry = s_carry;
            const int lim = (m - c0) < kLT ? (m - c0) : kLT;
            int zero = s_zero, mx = s_max;
            for (int k = 0; k < lim; ++k) {
                // v = sh * 2^16 + sl + carry, |v| < 2^75: split the division
                const int64_t q1 = floor_div(sh[k], p);
                const int64_t r1 = sh[k] - q1 * (int64_t)p;
                const int64_t v2 = r1 * 65536 + sl[k] + carry;
                const int64_t q2 = floor_div(v2, p);
                const int64_t dig = v2 - q2 * (int64_t)p;
                carry = q1 * 65536 + q2;
                const int pos = c0 + k;
                if (yout) yout[pos] = dig;
                if (pos >= h) {
                    if (dig != 0) zero = 0;
                    if (dig != (int64_t)p - 1) mx = 0;
                }
            }
            s_carry = carry;
            s_zero = zero;
            s_max = mx;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && only < 0) flag[j] = (s_zero || s_max) ? 0 : 1;
}

// out = a * b (base-p digit vectors), single CTA: convolution + carries.
__global__ void __launch_bounds__(kLT)
k_mul_radix(const uint32_t *__restrict__ a, int la, const uint32_t *__restrict__ b, int lb,
            uint32_t p, uint32_t *__restrict__ out, int cap, int32_t *__restrict__ out_len) {
    __shared__ int64_t sh[kLT], sl[kLT];
    __shared__ int64_t s_carry;
    const int L = la + lb;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int c0 = 0; c0 < L && c0 < cap; c0 += kLT) {
        const int c = c0 + threadIdx.x;
        int64_t ah = 0, al = 0;
        if (c < L) {
            const int alo = c - (lb - 1) > 0 ? c - (lb - 1) : 0;
            const int ahi = c < la - 1 ? c : la - 1;
            for (int i = alo; i <= ahi; ++i) {
                const int64_t bv = b[c - i];
                ah += (int64_t)(a[i] >> 16) * bv;
                al += (int64_t)(a[i] & 0xffff) * bv;
            }
        }
        sh[threadIdx.x] = ah;
        sl[threadIdx.x] = al;
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t carry = s_carry;
            const int lim = min(kLT, min(L, cap) - c0);
            for (int k = 0; k < lim; ++k) {
                const int64_t q1 = floor_div(sh[k], p);
                const int64_t r1 = sh[k] - q1 * (int64_t)p;
                const int64_t v2 = r1 * 65536 + sl[k] + carry;
                const int64_t q2 = floor_div(v2, p);
                out[c0 + k] = (uint32_t)(v2 - q2 * (int64_t)p);
                carry = q1 * 65536 + q2;
            }
            s_carry = carry;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int l = min(L, cap);
        while (l > 0 && out[l - 1] == 0) --l;
        *out_len = l;
    }
}

// z[i] = digits[i][j] (column j of the lifting digits), as int64.
__global__ void k_gather_col(const int32_t *__restrict__ digits, int64_t n, int m, int64_t j,
                             int64_t *__restrict__ z) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) z[i] = digits[(int64_t)i * n + j];
}

size_t check_smem(int m, int dlen) {
    return sizeof(int32_t) * ((size_t)m + 2 * (size_t)dlen) + 16 + 2 * sizeof(int64_t) * kLT;
}

}  // namespace

int launch_lif_check(const int32_t *digits, int64_t n, int m, const uint32_t *D, int dlen,
                     uint32_t p, int h, int32_t *flag, cudaStream_t s) {
    const size_t smem = check_smem(m, dlen);
    if (smem > 200 * 1024) {
        set_last_error("largest invariant factor: lift too long for the per-entry check");
        return IDET_ERR_ARG;
    }
    IDET_TRY(allow_max_smem((const void *)k_lif_check));
    k_lif_check<<<(unsigned)n, kLT, smem, s>>>(digits, n, m, D, dlen, p, h, flag, -1, nullptr);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

int launch_lif_entry(const int32_t *digits, int64_t n, int m, const uint32_t *D, int dlen,
                     uint32_t p, int64_t j, int64_t *yout, cudaStream_t s) {
    const size_t smem = check_smem(m, dlen);
    IDET_TRY(allow_max_smem((const void *)k_lif_check));
    k_lif_check<<<1, kLT, smem, s>>>(digits, n, m, D, dlen, p, m, nullptr, j, yout);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

int launch_gather_col(const int32_t *digits, int64_t n, int m, int64_t j, int64_t *z,
                      cudaStream_t s) {
    k_gather_col<<<(m + kLT - 1) / kLT, kLT, 0, s>>>(digits, n, m, j, z);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

int launch_mul_radix(const uint32_t *a, int la, const uint32_t *b, int lb, uint32_t p,
                     uint32_t *out, int cap, int32_t *out_len, cudaStream_t s) {
    k_mul_radix<<<1, kLT, 0, s>>>(a, la, b, lb, p, out, cap, out_len);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

}  // namespace idet
