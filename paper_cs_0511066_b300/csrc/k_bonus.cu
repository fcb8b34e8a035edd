// The extended bonus of Section 3.2: from k solutions X = A^{-1} B (their
// p-adic digits), their common denominator s~ and a random k x n matrix R,
//     pi~_k = s~^k / gcd(det(R N), s~^k),   N = s~ X,
// a factor of the product of the k largest invariant factors of A.
//
// Everything runs in radix p on the p-adic digits of the lift (k = 2 here,
// the number of solves Alg. 4.1 makes with i_max = 2):
//  * (R X)_{kl} = sum_i p^i (R_k . x_{i,l}): the projections of every digit
//    vector on the rows of R, exact in 128-bit arithmetic (k_proj_rx), then
//    carried into radix-p digits modulo p^m (k_sums_to_radix);
//  * det(R X) mod p^m by radix-p products (k_mul_radix) and a subtraction;
//  * det(R N) = s~^k det(R X) mod p^m; the lift is long enough that
//    p^m > 2 |det(R N)|, so its balanced representative is det(R N) itself;
//  * pi~_k = s~^k / gcd(s~^k, |det(R N)|), the cofactor that the extended
//    Euclidean algorithm on (s~^k, |det(R N)|) leaves at its zero remainder
//    (k_ratrecon with a given first operand).
#include <vector>

#include "idet_internal.cuh"

namespace idet {

namespace {

constexpr int kBT = 256;

__device__ __forceinline__ __int128 warp_sum128(__int128 v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const uint64_t lo = __shfl_xor_sync(0xffffffffu, (unsigned long long)(uint64_t)v, o);
        const int64_t hi = __shfl_xor_sync(0xffffffffu, (long long)(int64_t)(v >> 64), o);
        v += (__int128)(((unsigned __int128)(uint64_t)hi << 64) | lo);
    }
    return v;
}

// zz[t][k][l] = sum_j R[k][j] x_{t,l}[j] for the digit vectors of the K
// right-hand sides (dig: [l][t][j], m x n each), one CTA per digit index t.
// |R| < 2^62 and |x| < 2^30: each product is below 2^92 and the n-term sum
// below 2^108.
template <int K>
__global__ void __launch_bounds__(kBT)
k_proj_rx(const int32_t *__restrict__ dig, int64_t n, int m, const int64_t *__restrict__ R,
          __int128 *__restrict__ zz) {
    __shared__ __int128 part[kBT / 32][K * K];
    const int t = blockIdx.x;
    __int128 acc[K][K];
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int l = 0; l < K; ++l) acc[k][l] = 0;
    for (int64_t j = threadIdx.x; j < n; j += kBT) {
        int64_t r[K];
#pragma unroll
        for (int k = 0; k < K; ++k) r[k] = R[k * n + j];
#pragma unroll
        for (int l = 0; l < K; ++l) {
            const int64_t x = dig[((int64_t)l * m + t) * n + j];
#pragma unroll
            for (int k = 0; k < K; ++k) acc[k][l] += (__int128)r[k] * x;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int l = 0; l < K; ++l) {
            const __int128 v = warp_sum128(acc[k][l]);
            if (lane == 0) part[warp][k * K + l] = v;
        }
    __syncthreads();
    if (threadIdx.x < K * K) {
        __int128 v = 0;
        for (int w = 0; w < kBT / 32; ++w) v += part[w][threadIdx.x];
        zz[(int64_t)t * K * K + threadIdx.x] = v;
    }
}

// Non-negative representative of v mod p for |v| < 2^126 (r64 = 2^64 mod p).
__device__ __forceinline__ uint32_t mod128(__int128 v, const ModP &M, uint64_t r64) {
    const int64_t hi = (int64_t)(v >> 64);
    const uint64_t lo = (uint64_t)v;
    uint64_t r = lo - __umul64hi(lo, M.m) * (uint64_t)M.p;
    if (r >= M.p) r -= M.p;
    if (r >= M.p) r -= M.p;
    return red_pos((int64_t)red_bal(hi, M) * (int64_t)r64 + (int64_t)r, M);
}

// out = (sum_t zz[t * stride] p^t) mod p^m as m digits in [0, p): one
// thread, the carry divided exactly by p through p^{-1} mod 2^128.
__global__ void k_sums_to_radix(const __int128 *__restrict__ zz, int stride, int m, ModP M,
                                uint64_t r64, uint64_t pinv_lo, uint64_t pinv_hi,
                                uint32_t *__restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const unsigned __int128 pinv = ((unsigned __int128)pinv_hi << 64) | pinv_lo;
    __int128 carry = 0;
    for (int t = 0; t < m; ++t) {
        const __int128 v = zz[(int64_t)t * stride] + carry;
        const uint32_t d = mod128(v, M, r64);
        out[t] = d;
        carry = (__int128)((unsigned __int128)(v - (__int128)d) * pinv);
    }
}

// out = (x - y) mod p^m (m digits each, in [0, p)).
__global__ void k_radix_sub(const uint32_t *__restrict__ x, const uint32_t *__restrict__ y, int m,
                            uint32_t p, uint32_t *__restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t borrow = 0;
    for (int t = 0; t < m; ++t) {
        int64_t v = (int64_t)x[t] - (int64_t)y[t] - borrow;
        borrow = v < 0;
        out[t] = (uint32_t)(v < 0 ? v + p : v);
    }
}

// v (m digits in [0, p)) taken in the balanced range (-p^m/2, p^m/2): out =
// |v| as digits, info[0] = its length, info[1] = 1 when negative.
__global__ void k_radix_abs(const uint32_t *__restrict__ v, int m, uint32_t p,
                            uint32_t *__restrict__ out, int32_t *__restrict__ info) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const uint32_t h = (p - 1) / 2;  // (p^m - 1)/2 has every digit h
    int neg = 0;
    for (int t = m - 1; t >= 0; --t)
        if (v[t] != h) {
            neg = v[t] > h;
            break;
        }
    if (neg) {  // p^m - v = (p^m - 1 - v) + 1
        uint32_t carry = 1;
        for (int t = 0; t < m; ++t) {
            uint32_t d = (p - 1 - v[t]) + carry;
            carry = d >= p;
            out[t] = carry ? d - p : d;
        }
    } else {
        for (int t = 0; t < m; ++t) out[t] = v[t];
    }
    int len = m;
    while (len > 0 && out[len - 1] == 0) --len;
    info[0] = len;
    info[1] = neg;
}

__global__ void k_digits_to_i64(const uint32_t *__restrict__ d, int len, int64_t *__restrict__ z) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) z[i] = d[i];
}

unsigned __int128 inv_mod_2_128(uint64_t p) {
    unsigned __int128 x = p;  // p * p = 1 mod 8
    for (int i = 0; i < 7; ++i) x *= 2 - (unsigned __int128)p * x;
    return x;
}

}  // namespace

int lcm_radix(const uint32_t *a, int la, const uint32_t *b, int lb, uint32_t p, Workspace &ws,
              uint32_t **out, int *lout) {
    cudaStream_t s = ws.stream();
    const int cap = la + lb + 4;
    uint32_t *cof = nullptr, *res = nullptr;
    int64_t *zb = nullptr;
    int32_t *info = nullptr, *len = nullptr;
    IDET_TRY(ws.alloc_n(&cof, cap));
    IDET_TRY(ws.alloc_n(&res, cap));
    IDET_TRY(ws.alloc_n(&zb, lb + 1));
    IDET_TRY(ws.alloc_n(&info, 4));
    IDET_TRY(ws.alloc_n(&len, 1));
    k_digits_to_i64<<<(lb + kBT - 1) / kBT + 1, kBT, 0, s>>>(b, lb, zb);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    // a / gcd(a, b): the cofactor of b at the zero remainder of Euclid (a, b)
    IDET_TRY(launch_ratrecon(zb, lb, p, 0, cap, cof, cap, info, ws, a, la));
    int32_t hi[2] = {0, 0};
    IDET_CUDA_TRY(cudaMemcpyAsync(hi, info, 8, cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaStreamSynchronize(s));
    if (hi[0] != 0) {
        set_last_error("lcm of radix-p numbers: gcd failed (code %d)", hi[0]);
        return IDET_ERR_INTERNAL;
    }
    IDET_TRY(launch_mul_radix(b, lb, cof, hi[1], p, res, cap, len, s));
    int32_t hl = 0;
    IDET_CUDA_TRY(cudaMemcpyAsync(&hl, len, 4, cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaStreamSynchronize(s));
    *out = res;
    *lout = hl;
    return IDET_OK;
}

int bonus_pi2(const int32_t *dig, int64_t n, int m, uint32_t p, const int64_t *R,
              const uint32_t *sdig, int slen, Workspace &ws, uint32_t **pi, int *plen) {
    cudaStream_t s = ws.stream();
    const ModP M = make_mod(p);
    const unsigned __int128 pinv = inv_mod_2_128(p);
    const uint64_t r64 = (uint64_t)(((unsigned __int128)1 << 64) % p);
    __int128 *zz = nullptr;
    uint32_t *rx = nullptr, *t1 = nullptr, *t2 = nullptr, *dt = nullptr, *s2 = nullptr,
             *drn = nullptr, *ab = nullptr, *cof = nullptr;
    int32_t *len = nullptr, *info = nullptr;
    int64_t *zd = nullptr;
    const int cap2 = 2 * slen + 4, capc = cap2 + 4;
    IDET_TRY(ws.alloc_n(&zz, (size_t)m * 4));
    IDET_TRY(ws.alloc_n(&rx, 4 * (size_t)m));
    IDET_TRY(ws.alloc_n(&t1, m));
    IDET_TRY(ws.alloc_n(&t2, m));
    IDET_TRY(ws.alloc_n(&dt, m));
    IDET_TRY(ws.alloc_n(&s2, cap2));
    IDET_TRY(ws.alloc_n(&drn, m));
    IDET_TRY(ws.alloc_n(&ab, m));
    IDET_TRY(ws.alloc_n(&cof, capc));
    IDET_TRY(ws.alloc_n(&zd, m));
    IDET_TRY(ws.alloc_n(&len, 1));
    IDET_TRY(ws.alloc_n(&info, 4));
    k_proj_rx<2><<<(unsigned)m, kBT, 0, s>>>(dig, n, m, R, zz);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    for (int q = 0; q < 4; ++q) {  // (R X)_{kl}, q = 2 k + l
        k_sums_to_radix<<<1, 1, 0, s>>>(zz + q, 4, m, M, r64, (uint64_t)pinv,
                                        (uint64_t)(pinv >> 64), rx + (size_t)q * m);
        count_launch();
        IDET_CUDA_TRY(cudaGetLastError());
    }
    // det(R X) = (RX)_00 (RX)_11 - (RX)_01 (RX)_10 mod p^m
    IDET_TRY(launch_mul_radix(rx, m, rx + 3 * (size_t)m, m, p, t1, m, len, s));
    IDET_TRY(launch_mul_radix(rx + (size_t)m, m, rx + 2 * (size_t)m, m, p, t2, m, len, s));
    k_radix_sub<<<1, 1, 0, s>>>(t1, t2, m, p, dt);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    // det(R N) = s~^2 det(R X) mod p^m, balanced
    IDET_TRY(launch_mul_radix(sdig, slen, sdig, slen, p, s2, cap2, len, s));
    int32_t l2 = 0;
    IDET_CUDA_TRY(cudaMemcpyAsync(&l2, len, 4, cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaStreamSynchronize(s));
    IDET_TRY(launch_mul_radix(dt, m, s2, l2, p, drn, m, len, s));
    k_radix_abs<<<1, 1, 0, s>>>(drn, m, p, ab, info);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    int32_t hi[2] = {0, 0};
    IDET_CUDA_TRY(cudaMemcpyAsync(hi, info, 8, cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaStreamSynchronize(s));
    const int la = hi[0];
    if (la == 0) {  // det(R N) = 0: gcd = s~^2, pi~ = 1
        uint32_t one = 1;
        IDET_CUDA_TRY(cudaMemcpyAsync(cof, &one, 4, cudaMemcpyHostToDevice, s));
        IDET_CUDA_TRY(cudaStreamSynchronize(s));
        *pi = cof;
        *plen = 1;
        return IDET_OK;
    }
    k_digits_to_i64<<<(la + kBT - 1) / kBT, kBT, 0, s>>>(ab, la, zd);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    IDET_TRY(launch_ratrecon(zd, la, p, 0, capc, cof, capc, info, ws, s2, l2));
    IDET_CUDA_TRY(cudaMemcpyAsync(hi, info, 8, cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaStreamSynchronize(s));
    if (hi[0] != 0) {
        set_last_error("extended bonus: gcd with s~^2 failed (code %d)", hi[0]);
        return IDET_ERR_INTERNAL;
    }
    *pi = cof;
    *plen = hi[1];
    return IDET_OK;
}

}  // namespace idet
