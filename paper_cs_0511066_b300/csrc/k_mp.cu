// Matrices with multi-word entries (entries of hundreds of bits, e.g.
// A = U diag(1, ..., 1, d) V with a 600-bit d): entry (i, j) is given as
// sign[i][j] in {-1, 0, 1} times a magnitude of L little-endian base-2^32
// limbs mag[(i n + j) L + l].
//
//   k_mp_reduce   A mod p_k for a wave of primes (Section 2.1 needs only the
//                 residues; the LU then runs on int32 residues as usual).
//   k_mp_log2     log2 |a_ij| (double) for the Hadamard bound H.
//   k_mp_norms    log2 of the Euclidean norm of every row or column.
//   k_mp_planes   A as T planes of signed base-2^15 digits (int16):
//                 a_ij = sum_t D_t[i][j] 2^(15 t), |D_t| <= 2^14.
//   k_mp_cx /     one Dixon step (Section 2.2) with a multi-word residual:
//   k_mp_update   x = C (r mod p) mod p, then r <- (r - A x) / p, where
//                 (A x)_i = sum_t 2^(15 t) (D_t x)_i and the exact division by
//                 p runs from the lowest base-2^15 digit up with p^{-1} mod
//                 2^15 (Jebelean's exact division).
//
// Residual layout: rd[i][k], k < len, base-2^15 digits, digits 0..len-2 in
// [0, 2^15), digit len-1 signed (two's complement value of r_i).
#include <cfloat>

#include "idet_internal.cuh"

namespace idet {

namespace {

constexpr int kMT = 256;
constexpr int kMaxW = 8;  // primes per pass of k_mp_reduce

__global__ void __launch_bounds__(kMT)
k_mp_reduce(const uint32_t *__restrict__ mag, const int8_t *__restrict__ sgn, int64_t nn, int L,
            const ModP *__restrict__ mods, int W, int32_t *__restrict__ R) {
    ModP M[kMaxW];
    int32_t c32[kMaxW];
#pragma unroll
    for (int k = 0; k < kMaxW; ++k) {
        M[k] = mods[k < W ? k : 0];
        c32[k] = red_bal((int64_t)1 << 32, M[k]);
    }
    for (int64_t e = blockIdx.x * (int64_t)kMT + threadIdx.x; e < nn;
         e += (int64_t)gridDim.x * kMT) {
        const int s = sgn[e];
        int32_t r[kMaxW];
#pragma unroll
        for (int k = 0; k < kMaxW; ++k) r[k] = 0;
        if (s != 0) {
            const uint32_t *a = mag + e * L;
            for (int l = L - 1; l >= 0; --l) {
                const int64_t limb = (int64_t)__ldg(a + l);
#pragma unroll
                for (int k = 0; k < kMaxW; ++k)
                    if (k < W) r[k] = red_bal((int64_t)r[k] * c32[k] + limb, M[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < kMaxW; ++k)
            if (k < W) R[(int64_t)k * nn + e] = s < 0 ? -r[k] : r[k];
    }
}

__global__ void __launch_bounds__(kMT)
k_mp_log2(const uint32_t *__restrict__ mag, const int8_t *__restrict__ sgn, int64_t nn, int L,
          double *__restrict__ E, unsigned int *__restrict__ maxbits) {
    unsigned int mb = 0;
    for (int64_t e = blockIdx.x * (int64_t)kMT + threadIdx.x; e < nn;
         e += (int64_t)gridDim.x * kMT) {
        const uint32_t *a = mag + e * L;
        int t = L - 1;
        while (t >= 0 && a[t] == 0) --t;
        if (sgn[e] == 0 || t < 0) {
            E[e] = -INFINITY;
            continue;
        }
        const unsigned int bits = 32u * (unsigned)t + (32u - (unsigned)__clz(a[t]));
        mb = max(mb, bits);
        // |a| < (a_t + 1) 2^(32 t): an upper bound, from the top limb
        E[e] = log2((double)a[t] + 1.0) + 32.0 * t;
    }
    for (int o = 16; o; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    if ((threadIdx.x & 31) == 0) atomicMax(maxbits, mb);
}

// out[v] = log2 sqrt(sum_w 2^(2 E[v][w])) over rows (cols = 0) or columns.
__global__ void __launch_bounds__(kMT)
k_mp_norms(const double *__restrict__ E, int64_t n, int cols, double *__restrict__ out) {
    __shared__ double s_red[kMT / 32];
    const int64_t v = blockIdx.x;
    auto at = [&](int64_t w) { return cols ? E[w * n + v] : E[v * n + w]; };
    double mx = -INFINITY;
    for (int64_t w = threadIdx.x; w < n; w += kMT) mx = fmax(mx, at(w));
    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = -INFINITY;
    for (int k = 0; k < kMT / 32; ++k) mx = fmax(mx, s_red[k]);
    __syncthreads();
    if (mx == -INFINITY) {
        if (threadIdx.x == 0) out[v] = -INFINITY;
        return;
    }
    double sum = 0;
    for (int64_t w = threadIdx.x; w < n; w += kMT) {
        const double e = at(w);
        if (e != -INFINITY) sum += exp2(2.0 * (e - mx));
    }
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int k = 0; k < kMT / 32; ++k) t += s_red[k];
        out[v] = mx + 0.5 * log2(t);
    }
}

// Signed base-2^15 digits: the magnitude's digits are made balanced in
// [-2^14, 2^14) from the lowest up, then multiplied by the sign.
// planes: T x n x ldp int16 (row padding zeroed by the caller).
__global__ void __launch_bounds__(kMT)
k_mp_planes(const uint32_t *__restrict__ mag, const int8_t *__restrict__ sgn, int64_t n, int L,
            int T, int64_t ldp, int16_t *__restrict__ planes) {
    const int64_t nn = n * n;
    const int64_t plane = n * ldp;
    for (int64_t e = blockIdx.x * (int64_t)kMT + threadIdx.x; e < nn;
         e += (int64_t)gridDim.x * kMT) {
        const int64_t i = e / n, j = e - i * n;
        const int s = sgn[e];
        const uint32_t *a = mag + e * L;
        int carry = 0;
        int bitpos = 0;  // next bit of the magnitude
        for (int t = 0; t < T; ++t) {
            // 15 bits starting at bitpos
            int d = 0;
            const int l = bitpos >> 5, o = bitpos & 31;
            if (l < L) {
                uint64_t w = a[l];
                if (l + 1 < L) w |= (uint64_t)a[l + 1] << 32;
                d = (int)((w >> o) & 0x7fff);
            }
            bitpos += 15;
            d += carry;
            carry = 0;
            if (d >= (1 << 14)) {
                d -= 1 << 15;
                carry = 1;
            }
            planes[(int64_t)t * plane + i * ldp + j] = (int16_t)(s < 0 ? -d : (s > 0 ? d : 0));
        }
    }
}

__device__ __forceinline__ int64_t wsum64(int64_t v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// x = C (r mod p) mod p, one warp per row; digits[it][i] = x_i; z[it] += u.x
__global__ void __launch_bounds__(kMT)
k_mp_cx(const int32_t *__restrict__ C, int64_t ldc, int64_t n, const int32_t *__restrict__ rm,
        ModP M, const int32_t *__restrict__ u, int32_t *__restrict__ x,
        int32_t *__restrict__ digits, unsigned long long *__restrict__ z) {
    extern __shared__ int32_t s_rm[];
    __shared__ long long s_z[kMT / 32];
    for (int64_t j = threadIdx.x; j < n; j += kMT) s_rm[j] = rm[j];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * (kMT / 32) + warp;
    long long zp = 0;
    if (i < n) {
        const int32_t *c = C + i * ldc;
        int64_t lo = 0, hi = 0;
        for (int64_t j = lane; j < n; j += 32) {
            const int32_t v = s_rm[j];
            const int64_t cv = __ldg(c + j);
            lo += cv * (int64_t)(v & 0xffff);
            hi += cv * (int64_t)(v >> 16);
        }
        lo = wsum64(lo);
        hi = wsum64(hi);
        if (lane == 0) {
            const int32_t xi = red_bal((int64_t)red_bal(hi, M) * 65536 + red_bal(lo, M), M);
            x[i] = xi;
            digits[i] = xi;
            zp = (long long)u[i] * xi;
        }
    }
    if (lane == 0) s_z[warp] = zp;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int k = 0; k < kMT / 32; ++k) t += s_z[k];
        atomicAdd(z, (unsigned long long)t);
    }
}

// r_i <- (r_i - sum_t 2^(15 t) (D_t x)_i) / p and rm_i = r_i mod p; one CTA
// per row. info[0] is set if r - A x does not fit the len digits (cannot
// happen under the bounds the host sizes len with; checked anyway).
__global__ void __launch_bounds__(kMT)
k_mp_update(const int16_t *__restrict__ planes, int T, int64_t ldp, int64_t n,
            const int32_t *__restrict__ x, int32_t *__restrict__ rd, int len, ModP M,
            uint32_t pinv15, int32_t *__restrict__ rm, int32_t *__restrict__ info) {
    extern __shared__ __align__(16) unsigned char smu[];
    int32_t *sx = (int32_t *)smu;                        // n
    int64_t *S = (int64_t *)(sx + ((n + 3) & ~3ll));     // T
    int64_t *dg = S + T;                                 // len
    const int64_t i = blockIdx.x;
    for (int64_t j = threadIdx.x; j < n; j += kMT) sx[j] = x[j];
    for (int k = threadIdx.x; k < len; k += kMT) dg[k] = rd[i * len + k];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t plane = n * ldp;
    for (int t = warp; t < T; t += kMT / 32) {
        const int16_t *row = planes + (int64_t)t * plane + i * ldp;
        int64_t acc = 0;
        // ldp is a multiple of 8: 4 digits per 8-byte load
        for (int64_t j = 4 * lane; j < n; j += 128) {
            const short4 a = *(const short4 *)(row + j);
            acc += (int64_t)a.x * sx[j];
            if (j + 1 < n) acc += (int64_t)a.y * sx[j + 1];
            if (j + 2 < n) acc += (int64_t)a.z * sx[j + 2];
            if (j + 3 < n) acc += (int64_t)a.w * sx[j + 3];
        }
        acc = wsum64(acc);
        if (lane == 0) S[t] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // v = r - sum_t S_t 2^(15 t), normalised: digits < len-1 in [0, 2^15)
        int64_t carry = 0;
        for (int k = 0; k < len; ++k) {
            int64_t v = dg[k] + carry - (k < T ? S[k] : 0);
            if (k < len - 1) {
                dg[k] = v & 0x7fff;
                carry = v >> 15;  // arithmetic: floor division
            } else {
                dg[k] = v;
            }
        }
        // the host sizes len so that |r - A x| < 2^(15 (len - 1) + 14)
        if (dg[len - 1] >= (1 << 14) || dg[len - 1] < -(1 << 14)) atomicExch(info, 1);
        // exact division by p from the bottom: q_k = w p^{-1} mod 2^15
        carry = 0;
        const int64_t p = M.p;
        for (int k = 0; k < len; ++k) {
            const int64_t w = dg[k] + carry;
            const int64_t q = (int64_t)(((uint64_t)w * pinv15) & 0x7fff);
            carry = (w - q * p) >> 15;  // exact: w - q p = 0 mod 2^15
            dg[k] = q;
        }
        // q = sum q_k 2^(15 k) mod 2^(15 len): top digit as signed
        if (dg[len - 1] >= (1 << 14)) dg[len - 1] -= 1 << 15;
        int32_t h = (int32_t)dg[len - 1];
        for (int k = len - 2; k >= 0; --k) h = red_bal((int64_t)h * 32768 + dg[k], M);
        rm[i] = h;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < len; k += kMT) rd[i * len + k] = (int32_t)dg[k];
}

int grid_for(int64_t items) {
    int64_t g = (items + kMT - 1) / kMT;
    if (g > 148 * 16) g = 148 * 16;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

int launch_reduce_mp(const uint32_t *mag, const int8_t *sgn, int64_t n, int L, const ModP *mods,
                     int W, int32_t *R, cudaStream_t s) {
    const int64_t nn = n * n;
    for (int w0 = 0; w0 < W; w0 += kMaxW) {
        const int Wc = (W - w0) < kMaxW ? (W - w0) : kMaxW;
        k_mp_reduce<<<grid_for(nn), kMT, 0, s>>>(mag, sgn, nn, L, mods + w0, Wc, R + w0 * nn);
        count_launch();
        IDET_CUDA_TRY(cudaGetLastError());
    }
    return IDET_OK;
}

int launch_mp_stats(const uint32_t *mag, const int8_t *sgn, int64_t n, int L, double *E,
                    double *rowl2, double *coll2, unsigned int *maxbits, cudaStream_t s) {
    const int64_t nn = n * n;
    IDET_CUDA_TRY(cudaMemsetAsync(maxbits, 0, sizeof(unsigned int), s));
    k_mp_log2<<<grid_for(nn), kMT, 0, s>>>(mag, sgn, nn, L, E, maxbits);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    k_mp_norms<<<(unsigned)n, kMT, 0, s>>>(E, n, 0, rowl2);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    k_mp_norms<<<(unsigned)n, kMT, 0, s>>>(E, n, 1, coll2);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

int launch_mp_planes(const uint32_t *mag, const int8_t *sgn, int64_t n, int L, int T, int64_t ldp,
                     int16_t *planes, cudaStream_t s) {
    if (ldp % 8 != 0 || ldp < n) {
        set_last_error("digit planes: row length must be a multiple of 8");
        return IDET_ERR_INTERNAL;
    }
    IDET_CUDA_TRY(cudaMemsetAsync(planes, 0, sizeof(int16_t) * (size_t)T * n * ldp, s));
    k_mp_planes<<<grid_for(n * n), kMT, 0, s>>>(mag, sgn, n, L, T, ldp, planes);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

int launch_mp_step(const MpLiftArgs &a, int it, cudaStream_t s) {
    const size_t smx = sizeof(int32_t) * (size_t)a.n;
    if (smx > 200 * 1024) {
        set_last_error("multi-word lift: n too large");
        return IDET_ERR_ARG;
    }
    if (smx > 48 * 1024)
        IDET_TRY(allow_max_smem((const void *)k_mp_cx));
    k_mp_cx<<<(unsigned)((a.n + kMT / 32 - 1) / (kMT / 32)), kMT, smx, s>>>(
        a.C, a.ldc, a.n, a.rm, a.mod, a.u, a.x, a.digits + (int64_t)it * a.n,
        (unsigned long long *)(a.z + it));
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    const size_t smu = sizeof(int32_t) * (size_t)((a.n + 3) & ~3ll) + sizeof(int64_t) * (a.T + a.len);
    if (smu > 200 * 1024) {
        set_last_error("multi-word lift: n too large");
        return IDET_ERR_ARG;
    }
    if (smu > 48 * 1024)
        IDET_TRY(allow_max_smem((const void *)k_mp_update));
    k_mp_update<<<(unsigned)a.n, kMT, smu, s>>>(a.planes, a.T, a.ldp, a.n, a.x, a.rd, a.len, a.mod,
                                                a.pinv15, a.rm, a.info);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

}  // namespace idet
