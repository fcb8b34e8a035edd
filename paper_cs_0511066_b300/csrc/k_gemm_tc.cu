// Trailing update of the LU over Z/p on the tensor cores, kept exact.
//
//   C <- C - A B  mod p        (A22 <- A22 - L21 U12, Section 2.1's LU)
//
// for 21-bit primes with balanced residues |x| < 2^20 and K <= 128 (one block
// column), staged through shared memory 32 columns of K at a time.
// Three arithmetic variants, selected per call:
//
//  * I8  : every residue is split into signed 7-bit limbs,
//            x = x0 + 2^7 x1 + 2^14 x2,  x0, x1 in [-64, 63], x2 in [-64, 64],
//          and the nine limb products are accumulated exactly in int32 by
//          mma.sync m16n8k32 s8, grouped by s = i + j:
//            P_s = sum_{i+j=s} A_i B_j,  |P_s| <= 3 * 128 * 64^2 < 2^21,
//          then recombined as sum_s 2^{7s} P_s in int64 and reduced mod p.
//  * BF16: the same limbs (exact in bf16: |x_i| <= 2^8) and groups with
//          fp32 accumulation by mma.sync m16n8k16 bf16; every partial sum is an
//          integer below 2^24 in magnitude, so fp32 holds it exactly.
//  * F64 : residues as doubles, mma.sync m8n8k4 f64: |sum| <= 128 * 2^40 =
//          2^47 < 2^53, exact; one reduction per output.
//
// Tiling: 64 x 64 outputs per CTA, 8 warps as 4 (M) x 2 (N), 16 x 32 per
// warp; the K = 32 slab of A and B is converted once into limbs in shared
// memory (B stored transposed, K contiguous, so fragments are 32-bit loads).
// Batched over primes by blockIdx.z; dead primes (det = 0 mod p) skip.
#include "idet_internal.cuh"

namespace idet {

namespace {

constexpr int TBM = 64, TBN = 64, TK = 32;
constexpr int kTcThreads = 256;

__device__ __forceinline__ void split7(int32_t x, int32_t &l0, int32_t &l1, int32_t &l2) {
    l0 = ((x + 64) & 127) - 64;
    int32_t t = (x - l0) >> 7;
    l1 = ((t + 64) & 127) - 64;
    l2 = (t - l1) >> 7;
}

// ---- int8 ------------------------------------------------------------------

__device__ __forceinline__ void mma_s8(int32_t (&c)[4], const uint32_t (&a)[4],
                                       const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void mma_f64(double (&c)[2], double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(c[0]), "+d"(c[1])
                 : "d"(a), "d"(b));
}

// bf16 bit pattern of a small integer |v| <= 256 (exact).
__device__ __forceinline__ uint16_t bf16_of(int32_t v) {
    float f = (float)v;
    return (uint16_t)(__float_as_uint(f) >> 16);
}

template <int PATH>
__device__ __forceinline__ void stage_slab(unsigned char *sm, const int32_t *__restrict__ a,
                                           int64_t lda, const int32_t *__restrict__ b, int64_t ldb,
                                           int m0, int n0, int k0, int M, int N, int K, int tid) {
    __syncthreads();  // the previous slab is no longer read
    for (int e = tid; e < TBM * TK; e += kTcThreads) {
        const int r = e / TK, k = e % TK;
        const int gk = k0 + k;
        const int gm = m0 + r;
        const int32_t av = (gm < M && gk < K) ? a[(int64_t)gm * lda + gk] : 0;
        const int gn = n0 + r;  // B^T row r = column gn of B
        const int32_t bv = (gn < N && gk < K) ? b[(int64_t)gk * ldb + gn] : 0;
        if (PATH == IDET_PATH_I8) {
            int8_t *sa = (int8_t *)sm, *sb = sa + 3 * 64 * 48;
            int32_t l0, l1, l2;
            split7(av, l0, l1, l2);
            sa[(0 * 64 + r) * 48 + k] = (int8_t)l0;
            sa[(1 * 64 + r) * 48 + k] = (int8_t)l1;
            sa[(2 * 64 + r) * 48 + k] = (int8_t)l2;
            split7(bv, l0, l1, l2);
            sb[(0 * 64 + r) * 48 + k] = (int8_t)l0;
            sb[(1 * 64 + r) * 48 + k] = (int8_t)l1;
            sb[(2 * 64 + r) * 48 + k] = (int8_t)l2;
        } else if (PATH == IDET_PATH_BF16) {
            uint16_t *sa = (uint16_t *)sm, *sb = sa + 3 * 64 * 40;
            int32_t l0, l1, l2;
            split7(av, l0, l1, l2);
            sa[(0 * 64 + r) * 40 + k] = bf16_of(l0);
            sa[(1 * 64 + r) * 40 + k] = bf16_of(l1);
            sa[(2 * 64 + r) * 40 + k] = bf16_of(l2);
            split7(bv, l0, l1, l2);
            sb[(0 * 64 + r) * 40 + k] = bf16_of(l0);
            sb[(1 * 64 + r) * 40 + k] = bf16_of(l1);
            sb[(2 * 64 + r) * 40 + k] = bf16_of(l2);
        } else {
            double *sa = (double *)sm, *sb = sa + 64 * 33;
            sa[r * 33 + k] = (double)av;
            sb[r * 33 + k] = (double)bv;
        }
    }
    __syncthreads();
}

template <int PATH>
__global__ void __launch_bounds__(kTcThreads)
k_gemm_tc(const int32_t *__restrict__ A, int64_t lda, int64_t sA, const int32_t *__restrict__ B,
          int64_t ldb, int64_t sB, int32_t *__restrict__ C, int64_t ldc, int64_t sC, int M, int N,
          int K, const ModP *__restrict__ mods, const LUState *__restrict__ st) {
    // shared layout (bytes): I8: A limbs [3][64][32+16] s8, B limbs [3][64][32+16] s8
    //                        BF16: A [3][64][40] bf16, B [3][64][40] bf16
    //                        F64: A [64][33] f64, B [64][33] f64
    __shared__ __align__(16) unsigned char sm[2 * 3 * 64 * 40 * 2 > 2 * 64 * 33 * 8
                                                  ? 2 * 3 * 64 * 40 * 2
                                                  : 2 * 64 * 33 * 8];
    const int w = blockIdx.z;
    if (st && st[w].dead) return;
    const ModP Mo = mods[w];
    const int32_t *a = A + (int64_t)w * sA;
    const int32_t *b = B + (int64_t)w * sB;
    int32_t *c = C + (int64_t)w * sC;
    const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp & 3) * 16, wn = (warp >> 2) * 32;
    const int g = lane >> 2, t = lane & 3;

    // ---- products; acc[s][nt] for s = 0..4 (I8/BF16), acc[nt] (F64)
    int64_t out[4][4];  // [nt][element] exact products as int64
    if (PATH == IDET_PATH_I8) {
        const int8_t *sa = (const int8_t *)sm, *sb = sa + 3 * 64 * 48;
        int32_t acc[5][4][4];
#pragma unroll
        for (int s = 0; s < 5; ++s)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[s][nt][q] = 0;
        for (int k0 = 0; k0 < K; k0 += TK) {
        stage_slab<PATH>(sm, a, lda, b, ldb, m0, n0, k0, M, N, K, tid);
        uint32_t fa[3][4], fb[3][4][2];
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            const int8_t *base = sa + (l * 64 + wm) * 48;
            fa[l][0] = *(const uint32_t *)(base + g * 48 + 4 * t);
            fa[l][1] = *(const uint32_t *)(base + (g + 8) * 48 + 4 * t);
            fa[l][2] = *(const uint32_t *)(base + g * 48 + 16 + 4 * t);
            fa[l][3] = *(const uint32_t *)(base + (g + 8) * 48 + 16 + 4 * t);
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int8_t *bb = sb + (l * 64 + wn + nt * 8 + g) * 48;
                fb[l][nt][0] = *(const uint32_t *)(bb + 4 * t);
                fb[l][nt][1] = *(const uint32_t *)(bb + 16 + 4 * t);
            }
        }
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) mma_s8(acc[i + j][nt], fa[i], fb[j][nt]);
        }
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q)
                out[nt][q] = (int64_t)acc[0][nt][q] + ((int64_t)acc[1][nt][q] << 7) +
                             ((int64_t)acc[2][nt][q] << 14) + ((int64_t)acc[3][nt][q] << 21) +
                             ((int64_t)acc[4][nt][q] << 28);
    } else if (PATH == IDET_PATH_BF16) {
        const uint16_t *sa = (const uint16_t *)sm, *sb = sa + 3 * 64 * 40;
        float acc[5][4][4];
#pragma unroll
        for (int s = 0; s < 5; ++s)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[s][nt][q] = 0.f;
        for (int k0 = 0; k0 < K; k0 += TK) {
        stage_slab<PATH>(sm, a, lda, b, ldb, m0, n0, k0, M, N, K, tid);
#pragma unroll
        for (int kk = 0; kk < TK; kk += 16) {
            uint32_t fa[3][4], fb[3][4][2];
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                const uint16_t *base = sa + (l * 64 + wm) * 40 + kk;
                fa[l][0] = *(const uint32_t *)(base + g * 40 + 2 * t);
                fa[l][1] = *(const uint32_t *)(base + (g + 8) * 40 + 2 * t);
                fa[l][2] = *(const uint32_t *)(base + g * 40 + 8 + 2 * t);
                fa[l][3] = *(const uint32_t *)(base + (g + 8) * 40 + 8 + 2 * t);
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    const uint16_t *bb = sb + (l * 64 + wn + nt * 8 + g) * 40 + kk;
                    fb[l][nt][0] = *(const uint32_t *)(bb + 2 * t);
                    fb[l][nt][1] = *(const uint32_t *)(bb + 8 + 2 * t);
                }
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) mma_bf16(acc[i + j][nt], fa[i], fb[j][nt]);
        }
        }
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q)
                out[nt][q] = (int64_t)acc[0][nt][q] + ((int64_t)acc[1][nt][q] << 7) +
                             ((int64_t)acc[2][nt][q] << 14) + ((int64_t)acc[3][nt][q] << 21) +
                             ((int64_t)acc[4][nt][q] << 28);
    } else {
        // F64: warp tile 16 x 32 = 2 (m8) x 4 (n8) tiles of m8n8k4
        const double *sa = (const double *)sm, *sb = sa + 64 * 33;
        double acc[2][4][2];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) acc[mt][nt][0] = acc[mt][nt][1] = 0.0;
        for (int k0 = 0; k0 < K; k0 += TK) {
        stage_slab<PATH>(sm, a, lda, b, ldb, m0, n0, k0, M, N, K, tid);
#pragma unroll
        for (int kk = 0; kk < TK; kk += 4) {
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const double av = sa[(wm + mt * 8 + g) * 33 + kk + t];
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    const double bv = sb[(wn + nt * 8 + g) * 33 + kk + t];
                    mma_f64(acc[mt][nt], av, bv);
                }
            }
        }
        }
        // map to the m16n8 output convention used below: rows g (mt = 0) and
        // g + 8 (mt = 1), columns 2t, 2t + 1
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            out[nt][0] = (int64_t)acc[0][nt][0];
            out[nt][1] = (int64_t)acc[0][nt][1];
            out[nt][2] = (int64_t)acc[1][nt][0];
            out[nt][3] = (int64_t)acc[1][nt][1];
        }
    }

    // ---- epilogue: C <- C - out mod p; element q: row g + 8 (q >> 1), col 2t + (q & 1)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int gm = m0 + wm + g + 8 * (q >> 1);
            const int gn = n0 + wn + nt * 8 + 2 * t + (q & 1);
            if (gm < M && gn < N) {
                int32_t *p = c + (int64_t)gm * ldc + gn;
                *p = red_bal((int64_t)*p - red_bal(out[nt][q], Mo), Mo);
            }
        }
}

}  // namespace

int gemm_sub_tc(int path, const int32_t *A, int64_t lda, int64_t sA, const int32_t *B, int64_t ldb,
                int64_t sB, int32_t *C, int64_t ldc, int64_t sC, int M, int N, int K,
                const ModP *mods, const LUState *st, int W, cudaStream_t s) {
    if (M <= 0 || N <= 0 || K <= 0) return IDET_OK;
    if (K > 128) {
        set_last_error("tensor trailing update: K must be at most 128 (exactness bound)");
        return IDET_ERR_INTERNAL;
    }
    dim3 grid((N + TBN - 1) / TBN, (M + TBM - 1) / TBM, W);
    if (path == IDET_PATH_I8)
        k_gemm_tc<IDET_PATH_I8><<<grid, kTcThreads, 0, s>>>(A, lda, sA, B, ldb, sB, C, ldc, sC, M, N,
                                                             K, mods, st);
    else if (path == IDET_PATH_BF16)
        k_gemm_tc<IDET_PATH_BF16><<<grid, kTcThreads, 0, s>>>(A, lda, sA, B, ldb, sB, C, ldc, sC, M,
                                                               N, K, mods, st);
    else
        k_gemm_tc<IDET_PATH_F64><<<grid, kTcThreads, 0, s>>>(A, lda, sA, B, ldb, sB, C, ldc, sC, M,
                                                              N, K, mods, st);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

}  // namespace idet
