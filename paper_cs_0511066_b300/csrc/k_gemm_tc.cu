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
// warp, K in slabs of 32. A first pass (k_pack_tc) converts the residues of
// A and of B^T (K contiguous, so fragments are 32-bit loads) into the limbs
// (or doubles) of every 64-row x 32-column tile, laid out in global memory
// exactly as the tile sits in shared memory, padding included. The GEMM
// kernel then feeds its shared memory with bulk asynchronous copies (the
// copy engine, cp.async.bulk completing on an mbarrier): one copy per tile,
// a two-stage ring over the K slabs, the copy of slab k + 1 in flight while
// slab k is multiplied. Waits are bounded; a wait that gives up records an
// error (tc_check_error), drains the copies issued and ends the CTA.
// Batched over primes by blockIdx.z; dead primes (det = 0 mod p) skip.
#include "idet_internal.cuh"
#include "lift_common.cuh"

namespace idet {

namespace {

constexpr int TBM = 64, TBN = 64, TK = 32;
constexpr int kTcThreads = 256;
constexpr int kMaxK = 128;  // the LU's block-column width

// Exactness of the accumulations for K <= kMaxK terms (balanced 21-bit
// residues |x| < 2^20, 7-bit limbs |l| <= 64, at most 3 limb products per
// group): int8 groups in int32, bf16 groups in fp32 (integers below 2^24),
// FP64 sums below 2^53. The FP64 bound itself would allow
// floor((2^53 - 1) / 2^40) = 8191 terms; the LU never needs more than 128.
static_assert(3LL * kMaxK * 64 * 64 < (1LL << 31), "int8-limb groups overflow int32");
static_assert(3LL * kMaxK * 64 * 64 < (1LL << 24), "bf16-limb groups are not exact in fp32");
static_assert((double)kMaxK * (double)(1LL << 40) < (double)(1LL << 53), "fp64 sums inexact");
static_assert(((1LL << 53) - 1) / (1LL << 40) == 8191, "the FP64 delayed-reduction bound");

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

// One 64-row x 32-column tile of limbs as it sits in shared memory: I8 three
// limb planes [3][64][48] s8, BF16 [3][64][40] bf16, F64 [64][33] f64 (rows
// padded against bank conflicts). Every tile size is a multiple of 16 bytes.
template <int PATH> struct Tile;
template <> struct Tile<IDET_PATH_I8> {
    static constexpr int kBytes = 3 * 64 * 48;
};
template <> struct Tile<IDET_PATH_BF16> {
    static constexpr int kBytes = 3 * 64 * 40 * 2;
};
template <> struct Tile<IDET_PATH_F64> {
    static constexpr int kBytes = 64 * 33 * 8;
};
static_assert(Tile<IDET_PATH_I8>::kBytes % 16 == 0 && Tile<IDET_PATH_BF16>::kBytes % 16 == 0 &&
                  Tile<IDET_PATH_F64>::kBytes % 16 == 0,
              "bulk copies move multiples of 16 bytes");

// Packed tiles of one operand: tile (w, block, slab) at
// ((w * blocks + block) * slabs + slab) * kBytes. The operand is A (rows of
// A, K along a row, transpose = false) or B^T (rows are columns of B,
// transpose = true). Entries past M (or N) and K are zero.
template <int PATH>
__global__ void k_pack_tc(const int32_t *__restrict__ X, int64_t ldx, int64_t sX, int rows,
                          int K, bool transpose, int blocks, int slabs,
                          unsigned char *__restrict__ out) {
    const int w = blockIdx.z, blk = blockIdx.y, slab = blockIdx.x;
    const int32_t *x = X + (int64_t)w * sX;
    unsigned char *t = out + (((int64_t)w * blocks + blk) * slabs + slab) * Tile<PATH>::kBytes;
    for (int e = threadIdx.x; e < 64 * TK; e += blockDim.x) {
        const int r = e / TK, k = e % TK;
        const int gr = blk * 64 + r, gk = slab * TK + k;
        int32_t v = 0;
        if (gr < rows && gk < K) v = transpose ? x[(int64_t)gk * ldx + gr] : x[(int64_t)gr * ldx + gk];
        if (PATH == IDET_PATH_I8) {
            int8_t *sa = (int8_t *)t;
            int32_t l0, l1, l2;
            split7(v, l0, l1, l2);
            sa[(0 * 64 + r) * 48 + k] = (int8_t)l0;
            sa[(1 * 64 + r) * 48 + k] = (int8_t)l1;
            sa[(2 * 64 + r) * 48 + k] = (int8_t)l2;
        } else if (PATH == IDET_PATH_BF16) {
            uint16_t *sa = (uint16_t *)t;
            int32_t l0, l1, l2;
            split7(v, l0, l1, l2);
            sa[(0 * 64 + r) * 40 + k] = bf16_of(l0);
            sa[(1 * 64 + r) * 40 + k] = bf16_of(l1);
            sa[(2 * 64 + r) * 40 + k] = bf16_of(l2);
        } else {
            ((double *)t)[r * 33 + k] = (double)v;
        }
    }
    // the padding columns are never read; zero them so the buffer is defined
    if (PATH == IDET_PATH_I8)
        for (int e = threadIdx.x; e < 3 * 64 * 16; e += blockDim.x)
            ((int8_t *)t)[(e / 16) * 48 + 32 + e % 16] = 0;
    else if (PATH == IDET_PATH_BF16)
        for (int e = threadIdx.x; e < 3 * 64 * 8; e += blockDim.x)
            ((uint16_t *)t)[(e / 8) * 40 + 32 + e % 8] = 0;
    else
        for (int e = threadIdx.x; e < 64; e += blockDim.x) ((double *)t)[e * 33 + 32] = 0.0;
}

__device__ int g_tc_err;  // first bounded wait that gave up, of any CTA

// Feeds the two stages of a CTA: slab k of the CTA's A tile row and B tile
// column goes to stage k % 2 (A then B, one bulk copy each), completing on
// full[k % 2].
template <int PATH> struct Feed {
    const unsigned char *pa, *pb;  // first slab of this CTA's A / B tiles
    unsigned char *sm;             // stage s at sm + s * 2 * kBytes
    uint64_t *full;
    __device__ void issue(int k) const {
        constexpr unsigned T = Tile<PATH>::kBytes;
        unsigned char *dst = sm + (k & 1) * 2 * T;
        lift::mbar_expect_tx(&full[k & 1], 2 * T);
        lift::bulk_g2s(dst, pa + (int64_t)k * T, T, &full[k & 1], pol());
        lift::bulk_g2s(dst + T, pb + (int64_t)k * T, T, &full[k & 1], pol());
    }
    static __device__ uint64_t pol() { return lift::policy_evict_last(); }
};

// Bounded wait for stage (k % 2) of slab k; on failure the error is recorded.
__device__ __forceinline__ bool wait_stage(uint64_t *full, int k, long long limit) {
    const uint32_t addr = lift::smem_u32(&full[k & 1]);
    const unsigned parity = (unsigned)((k >> 1) & 1);
    const long long t0 = clock64();
    while (!lift::mbar_test(addr, parity)) {
        if (clock64() - t0 > limit) {
            atomicCAS(&g_tc_err, 0, 1);
            return false;
        }
    }
    return true;
}

template <int PATH>
__global__ void __launch_bounds__(kTcThreads)
k_gemm_tc(const unsigned char *__restrict__ PA, const unsigned char *__restrict__ PB, int mblocks,
          int nblocks, int slabs, int32_t *__restrict__ C, int64_t ldc, int64_t sC, int M, int N,
          int K, const ModP *__restrict__ mods, const LUState *__restrict__ st, long long limit) {
    // shared layout: two stages of (A tile, B tile), Tile<PATH>::kBytes each
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t full[2];
    __shared__ int s_fail;
    const int w = blockIdx.z;
    if (st && st[w].dead) return;
    const ModP Mo = mods[w];
    int32_t *c = C + (int64_t)w * sC;
    const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp & 3) * 16, wn = (warp >> 2) * 32;
    const int g = lane >> 2, t = lane & 3;
    constexpr int T = Tile<PATH>::kBytes;
    Feed<PATH> feed{PA + (((int64_t)w * mblocks + blockIdx.y) * slabs) * T,
                    PB + (((int64_t)w * nblocks + blockIdx.x) * slabs) * T, sm, full};
    if (tid == 0) {
        s_fail = 0;
        lift::mbar_init(&full[0], 1);
        lift::mbar_init(&full[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        feed.issue(0);
        if (slabs > 1) feed.issue(1);
    }
    __syncthreads();
    int issued = slabs > 1 ? 2 : 1;
    // slab k: wait for its stage; after the multiply, the stage is refilled
    // with slab k + 2 (all threads have left it: the barrier below)
    auto stage_in = [&](int k) -> const unsigned char * {
        if (!wait_stage(full, k, limit)) s_fail = 1;
        __syncthreads();
        return s_fail ? nullptr : sm + (k & 1) * 2 * T;
    };
    auto stage_out = [&](int k) {
        __syncthreads();
        if (tid == 0 && k + 2 < slabs) {
            feed.issue(k + 2);
            ++issued;
        }
    };

    // ---- products; acc[s][nt] for s = 0..4 (I8/BF16), acc[nt] (F64)
    int64_t out[4][4];  // [nt][element] exact products as int64
    if (PATH == IDET_PATH_I8) {
        int32_t acc[5][4][4];
#pragma unroll
        for (int s = 0; s < 5; ++s)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[s][nt][q] = 0;
        for (int k = 0; k < slabs; ++k) {
        const int8_t *sa = (const int8_t *)stage_in(k), *sb = sa + 3 * 64 * 48;
        if (!sa) break;
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
        stage_out(k);
        }
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q)
                out[nt][q] = (int64_t)acc[0][nt][q] + ((int64_t)acc[1][nt][q] << 7) +
                             ((int64_t)acc[2][nt][q] << 14) + ((int64_t)acc[3][nt][q] << 21) +
                             ((int64_t)acc[4][nt][q] << 28);
    } else if (PATH == IDET_PATH_BF16) {
        float acc[5][4][4];
#pragma unroll
        for (int s = 0; s < 5; ++s)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[s][nt][q] = 0.f;
        for (int k = 0; k < slabs; ++k) {
        const uint16_t *sa = (const uint16_t *)stage_in(k), *sb = sa + 3 * 64 * 40;
        if (!sa) break;
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
        stage_out(k);
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
        double acc[2][4][2];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) acc[mt][nt][0] = acc[mt][nt][1] = 0.0;
        for (int k = 0; k < slabs; ++k) {
        const double *sa = (const double *)stage_in(k), *sb = sa + 64 * 33;
        if (!sa) break;
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
        stage_out(k);
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

    if (s_fail) {
        // no copy may be in flight when the CTA exits: wait (default limit)
        // for the last phase of every stage used
        if (tid == 0)
            for (int k = issued - 2 < 0 ? 0 : issued - 2; k < issued; ++k) {
                const uint32_t addr = lift::smem_u32(&full[k & 1]);
                const long long t0 = clock64();
                while (!lift::mbar_test(addr, (unsigned)((k >> 1) & 1)) &&
                       clock64() - t0 <= lift::kDefaultWaitCycles) {
                }
            }
        return;
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

size_t tc_scratch_bytes(int64_t n, int W, int path) {
    const int64_t blocks = (n + 63) / 64, slabs = 4;  // K <= 128
    const int64_t T = path == IDET_PATH_I8 ? Tile<IDET_PATH_I8>::kBytes
                      : path == IDET_PATH_BF16 ? Tile<IDET_PATH_BF16>::kBytes
                                               : Tile<IDET_PATH_F64>::kBytes;
    return (size_t)(2 * W * blocks * slabs * T);
}

int tc_check_error(cudaStream_t s) {
    int e = 0;
    IDET_CUDA_TRY(cudaMemcpyFromSymbolAsync(&e, g_tc_err, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaStreamSynchronize(s));
    if (e != 0) {
        const int z = 0;
        IDET_CUDA_TRY(cudaMemcpyToSymbolAsync(g_tc_err, &z, sizeof(int), 0, cudaMemcpyHostToDevice, s));
        set_last_error("tensor trailing update: a bounded wait for a tile copy gave up");
        return IDET_ERR_TIMEOUT;
    }
    return IDET_OK;
}

template <int PATH>
static int gemm_sub_tc_t(const int32_t *A, int64_t lda, int64_t sA, const int32_t *B, int64_t ldb,
                         int64_t sB, int32_t *C, int64_t ldc, int64_t sC, int M, int N, int K,
                         const ModP *mods, const LUState *st, int W, void *scratch, cudaStream_t s) {
    const int mb = (M + 63) / 64, nbk = (N + 63) / 64, slabs = (K + TK - 1) / TK;
    constexpr int T = Tile<PATH>::kBytes;
    unsigned char *PA = (unsigned char *)scratch;
    unsigned char *PB = PA + (size_t)W * mb * slabs * T;
    k_pack_tc<PATH><<<dim3(slabs, mb, W), 256, 0, s>>>(A, lda, sA, M, K, false, mb, slabs, PA);
    k_pack_tc<PATH><<<dim3(slabs, nbk, W), 256, 0, s>>>(B, ldb, sB, N, K, true, nbk, slabs, PB);
    count_launch(2);
    const size_t smem = 2 * 2 * (size_t)T;
    IDET_TRY(allow_max_smem((const void *)k_gemm_tc<PATH>));
    k_gemm_tc<PATH><<<dim3(nbk, mb, W), kTcThreads, smem, s>>>(PA, PB, mb, nbk, slabs, C, ldc, sC,
                                                              M, N, K, mods, st,
                                                              lift_wait_cycles());
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

int gemm_sub_tc(int path, const int32_t *A, int64_t lda, int64_t sA, const int32_t *B, int64_t ldb,
                int64_t sB, int32_t *C, int64_t ldc, int64_t sC, int M, int N, int K,
                const ModP *mods, const LUState *st, int W, void *scratch, cudaStream_t s) {
    if (M <= 0 || N <= 0 || K <= 0) return IDET_OK;
    if (K > kMaxK) {
        set_last_error("tensor trailing update: K must be at most 128 (exactness bound)");
        return IDET_ERR_INTERNAL;
    }
    if (path == IDET_PATH_I8)
        return gemm_sub_tc_t<IDET_PATH_I8>(A, lda, sA, B, ldb, sB, C, ldc, sC, M, N, K, mods, st,
                                           W, scratch, s);
    if (path == IDET_PATH_BF16)
        return gemm_sub_tc_t<IDET_PATH_BF16>(A, lda, sA, B, ldb, sB, C, ldc, sC, M, N, K, mods, st,
                                             W, scratch, s);
    return gemm_sub_tc_t<IDET_PATH_F64>(A, lda, sA, B, ldb, sB, C, ldc, sC, M, N, K, mods, st, W,
                                        scratch, s);
}

}  // namespace idet
