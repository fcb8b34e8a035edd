// Trailing update of the LU over Z/p on the fifth-generation tensor cores
// (tcgen05), kept exact:
//
//   C <- C - A B  mod p        (A22 <- A22 - L21 U12, Section 2.1's LU)
//
// for 21-bit primes, balanced residues |x| < 2^20, K <= 128. Every residue
// is split into three signed 7-bit limbs, x = x0 + 2^7 x1 + 2^14 x2 with
// |x_i| <= 64 (exact in bf16). The nine limb products A_a B_b are grouped by
// shift g = a + b into five accumulators
//
//   P_g = sum_{a+b=g} A_a B_b,   |P_g| <= 3 * 128 * 64^2 < 2^21,
//
// each an fp32 sum of integer products below 2^24 in magnitude, hence exact;
// C - sum_g 2^(7g) P_g is then formed in int64 and reduced mod p.
//
// k_pack_limbs writes A (M x K, row-major residues) and B^T (N x K) as bf16
// limb matrices of K' = 3 Kp columns (Kp = K rounded up to 16, limb-major
// blocks of Kp), already in the tcgen05 K-major no-swizzle core-matrix
// layout of one CTA tile: core matrices of 8 rows x 8 elements (128 bytes)
// with the row groups of a tile adjacent (stride 128 B, the descriptor's
// stride offset) and the K groups ROWS/8 core matrices apart (the leading
// offset). A tile is then one contiguous block that k_gemm_tc05 fetches with
// cp.async.bulk into shared memory.
//
// k_gemm_tc05: persistent, one CTA per SM looping over 128 x 48 output
// tiles (all primes' tiles in one launch). Warp-specialised:
//   warp 0 (one thread): producer, cp.async.bulk of 16-wide K chunks of the
//     three limbs of A and B into a ring of shared-memory stages, each
//     tracked by a full (transaction bytes) and an empty mbarrier;
//   warp 1 (one thread): MMA issuer, 9 tcgen05.mma (128 x 48 x 16, bf16 in,
//     fp32 out) per stage into five tensor-memory accumulators of 48
//     columns (one per group); tcgen05.commit frees the stage, and after the
//     last chunk of a tile signals its accumulator set full; two sets
//     alternate between tiles; warp 1 also owns the tensor-memory
//     allocation (512 columns);
//   warps 2-5 and 6-9: two epilogue groups, one per accumulator set; each
//     warp prefetches its 32 rows of C while the MMAs run, reads its 32-lane
//     quarter of the accumulators with tcgen05.ld, recombines in int64,
//     reduces mod p and writes C (16-byte accesses where aligned), then
//     releases the set to the issuer.
// The epilogue of a tile overlaps the loads and MMAs of the next one. Every wait is bounded (about 2 s); a wait that gives up records an
// error and raises a block-wide abort flag, after which every role leaves
// its loop; bulk copies and MMAs already started are drained (bounded)
// before the tensor memory is freed.
#include "idet_internal.cuh"

#include <cuda_bf16.h>

namespace idet {

namespace {

constexpr int kTM = 128, kTN = 48;
constexpr int kTmemCols = 512;
constexpr int kKc = 16;         // K of one stage
constexpr uint32_t kLimbA = kTM * kKc * 2, kLimbB = kTN * kKc * 2;  // bytes per limb chunk

// L limbs per residue: 3 for 21-bit primes (5 groups, two accumulator sets
// of 5 x 48 columns), 5 for 31-bit primes (9 groups of 48 columns: one set).
template <int L>
struct Tc {
    static constexpr int kGroups = 2 * L - 1;
    static constexpr int kBufs = L == 3 ? 2 : 1;
    static constexpr int kAccCols = L == 3 ? 256 : 512;
    static constexpr int kThreads = 64 + 128 * kBufs;
    static constexpr uint32_t kStageBytes = L * (kLimbA + kLimbB);
    static constexpr int kStages = L == 3 ? 12 : 7;
};

__device__ int g_tc05_err;  // first error code (1 load, 2 MMA) of any CTA

__device__ __forceinline__ uint32_t sa(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// x = sum_{l<L} x_l 2^(7 l), x_l in [-64, 63] for l < L-1 and |x_{L-1}| <= 64
// (|x| < 2^20 for L = 3, |x| < 2^30 for L = 5).
template <int L>
__device__ __forceinline__ void split7(int32_t x, int32_t (&l)[L]) {
#pragma unroll
    for (int i = 0; i < L - 1; ++i) {
        l[i] = ((x + 64) & 127) - 64;
        x = (x - l[i]) >> 7;
    }
    l[L - 1] = x;
}

// Element (r, k') of a ROWS x K' tile in the core-matrix layout.
template <int ROWS>
__device__ __forceinline__ int64_t core_off(int r, int k) {
    return ((int64_t)((k >> 3) * (ROWS / 8) + (r >> 3)) * 8 + (r & 7)) * 8 + (k & 7);
}

// One thread per (row, k) of each operand tile, for every prime (z).
// A: rows m of A (M x K at lda); B: columns n of B (K x N at ldb), stored as
// rows of B^T. Rows >= M (N) and k >= K are zero.
template <int L>
__global__ void k_pack_limbs(const int32_t *__restrict__ A, int64_t lda, int64_t sA,
                             const int32_t *__restrict__ B, int64_t ldb, int64_t sB, int M, int N,
                             int K, int Kp, int Mt, int Nt, __nv_bfloat16 *__restrict__ Apk,
                             __nv_bfloat16 *__restrict__ Bpk) {
    const int w = blockIdx.z;
    const int Kq = L * Kp;
    const int64_t atile = (int64_t)kTM * Kq, btile = (int64_t)kTN * Kq;
    const int64_t arows = (int64_t)Mt * kTM, total = (arows + (int64_t)Nt * kTN) * Kp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = e / Kp;
        const int k = (int)(e - row * Kp);
        int32_t x = 0;
        int32_t l[L];
        if (row < arows) {
            const int m = (int)row;
            if (m < M && k < K) x = A[(int64_t)w * sA + (int64_t)m * lda + k];
            const int mt = m / kTM, r = m % kTM;
            __nv_bfloat16 *dst = Apk + ((int64_t)w * Mt + mt) * atile;
            split7<L>(x, l);
#pragma unroll
            for (int i = 0; i < L; ++i) dst[core_off<kTM>(r, i * Kp + k)] = __int2bfloat16_rn(l[i]);
        } else {
            const int n = (int)(row - arows);
            if (n < N && k < K) x = B[(int64_t)w * sB + (int64_t)k * ldb + n];
            const int nt = n / kTN, r = n % kTN;
            __nv_bfloat16 *dst = Bpk + ((int64_t)w * Nt + nt) * btile;
            split7<L>(x, l);
#pragma unroll
            for (int i = 0; i < L; ++i) dst[core_off<kTN>(r, i * Kp + k)] = __int2bfloat16_rn(l[i]);
        }
    }
}

// ---- PTX wrappers ------------------------------------------------------------

__device__ __forceinline__ void mbar_init(uint64_t *m, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(m)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *m, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(m)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *m, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(sa(m)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false after about 2 s (clock64 at up to 2.1 GHz).
__device__ __forceinline__ bool mbar_wait(uint64_t *m, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try(m, parity))
        if (clock64() - t0 > 4000000000ll) return false;
    return true;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *m) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            sa(dst)),
        "l"(src), "r"(bytes), "r"(sa(m))
        : "memory");
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    // start address, leading and stride byte offsets (all >> 4), descriptor
    // version 1 (bits 46-47), no swizzle (bits 61-63 = 0), base offset 0
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *m) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     sa(m))
                 : "memory");
}

// Instruction descriptor, kind::f16: fp32 accumulator (bits 4-5 = 1), A and
// B bf16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTN >> 3) << 17) |
                            ((uint32_t)(kTM >> 4) << 24);

__device__ __forceinline__ void mbar_arrive(uint64_t *m) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa(m)) : "memory");
}

template <int L>
struct Tc05Shared {
    uint64_t full[Tc<L>::kStages], empty[Tc<L>::kStages], acc_full[2], acc_empty[2], drain;
    uint32_t taddr;
    volatile int abort;
    int prod_iter, mma_iter;
};

// Bounded wait with back-off, for warps that wait through whole tiles.
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t *m, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try(m, parity)) {
        __nanosleep(64);
        if (clock64() - t0 > 4000000000ll) return false;
    }
    return true;
}

template <int L>
__global__ void __launch_bounds__(Tc<L>::kThreads, 1)
k_gemm_tc05(const __nv_bfloat16 *__restrict__ Apk, const __nv_bfloat16 *__restrict__ Bpk, int Kp,
            int Mt, int Nt, int W, int32_t *__restrict__ C, int64_t ldc, int64_t sC, int M, int N,
            const ModP *__restrict__ mods, const LUState *__restrict__ st) {
    constexpr int kGroups = Tc<L>::kGroups, kBufs = Tc<L>::kBufs, kAccCols = Tc<L>::kAccCols;
    constexpr int kStages = Tc<L>::kStages;
    constexpr uint32_t kStageBytes = Tc<L>::kStageBytes;
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ Tc05Shared<L> S;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Kq = L * Kp, nck = Kp / kKc;
    const int64_t tiles = (int64_t)W * Mt * Nt;
    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&S.full[i], 1);
            mbar_init(&S.empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&S.acc_full[i], 1);
            mbar_init(&S.acc_empty[i], 4);
        }
        mbar_init(&S.drain, 1);
        S.abort = 0;
        S.prod_iter = 0;
        S.mma_iter = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         sa(&S.taddr)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = S.taddr;
    auto fail = [&](int code) {
        atomicCAS(&g_tc05_err, 0, code);
        S.abort = 1;
    };
    if (warp == 0) {
        if (lane == 0) {  // producer
            int it = 0;
            for (int64_t t = blockIdx.x; t < tiles && !S.abort; t += gridDim.x) {
                const int w = (int)(t / ((int64_t)Mt * Nt));
                const int mt = (int)((t / Nt) % Mt), nt = (int)(t % Nt);
                if (st[w].dead) continue;
                const unsigned char *gA =
                    (const unsigned char *)(Apk + ((int64_t)w * Mt + mt) * ((int64_t)kTM * Kq));
                const unsigned char *gB =
                    (const unsigned char *)(Bpk + ((int64_t)w * Nt + nt) * ((int64_t)kTN * Kq));
                for (int c = 0; c < nck; ++c, ++it) {
                    const int stg = it % kStages;
                    const uint32_t ph = (uint32_t)(it / kStages) & 1u;
                    if (!mbar_wait(&S.empty[stg], ph ^ 1u)) {
                        fail(1);
                        break;
                    }
                    unsigned char *dst = sm + (size_t)stg * kStageBytes;
                    mbar_expect_tx(&S.full[stg], kStageBytes);
                    for (int l = 0; l < L; ++l) {
                        const int kb = (l * Kp + c * kKc) / 8;
                        bulk_g2s(dst + l * kLimbA, gA + (size_t)kb * (kTM / 8) * 128, kLimbA,
                                 &S.full[stg]);
                        bulk_g2s(dst + L * kLimbA + l * kLimbB, gB + (size_t)kb * (kTN / 8) * 128,
                                 kLimbB, &S.full[stg]);
                    }
                    S.prod_iter = it + 1;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            int it = 0, tile = 0;
            const uint32_t lboA = (kTM / 8) * 128, lboB = (kTN / 8) * 128;
            for (int64_t t = blockIdx.x; t < tiles && !S.abort; t += gridDim.x) {
                const int w = (int)(t / ((int64_t)Mt * Nt));
                if (st[w].dead) continue;
                const int buf = tile % kBufs;
                if (!mbar_wait(&S.acc_empty[buf], ((uint32_t)(tile / kBufs) & 1u) ^ 1u)) {
                    fail(2);
                    break;
                }
                const uint32_t dacc = taddr + (uint32_t)(buf * kAccCols);
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                for (int c = 0; c < nck; ++c, ++it) {
                    const int stg = it % kStages;
                    const uint32_t ph = (uint32_t)(it / kStages) & 1u;
                    if (!mbar_wait(&S.full[stg], ph)) {
                        fail(3);
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a0 = sa(sm + (size_t)stg * kStageBytes);
                    const uint32_t b0 = a0 + L * kLimbA;
                    for (int g = 0; g < kGroups; ++g) {
                        uint32_t acc = c > 0 ? 1u : 0u;
                        for (int a = (g > L - 1 ? g - (L - 1) : 0); a <= (g < L - 1 ? g : L - 1); ++a) {
                            const int b = g - a;
                            const uint64_t ad = smem_desc(a0 + a * kLimbA, lboA, 128);
                            const uint64_t bd = smem_desc(b0 + b * kLimbB, lboB, 128);
                            mma_bf16(dacc + (uint32_t)(g * kTN), ad, bd, kIdesc, acc);
                            acc = 1u;
                        }
                    }
                    mma_commit(&S.empty[stg]);
                    S.mma_iter = it + 1;
                }
                if (S.abort) break;
                mma_commit(&S.acc_full[buf]);
                ++tile;
            }
        }
    } else {  // epilogue groups: warps 2-5 (set 0), 6-9 (set 1 when two sets)
        const int grp = (warp - 2) >> 2, q = warp & 3;
        const bool vec = (ldc % 4 == 0) && (sC % 4 == 0) && (((uintptr_t)C & 15) == 0);
        int tile = 0;
        for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
            const int w = (int)(t / ((int64_t)Mt * Nt));
            const int mt = (int)((t / Nt) % Mt), nt = (int)(t % Nt);
            if (st[w].dead) continue;
            const int buf = tile % kBufs;
            const uint32_t use = (uint32_t)(tile / kBufs) & 1u;
            ++tile;
            if (buf != grp) continue;
            const int r = mt * kTM + q * 32 + lane;
            const int cb = nt * kTN;
            int32_t *crow = C + (int64_t)w * sC + (int64_t)r * ldc + cb;
            const bool rowok = r < M;
            const bool full = vec && cb + kTN <= N;
            // prefetch this thread's 48 entries of C while the MMAs run
            int32_t cv[kTN];
            if (rowok && full) {
#pragma unroll
                for (int u = 0; u < kTN / 4; ++u) {
                    const int4 x = *(const int4 *)(crow + 4 * u);
                    cv[4 * u] = x.x;
                    cv[4 * u + 1] = x.y;
                    cv[4 * u + 2] = x.z;
                    cv[4 * u + 3] = x.w;
                }
            } else {
#pragma unroll
                for (int j = 0; j < kTN; ++j) cv[j] = (rowok && cb + j < N) ? crow[j] : 0;
            }
            const bool ok = mbar_wait_sleep(&S.acc_full[buf], use);
            if (__any_sync(0xffffffffu, !ok || S.abort)) {
                if (lane == 0 && !ok) fail(4);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const ModP Md = mods[w];
            const uint32_t tl = taddr + (uint32_t)(buf * kAccCols) + ((uint32_t)(q * 32) << 16);
#pragma unroll
            for (int c0 = 0; c0 < kTN; c0 += 16) {
                uint32_t rv[kGroups][16];
#pragma unroll
                for (int g = 0; g < kGroups; ++g)
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,"
                        "%10,%11,%12,%13,%14,%15}, [%16];\n"
                        : "=r"(rv[g][0]), "=r"(rv[g][1]), "=r"(rv[g][2]), "=r"(rv[g][3]),
                          "=r"(rv[g][4]), "=r"(rv[g][5]), "=r"(rv[g][6]), "=r"(rv[g][7]),
                          "=r"(rv[g][8]), "=r"(rv[g][9]), "=r"(rv[g][10]), "=r"(rv[g][11]),
                          "=r"(rv[g][12]), "=r"(rv[g][13]), "=r"(rv[g][14]), "=r"(rv[g][15])
                        : "r"(tl + (uint32_t)(g * kTN + c0)));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    // sum_g 2^(7g) P_g: groups 0..3 (< 2^43) and, reduced first,
                    // groups 4.. (< 2^50) times 2^28
                    int64_t lo = 0, hi = 0;
#pragma unroll
                    for (int g = kGroups - 1; g >= 0; --g) {
                        const int64_t v = (int64_t)(int32_t)__float2int_rn(__uint_as_float(rv[g][j]));
                        if (g >= 4) hi = hi * 128 + v;
                        else lo = lo * 128 + v;
                    }
                    const int64_t s = L == 3 ? lo + hi * (1ll << 28)
                                             : (int64_t)red_bal(hi, Md) * (1ll << 28) + lo;
                    cv[c0 + j] = red_bal((int64_t)cv[c0 + j] - s, Md);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.acc_empty[buf]);
            if (rowok && full) {
#pragma unroll
                for (int u = 0; u < kTN / 4; ++u)
                    *(int4 *)(crow + 4 * u) =
                        make_int4(cv[4 * u], cv[4 * u + 1], cv[4 * u + 2], cv[4 * u + 3]);
            } else if (rowok) {
#pragma unroll
                for (int j = 0; j < kTN; ++j)
                    if (cb + j < N) crow[j] = cv[j];
            }
        }
    }
    __syncthreads();
    if (S.abort && tid == 32) {
        // drain: every MMA this thread issued, then every armed bulk copy
        mma_commit(&S.drain);
        mbar_wait(&S.drain, 0);
        for (int i = S.mma_iter; i < S.prod_iter; ++i)
            mbar_wait(&S.full[i % kStages], (uint32_t)(i / kStages) & 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                     "r"(kTmemCols)
                     : "memory");
}

}  // namespace

size_t tc05_scratch_bytes(int64_t n, int W, int L) {
    const int64_t Mt = (n + kTM - 1) / kTM, Nt = (n + kTN - 1) / kTN;
    return (size_t)W * 2 * L * 128 * (size_t)(Mt * kTM + Nt * kTN) + 1024;
}

template <int L>
static int gemm_tc05_l(const int32_t *A, int64_t lda, int64_t sA, const int32_t *B, int64_t ldb,
                       int64_t sB, int32_t *C, int64_t ldc, int64_t sC, int M, int N, int K,
                       const ModP *mods, const LUState *st, int W, void *scratch, cudaStream_t s) {
    const int Kp = (K + 15) / 16 * 16;
    const int Mt = (M + kTM - 1) / kTM, Nt = (N + kTN - 1) / kTN;
    __nv_bfloat16 *Apk = (__nv_bfloat16 *)scratch;
    __nv_bfloat16 *Bpk = Apk + (size_t)W * Mt * kTM * L * Kp;
    const int64_t total = ((int64_t)Mt * kTM + (int64_t)Nt * kTN) * Kp;
    int pg = (int)std::min<int64_t>((total + 255) / 256, 148 * 8);
    k_pack_limbs<L><<<dim3(pg, 1, W), 256, 0, s>>>(A, lda, sA, B, ldb, sB, M, N, K, Kp, Mt, Nt,
                                                    Apk, Bpk);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    const size_t smem = (size_t)Tc<L>::kStages * Tc<L>::kStageBytes;
    IDET_TRY(allow_max_smem((const void *)k_gemm_tc05<L>));
    const int64_t tiles = (int64_t)W * Mt * Nt;
    const int grid = (int)std::min<int64_t>(tiles, 148);
    k_gemm_tc05<L><<<grid, Tc<L>::kThreads, smem, s>>>(Apk, Bpk, Kp, Mt, Nt, W, C, ldc, sC, M, N,
                                                       mods, st);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

int gemm_sub_tc05(const int32_t *A, int64_t lda, int64_t sA, const int32_t *B, int64_t ldb,
                  int64_t sB, int32_t *C, int64_t ldc, int64_t sC, int M, int N, int K,
                  const ModP *mods, const LUState *st, int W, void *scratch, cudaStream_t s,
                  int L) {
    if (M <= 0 || N <= 0 || K <= 0) return IDET_OK;
    if (K > 128) {
        set_last_error("tcgen05 trailing update: K must be at most 128 (exactness bound)");
        return IDET_ERR_INTERNAL;
    }
    if (L == 5) return gemm_tc05_l<5>(A, lda, sA, B, ldb, sB, C, ldc, sC, M, N, K, mods, st, W, scratch, s);
    return gemm_tc05_l<3>(A, lda, sA, B, ldb, sB, C, ldc, sC, M, N, K, mods, st, W, scratch, s);
}

int tc05_check_error(cudaStream_t s) {
    int e = 0;
    IDET_CUDA_TRY(cudaMemcpyFromSymbolAsync(&e, g_tc05_err, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaStreamSynchronize(s));
    if (e != 0) {
        const int z = 0;
        IDET_CUDA_TRY(cudaMemcpyToSymbolAsync(g_tc05_err, &z, sizeof(int), 0, cudaMemcpyHostToDevice, s));
        set_last_error("tcgen05 trailing update: a bounded wait gave up (code %d)", e);
        return IDET_ERR_TIMEOUT;
    }
    return IDET_OK;
}

}  // namespace idet
