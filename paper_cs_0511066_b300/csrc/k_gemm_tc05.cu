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
// k_pack_limbs writes A (M x K, row-major residues) as a bf16 limb matrix of
// K' = 3 Kp columns (Kp = K rounded up to 16, limb-major blocks of Kp), and
// B^T (N x K) with its three limbs stacked as rows (limb l's rows l kTN ..),
// already in the tcgen05 K-major no-swizzle core-matrix layout of one CTA
// tile: core matrices of 8 rows x 8 elements (128 bytes) with the row groups
// of a tile adjacent (stride 128 B, the descriptor's stride offset) and the K
// groups ROWS/8 core matrices apart (the leading offset). A tile is then one
// contiguous block that k_gemm_tc05 fetches with cp.async.bulk into shared
// memory.
//
// k_gemm_tc05: persistent, one CTA per SM looping over 128 x 48 output
// tiles (all primes' tiles in one launch). Warp-specialised:
//   warp 0 (one thread): producer, cp.async.bulk of 16-wide K chunks of the
//     three limbs of A and B into a ring of shared-memory stages, each
//     tracked by a full (transaction bytes) and an empty mbarrier;
//   warp 1 (one thread): MMA issuer into five tensor-memory accumulators of
//     48 columns (one per group, adjacent), with B's three limbs stacked as
//     144 rows: an MMA of A_a against limbs b0 .. b1 of B (128 x 48 (b1 - b0
//     + 1) x 16, bf16 in, fp32 out) lands exactly on groups a + b0 .. a + b1.
//     The first chunk of a tile takes 5 MMAs (each group started by exactly
//     one of them), the later chunks 3 (A_a against all of B) instead of one
//     per limb pair, 9: the issue rate of the single issuing thread (about
//     100 cycles per MMA), not the tensor pipe, bounds this kernel;
//     tcgen05.commit frees the stage, and after the last chunk of a tile
//     signals its accumulator set full; two sets alternate between tiles;
//     warp 1 also owns the tensor-memory allocation (512 columns);
//   warps 2-9 and 10-17: two epilogue groups of 8 warps, one per accumulator
//     set; each warp prefetches its 32 rows x 24 columns of C while the MMAs
//     run, reads its 32-lane quarter (warp id mod 4) of those columns of the
//     accumulators with tcgen05.ld, recombines in int64, reduces mod p and
//     writes C (16-byte accesses where aligned), then releases the set to the
//     issuer. (One set of 8 warps for five limbs.)
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
    static constexpr int kEpiWarps = 8;  // per accumulator set: 4 lane quarters x 2 column halves
    static constexpr int kThreads = 64 + 32 * kEpiWarps * kBufs;
    static constexpr uint32_t kStageBytes = L * (kLimbA + kLimbB);
    static constexpr int kStages = L == 3 ? 9 : 6;
    // C staging: one 128-row tile per accumulator set, rows padded to 52
    // words (16-byte accesses of a warp's 32 rows then fall in distinct banks)
    static constexpr int kCS = 52;
    static constexpr uint32_t kCBytes = kTM * kCS * 4;
    static constexpr size_t kSmem = (size_t)kStages * kStageBytes + (size_t)kBufs * kCBytes;
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

// One thread per row and group of eight k of each operand tile, for every
// prime (z): the eight residues of a group are split into limbs and each
// limb's eight bf16 values (16 contiguous bytes of one core-matrix row) are
// stored at once. A: rows m of A (M x K at lda), consecutive threads along a
// row; B: columns n of B (K x N at ldb), stored as rows of B^T, consecutive
// threads along n (coalesced loads of each k). Rows >= M (N) and k >= K are
// zero.
template <int L>
__global__ void k_pack_limbs(const int32_t *__restrict__ A, int64_t lda, int64_t sA,
                             const int32_t *__restrict__ B, int64_t ldb, int64_t sB, int M, int N,
                             int K, int Kp, int Mt, int Nt, __nv_bfloat16 *__restrict__ Apk,
                             __nv_bfloat16 *__restrict__ Bpk) {
    const int w = blockIdx.z;
    const int Kq = L * Kp, G = Kp / 8;
    const int64_t atile = (int64_t)kTM * Kq, btile = (int64_t)kTN * Kq;
    const int arows = Mt * kTM, brows = Nt * kTN;
    const int na = arows * G, total = na + brows * G;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        int32_t x[8];
        __nv_bfloat16 *dst[L];
        if (e < na) {
            const int m = e / G, k0 = 8 * (e - m * G);
            const int32_t *src = A + (int64_t)w * sA + (int64_t)m * lda + k0;
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = (m < M && k0 + i < K) ? src[i] : 0;
            __nv_bfloat16 *base = Apk + ((int64_t)w * Mt + m / kTM) * atile;
#pragma unroll
            for (int l = 0; l < L; ++l) dst[l] = base + core_off<kTM>(m % kTM, l * Kp + k0);
        } else {
            const int e2 = e - na, g = e2 / brows, nn = e2 - g * brows, k0 = 8 * g;
            const int32_t *src = B + (int64_t)w * sB + (int64_t)k0 * ldb + nn;
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = (nn < N && k0 + i < K) ? src[(int64_t)i * ldb] : 0;
            __nv_bfloat16 *base = Bpk + ((int64_t)w * Nt + nn / kTN) * btile;
#pragma unroll
            for (int l = 0; l < L; ++l) dst[l] = base + core_off<L * kTN>(l * kTN + nn % kTN, k0);
        }
        __align__(16) __nv_bfloat16 v[L][8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            int32_t li[L];
            split7<L>(x[i], li);
#pragma unroll
            for (int l = 0; l < L; ++l) v[l][i] = __int2bfloat16_rn(li[l]);
        }
#pragma unroll
        for (int l = 0; l < L; ++l)
            *reinterpret_cast<uint4 *>(dst[l]) = *reinterpret_cast<const uint4 *>(v[l]);
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
constexpr uint32_t idesc_n(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(kTM >> 4) << 24);
}
constexpr uint32_t kIdesc = idesc_n(kTN);

__device__ __forceinline__ void mbar_arrive(uint64_t *m) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa(m)) : "memory");
}

constexpr int kMaxWs = 64;  // primes whose state and reduction constants are cached in shared memory

// The epilogue's reduction of C - sum_g 2^(7g) P_g mod p in Montgomery form
// (R = 2^32): with weights w_g = 2^(7g) R mod p (balanced), t = sum_g w_g P_g
// is one multiply-add per group (|t| < 9 2^30 2^22 < 2^56), and
// v = (t - q p) / 2^32 with q = t p^{-1} mod 2^32 equals sum_g 2^(7g) P_g
// mod p with |v| <= 2^24 + p/2; C - v then needs one step either way into
// the balanced range. (Against two 64-bit Barrett reductions per entry.)
struct EpiMont {
    int32_t p, half;
    uint32_t pinv;  // p^{-1} mod 2^32
    int32_t w[9];
};

__device__ __forceinline__ EpiMont make_epi_mont(uint32_t p) {
    EpiMont e;
    e.p = (int32_t)p;
    e.half = (int32_t)((p - 1) / 2);
    uint32_t x = p;  // p p = 1 mod 8; each step doubles the correct bits
    for (int i = 0; i < 4; ++i) x *= 2u - p * x;
    e.pinv = x;
    int64_t r = (int64_t)((1ull << 32) % p);
    for (int g = 0; g < 9; ++g) {
        e.w[g] = (int32_t)(r > e.half ? r - p : r);
        r = (r * 128) % p;
    }
    return e;
}

template <int L>
struct Tc05Shared {
    uint64_t full[Tc<L>::kStages], empty[Tc<L>::kStages], acc_full[2], acc_empty[2], drain;
    uint32_t taddr;
    volatile int abort;
    int prod_iter, mma_iter;
    int dead[kMaxWs];
    EpiMont mont[kMaxWs];
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
    // tile t = (w Mt + mt) Nt + nt, in 32-bit arithmetic (W Mt Nt < 2^31)
    const int MN = Mt * Nt, tiles = W * MN;
    for (int i = tid; i < W && i < kMaxWs; i += blockDim.x) {
        S.dead[i] = st[i].dead;
        S.mont[i] = make_epi_mont(mods[i].p);
    }
    auto dead_of = [&](int w) { return w < kMaxWs ? S.dead[w] != 0 : st[w].dead != 0; };
    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&S.full[i], 1);
            mbar_init(&S.empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&S.acc_full[i], 1);
            mbar_init(&S.acc_empty[i], Tc<L>::kEpiWarps);
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
            for (int t = blockIdx.x; t < tiles && !S.abort; t += gridDim.x) {
                const int w = t / MN, rem = t - w * MN;
                const int mt = rem / Nt, nt = rem - mt * Nt;
                if (dead_of(w)) continue;
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
                    }
                    // B: the L limbs' rows stacked (L kTN rows), both K groups
                    // of the chunk in one copy
                    bulk_g2s(dst + L * kLimbA, gB + (size_t)(c * kKc / 8) * (L * kTN / 8) * 128,
                             L * kLimbB, &S.full[stg]);
                    S.prod_iter = it + 1;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            int it = 0, tile = 0;
            const uint32_t lboA = (kTM / 8) * 128, lboB = (L * kTN / 8) * 128;
            for (int t = blockIdx.x; t < tiles && !S.abort; t += gridDim.x) {
                const int w = t / MN;
                if (dead_of(w)) continue;
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
                    // one descriptor per operand and stage; the limbs' start
                    // addresses (>> 4 in the low field, no carry: shared
                    // memory is below 256 KB) are constant offsets from it
                    const uint32_t a0 = sa(sm + (size_t)stg * kStageBytes);
                    const uint64_t dA = smem_desc(a0, lboA, 128);
                    const uint64_t dB = smem_desc(a0 + L * kLimbA, lboB, 128);
                    if (c == 0) {
                        // first chunk of the tile: A_0 against all of B starts
                        // groups 0 .. L-1; then for each later limb a, A_a B_(L-1)
                        // starts group a + L - 1 and A_a against limbs 0 .. L-2
                        // adds into the groups already started: 2L - 1 MMAs
                        mma_bf16(dacc, dA, dB, idesc_n(L * kTN), 0u);
#pragma unroll
                        for (int a = 1; a < L; ++a) {
                            mma_bf16(dacc + (uint32_t)((a + L - 1) * kTN),
                                     dA + (uint64_t)((a * kLimbA) >> 4),
                                     dB + (uint64_t)((L - 1) * (kTN / 8) * 128 >> 4), kIdesc, 0u);
                            mma_bf16(dacc + (uint32_t)(a * kTN), dA + (uint64_t)((a * kLimbA) >> 4),
                                     dB, idesc_n((L - 1) * kTN), 1u);
                        }
                    } else {
                        // later chunks: A_a against the stacked limbs of B
                        // (L kTN columns) adds A_a B_b into group a + b for
                        // every b at once: L MMAs instead of L^2
#pragma unroll
                        for (int a = 0; a < L; ++a)
                            mma_bf16(dacc + (uint32_t)(a * kTN), dA + (uint64_t)((a * kLimbA) >> 4),
                                     dB, idesc_n(L * kTN), 1u);
                    }
                    mma_commit(&S.empty[stg]);
                    S.mma_iter = it + 1;
                }
                if (S.abort) break;
                mma_commit(&S.acc_full[buf]);
                ++tile;
            }
        }
    } else {  // epilogue: warps 2..9 (set 0), 10..17 (set 1 when two sets)
        // Each warp reads the accumulator lanes of its quarter (warp id mod 4:
        // the rows it may access) and one half of the 48 columns, so that 8
        // warps per set keep the conversions and reductions in flight. The
        // C entries of a tile are fetched into shared memory (cp.async) while
        // the set's previous tile is reduced, so their latency is hidden.
        constexpr int kHalf = kTN / 2, kCS = Tc<L>::kCS;
        const int e = warp - 2, grp = e / Tc<L>::kEpiWarps, q = warp & 3;
        const int h = (e % Tc<L>::kEpiWarps) / 4;
        const bool vec = (ldc % 4 == 0) && (sC % 4 == 0) && (((uintptr_t)C & 15) == 0);
        int32_t *cst = reinterpret_cast<int32_t *>(sm + (size_t)kStages * kStageBytes +
                                                   (size_t)grp * Tc<L>::kCBytes) +
                       (q * 32 + lane) * kCS + h * kHalf;
        // the next tile of this set from index u on; c counts the CTA's live
        // tiles (both sets), as the issuer does
        auto advance = [&](int u, int &c) -> int {
            for (; u < tiles; u += gridDim.x) {
                const int wu = u / MN;
                if (dead_of(wu)) continue;
                const int b = c % kBufs;
                ++c;
                if (b == grp) return u;
            }
            return tiles;
        };
        // where this thread's 24 entries of tile u live, and whether they
        // are fetched asynchronously (full 16-byte aligned row segments)
        auto locate = [&](int u, int32_t *&crow, bool &rowok, bool &full, int &cb) {
            const int w = u / MN, rem = u - w * MN;
            const int mt = rem / Nt, nt = rem - mt * Nt;
            const int r = mt * kTM + q * 32 + lane;
            cb = nt * kTN + h * kHalf;
            crow = C + (int64_t)w * sC + (int64_t)r * ldc + cb;
            rowok = r < M;
            full = vec && cb + kHalf <= N;
        };
        auto prefetch = [&](int u) {
            int32_t *crow;
            bool rowok, full;
            int cb;
            locate(u, crow, rowok, full, cb);
            if (!(rowok && full)) return;
#pragma unroll
            for (int v = 0; v < kHalf / 4; ++v)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa(cst + 4 * v)),
                             "l"(crow + 4 * v)
                             : "memory");
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        int cnt = 0;
        int t = advance(blockIdx.x, cnt);
        if (t < tiles) prefetch(t);
        while (t < tiles) {
            int cnext = cnt;
            const int tn = advance(t + gridDim.x, cnext);
            const int w = t / MN;
            const int buf = grp;
            const uint32_t use = (uint32_t)((cnt - 1) / kBufs) & 1u;
            int32_t *crow;
            bool rowok, full;
            int cb;
            locate(t, crow, rowok, full, cb);
            int32_t cv[kHalf];
            if (rowok && full) {
                asm volatile("cp.async.wait_all;" ::: "memory");
#pragma unroll
                for (int v = 0; v < kHalf / 4; ++v) {
                    const int4 x = *(const int4 *)(cst + 4 * v);
                    cv[4 * v] = x.x;
                    cv[4 * v + 1] = x.y;
                    cv[4 * v + 2] = x.z;
                    cv[4 * v + 3] = x.w;
                }
            } else {
#pragma unroll
                for (int j = 0; j < kHalf; ++j) cv[j] = (rowok && cb + j < N) ? crow[j] : 0;
            }
            const bool ok = mbar_wait_sleep(&S.acc_full[buf], use);
            if (__any_sync(0xffffffffu, !ok || S.abort)) {
                if (lane == 0 && !ok) fail(4);
                asm volatile("cp.async.wait_all;" ::: "memory");
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const EpiMont em = w < kMaxWs ? S.mont[w] : make_epi_mont(mods[w].p);
            const uint32_t tl = taddr + (uint32_t)(buf * kAccCols + h * kHalf) +
                                ((uint32_t)(q * 32) << 16);
#pragma unroll
            for (int c0 = 0; c0 < kHalf; c0 += 8) {
                uint32_t rv[kGroups][8];
#pragma unroll
                for (int g = 0; g < kGroups; ++g)
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                        : "=r"(rv[g][0]), "=r"(rv[g][1]), "=r"(rv[g][2]), "=r"(rv[g][3]),
                          "=r"(rv[g][4]), "=r"(rv[g][5]), "=r"(rv[g][6]), "=r"(rv[g][7])
                        : "r"(tl + (uint32_t)(g * kTN + c0)));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    // Each P_g is an integer below 2^22 in magnitude: adding
                    // 1.5 2^23 puts it in the low mantissa bits exactly (one
                    // full-rate add instead of a conversion instruction).
                    int64_t tsum = 0;
#pragma unroll
                    for (int g = 0; g < kGroups; ++g) {
                        const float f = __fadd_rn(__uint_as_float(rv[g][j]), 12582912.0f);
                        const int32_t v = (int32_t)__float_as_uint(f) - 0x4B400000;
                        tsum += (int64_t)em.w[g] * v;
                    }
                    const int32_t qm = (int32_t)((uint32_t)tsum * em.pinv);
                    const int32_t v = (int32_t)(tsum >> 32) - __mulhi(qm, em.p);
                    int64_t x = (int64_t)cv[c0 + j] - v;
                    if (x > em.half) x -= em.p;
                    if (x < -em.half) x += em.p;
                    cv[c0 + j] = (int32_t)x;
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.acc_empty[buf]);
            // the staging slot was consumed above: fetch the set's next tile
            if (tn < tiles) prefetch(tn);
            if (rowok && full) {
#pragma unroll
                for (int v = 0; v < kHalf / 4; ++v)
                    *(int4 *)(crow + 4 * v) =
                        make_int4(cv[4 * v], cv[4 * v + 1], cv[4 * v + 2], cv[4 * v + 3]);
            } else if (rowok) {
#pragma unroll
                for (int j = 0; j < kHalf; ++j)
                    if (cb + j < N) crow[j] = cv[j];
            }
            t = tn;
            cnt = cnext;
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
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
    const int64_t total = ((int64_t)Mt * kTM + (int64_t)Nt * kTN) * (Kp / 8);
    int pg = (int)std::min<int64_t>((total + 255) / 256, 148 * 8);
    k_pack_limbs<L><<<dim3(pg, 1, W), 256, 0, s>>>(A, lda, sA, B, ldb, sB, M, N, K, Kp, Mt, Nt,
                                                    Apk, Bpk);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    const size_t smem = Tc<L>::kSmem;
    IDET_TRY(allow_max_smem((const void *)k_gemm_tc05<L>));
    const int64_t tiles = (int64_t)W * Mt * Nt;
    int dev = 0, sms = 148;
    IDET_CUDA_TRY(cudaGetDevice(&dev));
    IDET_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // a CTA per SM, but none on SMs that a concurrent kernel of this thread
    // holds (a persistent CTA waiting for such an SM would hold up its tiles)
    const int grid = (int)std::min<int64_t>(tiles, std::max(1, sms - t_reserve_sms));
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
