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
// k_gemm_tc05: one CTA (128 threads) per 128 x 64 output tile and prime.
// Thread 0 issues the bulk copies and the 9 (Kp/16) MMAs (128 x 64 x 16,
// bf16 in, fp32 accumulate in tensor memory, one 64-column accumulator per
// group); completion is tracked by tcgen05.commit on an mbarrier; each warp
// then reads its 32 lanes (rows) of the five accumulators with tcgen05.ld,
// recombines and writes C. All waits are bounded (about 2 s): on a timeout
// the CTA records an error, lets its copies and MMAs drain (bounded too),
// frees its tensor memory and returns.
#include "idet_internal.cuh"

#include <cuda_bf16.h>

namespace idet {

namespace {

constexpr int kTM = 128, kTN = 64;
constexpr int kGroups = 5;
constexpr int kTmemCols = 512;  // 5 x 64 = 320 used (allocation: a power of two)
constexpr int kT05Threads = 128;

__device__ int g_tc05_err;  // first error code (1 load, 2 MMA) of any CTA

__device__ __forceinline__ uint32_t sa(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void split7(int32_t x, int32_t &l0, int32_t &l1, int32_t &l2) {
    l0 = ((x + 64) & 127) - 64;
    const int32_t t = (x - l0) >> 7;
    l1 = ((t + 64) & 127) - 64;
    l2 = (t - l1) >> 7;
}

// Element (r, k') of a ROWS x K' tile in the core-matrix layout.
template <int ROWS>
__device__ __forceinline__ int64_t core_off(int r, int k) {
    return ((int64_t)((k >> 3) * (ROWS / 8) + (r >> 3)) * 8 + (r & 7)) * 8 + (k & 7);
}

// One thread per (row, k) of each operand tile, for every prime (z).
// A: rows m of A (M x K at lda); B: columns n of B (K x N at ldb), stored as
// rows of B^T. Rows >= M (N) and k >= K are zero.
__global__ void k_pack_limbs(const int32_t *__restrict__ A, int64_t lda, int64_t sA,
                             const int32_t *__restrict__ B, int64_t ldb, int64_t sB, int M, int N,
                             int K, int Kp, int Mt, int Nt, __nv_bfloat16 *__restrict__ Apk,
                             __nv_bfloat16 *__restrict__ Bpk) {
    const int w = blockIdx.z;
    const int Kq = 3 * Kp;
    const int64_t atile = (int64_t)kTM * Kq, btile = (int64_t)kTN * Kq;
    const int64_t arows = (int64_t)Mt * kTM, total = (arows + (int64_t)Nt * kTN) * Kp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = e / Kp;
        const int k = (int)(e - row * Kp);
        int32_t x = 0;
        __nv_bfloat16 *dst;
        int64_t o0, o1, o2;
        if (row < arows) {
            const int m = (int)row;
            if (m < M && k < K) x = A[(int64_t)w * sA + (int64_t)m * lda + k];
            const int mt = m / kTM, r = m % kTM;
            dst = Apk + ((int64_t)w * Mt + mt) * atile;
            o0 = core_off<kTM>(r, k);
            o1 = core_off<kTM>(r, Kp + k);
            o2 = core_off<kTM>(r, 2 * Kp + k);
        } else {
            const int n = (int)(row - arows);
            if (n < N && k < K) x = B[(int64_t)w * sB + (int64_t)k * ldb + n];
            const int nt = n / kTN, r = n % kTN;
            dst = Bpk + ((int64_t)w * Nt + nt) * btile;
            o0 = core_off<kTN>(r, k);
            o1 = core_off<kTN>(r, Kp + k);
            o2 = core_off<kTN>(r, 2 * Kp + k);
        }
        int32_t l0, l1, l2;
        split7(x, l0, l1, l2);
        dst[o0] = __int2bfloat16_rn(l0);
        dst[o1] = __int2bfloat16_rn(l1);
        dst[o2] = __int2bfloat16_rn(l2);
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

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
        "%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Instruction descriptor, kind::f16: fp32 accumulator (bits 4-5 = 1), A and
// B bf16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTN >> 3) << 17) |
                            ((uint32_t)(kTM >> 4) << 24);

__global__ void __launch_bounds__(kT05Threads, 1)
k_gemm_tc05(const __nv_bfloat16 *__restrict__ Apk, const __nv_bfloat16 *__restrict__ Bpk, int Kp,
            int Mt, int Nt, int32_t *__restrict__ C, int64_t ldc, int64_t sC, int M, int N,
            const ModP *__restrict__ mods, const LUState *__restrict__ st) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar_load, bar_mma;
    __shared__ uint32_t s_taddr;
    const int w = blockIdx.z, nt = blockIdx.x, mt = blockIdx.y;
    if (st[w].dead) return;  // det = 0 mod p: nothing more to update
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Kq = 3 * Kp;
    const uint32_t abytes = (uint32_t)kTM * Kq * 2, bbytes = (uint32_t)kTN * Kq * 2;
    unsigned char *sA = sm, *sB = sm + abytes;
    if (tid == 0) {
        mbar_init(&bar_load, 1);
        mbar_init(&bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         sa(&s_taddr)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = s_taddr;
    const unsigned char *gA = (const unsigned char *)(Apk + ((int64_t)w * Mt + mt) * ((int64_t)kTM * Kq));
    const unsigned char *gB = (const unsigned char *)(Bpk + ((int64_t)w * Nt + nt) * ((int64_t)kTN * Kq));
    if (tid == 0) {
        mbar_expect_tx(&bar_load, abytes + bbytes);
        for (uint32_t o = 0; o < abytes; o += 32768)
            bulk_g2s(sA + o, gA + o, min(32768u, abytes - o), &bar_load);
        for (uint32_t o = 0; o < bbytes; o += 32768)
            bulk_g2s(sB + o, gB + o, min(32768u, bbytes - o), &bar_load);
    }
    // the error decisions are made block-uniform, so that no thread frees
    // the tensor memory while MMAs another thread issued are in flight
    int err = __syncthreads_or(!mbar_wait(&bar_load, 0)) ? 1 : 0;
    if (tid == 0 && !err) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = sa(sA), b0 = sa(sB);
        const uint32_t lboA = (kTM / 8) * 128, lboB = (kTN / 8) * 128;
        for (int g = 0; g < kGroups; ++g) {
            uint32_t acc = 0;
            for (int a = (g > 2 ? g - 2 : 0); a <= (g < 2 ? g : 2); ++a) {
                const int b = g - a;
                for (int ks = 0; ks < Kp; ks += 16) {
                    const uint32_t ka = (uint32_t)(a * Kp + ks) / 8, kb = (uint32_t)(b * Kp + ks) / 8;
                    const uint64_t ad = smem_desc(a0 + ka * lboA, lboA, 128);
                    const uint64_t bd = smem_desc(b0 + kb * lboB, lboB, 128);
                    mma_bf16(taddr + (uint32_t)(g * kTN), ad, bd, kIdesc, acc);
                    acc = 1;
                }
            }
        }
        mma_commit(&bar_mma);
    }
    if (!err) err = __syncthreads_or(!mbar_wait(&bar_mma, 0)) ? 2 : 0;
    if (err) {
        if (lane == 0) atomicCAS(&g_tc05_err, 0, err);
        // let what was started drain before the memory goes away
        mbar_wait(&bar_load, 0);
        if (err == 2) mbar_wait(&bar_mma, 0);
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const ModP Md = mods[w];
        const int r = mt * kTM + warp * 32 + lane;
        const uint32_t tl = taddr + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < kTN; c0 += 16) {
            float v[kGroups][16];
#pragma unroll
            for (int g = 0; g < kGroups; ++g) tmem_ld16(tl + (uint32_t)(g * kTN + c0), v[g]);
            if (r < M) {
                int32_t *crow = C + (int64_t)w * sC + (int64_t)r * ldc;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int c = nt * kTN + c0 + j;
                    if (c >= N) break;
                    int64_t s = 0;
#pragma unroll
                    for (int g = kGroups - 1; g >= 0; --g) s = s * 128 + (int64_t)v[g][j];
                    crow[c] = red_bal((int64_t)crow[c] - s, Md);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                     "r"(kTmemCols)
                     : "memory");
}

}  // namespace

size_t tc05_scratch_bytes(int64_t n, int W) {
    const int64_t Mt = (n + kTM - 1) / kTM, Nt = (n + kTN - 1) / kTN;
    return (size_t)W * 2 * 3 * 128 * (size_t)(Mt * kTM + Nt * kTN) + 1024;
}

int gemm_sub_tc05(const int32_t *A, int64_t lda, int64_t sA, const int32_t *B, int64_t ldb,
                  int64_t sB, int32_t *C, int64_t ldc, int64_t sC, int M, int N, int K,
                  const ModP *mods, const LUState *st, int W, void *scratch, cudaStream_t s) {
    if (M <= 0 || N <= 0 || K <= 0) return IDET_OK;
    if (K > 128) {
        set_last_error("tcgen05 trailing update: K must be at most 128 (exactness bound)");
        return IDET_ERR_INTERNAL;
    }
    const int Kp = (K + 15) / 16 * 16;
    const int Mt = (M + kTM - 1) / kTM, Nt = (N + kTN - 1) / kTN;
    __nv_bfloat16 *Apk = (__nv_bfloat16 *)scratch;
    __nv_bfloat16 *Bpk = Apk + (size_t)W * Mt * kTM * 3 * Kp;
    const int64_t total = ((int64_t)Mt * kTM + (int64_t)Nt * kTN) * Kp;
    int pg = (int)std::min<int64_t>((total + 255) / 256, 148 * 8);
    k_pack_limbs<<<dim3(pg, 1, W), 256, 0, s>>>(A, lda, sA, B, ldb, sB, M, N, K, Kp, Mt, Nt, Apk,
                                                 Bpk);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    const size_t smem = (size_t)(kTM + kTN) * 3 * Kp * 2;
    IDET_TRY(allow_max_smem((const void *)k_gemm_tc05));
    k_gemm_tc05<<<dim3(Nt, Mt, W), kT05Threads, smem, s>>>(Apk, Bpk, Kp, Mt, Nt, C, ldc, sC, M, N,
                                                            mods, st);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
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
