// Dixon p-adic lifting with one matrix-vector product and one grid-wide
// barrier per step (Section 2.2: the rational solution of A x = b "using
// Dixon p-adic lifting").
//
// The textbook iteration (C = A^{-1} mod p, balanced digits)
//     x_i = C r_i mods p,   r_{i+1} = (r_i - A x_i) / p
// streams both C and A every step. With the exact integer matrix
//     E = (C A - I) / p,   |E_jk| <= n max|a| (p - 1) / (2 p) + 1 / p,
// and the exact vector y_i = C r_i, the identity
//     C r_{i+1} = (C r_i - C A x_i) / p = (y_i - x_i - p E x_i) / p
// gives
//     x_i = y_i mods p,   y_{i+1} = (y_i - x_i) / p - E x_i,   y_0 = C b,
// the same digits x_i bit for bit, with one int32 matrix (E) read per step
// instead of two. The path applies when n max|a_ij| < 2^32 - 2, so that
// |E| < 2^31; otherwise the two-product kernel of k_lift.cu runs.
//
// E is formed once per solve: E mod 2^32 = (C A - I) (p^{-1} mod 2^32) mod
// 2^32 by a tiled integer GEMM on the CUDA cores in wrapping 32-bit
// arithmetic. The true E lies in (-2^31, 2^31), so its residue mod 2^32
// fixes it. y_0 = C b is formed in 128-bit arithmetic, one warp per row.
//
// The step kernel is persistent and cooperative: one CTA per SM owns a block
// of rows of E. Rows that fit stay in shared memory for the launch; the
// others are read from L2 every step (E of a few thousand rows fits in the
// 126 MB L2: after the first step no DRAM traffic is left; each warp keeps
// four 16-byte loads per lane in flight). Each warp takes a row:
// E_row . x as sums of four int32 x int32 products (each below 2^61, the sum
// below 2^63) folded into a 128-bit accumulator, a warp reduction, then the
// row's update of y (exact division by p as a product with p^{-1} mod 2^128)
// and its next digit. With two right-hand sides (the block lift) both
// vectors share every row of E read. One grid-wide barrier ends each step
// (bounded wait, lift_common.cuh).
//
// Sizes: |y_0| <= n 2^30 2^62 < 2^108 and |E x_i| < 2^16 2^31 2^30 = 2^77,
// so |y_i| < 2^109 throughout (n <= 2^16).
#include <algorithm>
#include <cstdlib>

#include "idet_internal.cuh"
#include "lift_common.cuh"

namespace idet {

namespace {

using namespace lift;

// ---------------------------------------------------------------------------
// E = (C A - I) / p by a GEMM in wrapping 32-bit arithmetic.

constexpr int kGT = 128;       // output tile rows and columns
constexpr int kGK = 16;        // k per shared-memory stage
constexpr int kGThreads = 256;

template <class TA> struct Oct;  // eight consecutive elements of a row of A
template <> struct Oct<int8_t> {
    static __device__ __forceinline__ void load(const int8_t *p, uint32_t (&w)[8]) {
        const uint2 v = *reinterpret_cast<const uint2 *>(p);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            w[t] = (uint32_t)(int32_t)(int8_t)(v.x >> (8 * t));
            w[4 + t] = (uint32_t)(int32_t)(int8_t)(v.y >> (8 * t));
        }
    }
};
template <> struct Oct<int16_t> {
    static __device__ __forceinline__ void load(const int16_t *p, uint32_t (&w)[8]) {
        const uint4 v = *reinterpret_cast<const uint4 *>(p);
        const uint32_t h[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            w[2 * t] = (uint32_t)(int32_t)(int16_t)(h[t] & 0xffff);
            w[2 * t + 1] = (uint32_t)(int32_t)(int16_t)(h[t] >> 16);
        }
    }
};
template <> struct Oct<int32_t> {
    static __device__ __forceinline__ void load(const int32_t *p, uint32_t (&w)[8]) {
        const uint4 v0 = *reinterpret_cast<const uint4 *>(p);
        const uint4 v1 = *reinterpret_cast<const uint4 *>(p + 4);
        w[0] = v0.x, w[1] = v0.y, w[2] = v0.z, w[3] = v0.w;
        w[4] = v1.x, w[5] = v1.y, w[6] = v1.z, w[7] = v1.w;
    }
};

// One CTA per 128 x 128 tile of E; each thread an 8 x 8 block of it (rows
// ty*4 + {0..3, 64..67}, columns tx*4 + {0..3, 64..67}). C has n rows of ld
// int32 (zero columns past n), A n rows of ld entries (zero columns past n);
// rows past n are read as zero. E gets n rows of ld int32.
template <class TA>
__global__ void __launch_bounds__(kGThreads)
k_e_gemm(const int32_t *__restrict__ C, const TA *__restrict__ A, int64_t n, int64_t ld,
         uint32_t pinv32, int32_t *__restrict__ E) {
    __shared__ __align__(16) uint32_t As[kGK][kGT + 4];  // As[k][i] = C[i0 + i][k0 + k]
    __shared__ __align__(16) uint32_t Bs[kGK][kGT + 4];  // Bs[k][j] = A[k0 + k][j0 + j]
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t i0 = (int64_t)blockIdx.y * kGT, j0 = (int64_t)blockIdx.x * kGT;
    // loaders: C row ai (a warp takes 32 consecutive rows: the transposed
    // stores hit 32 distinct banks), k ak..ak+7; A row bk, columns bj..bj+7
    const int ai = tid & 127, ak = (tid >> 7) * 8;
    const int bk = tid >> 4, bj = (tid & 15) * 8;
    uint32_t acc[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = 0;
    uint32_t ca[8], bw[8];
    auto fetch = [&](int64_t k0) {
#pragma unroll
        for (int t = 0; t < 8; ++t) ca[t] = 0, bw[t] = 0;
        if (i0 + ai < n) {
            const uint4 *src = reinterpret_cast<const uint4 *>(C + (i0 + ai) * ld + k0 + ak);
            const uint4 v0 = __ldg(src), v1 = __ldg(src + 1);
            ca[0] = v0.x, ca[1] = v0.y, ca[2] = v0.z, ca[3] = v0.w;
            ca[4] = v1.x, ca[5] = v1.y, ca[6] = v1.z, ca[7] = v1.w;
        }
        const int64_t kr = k0 + bk, jc = j0 + bj;
        if (kr < n && jc < ld) Oct<TA>::load(A + kr * ld + jc, bw);
    };
    fetch(0);
    for (int64_t k0 = 0; k0 < ld; k0 += kGK) {
#pragma unroll
        for (int t = 0; t < 8; ++t) As[ak + t][ai] = ca[t];
        *reinterpret_cast<uint4 *>(&Bs[bk][bj]) = make_uint4(bw[0], bw[1], bw[2], bw[3]);
        *reinterpret_cast<uint4 *>(&Bs[bk][bj + 4]) = make_uint4(bw[4], bw[5], bw[6], bw[7]);
        __syncthreads();
        if (k0 + kGK < ld) fetch(k0 + kGK);
#pragma unroll
        for (int k = 0; k < kGK; ++k) {
            const uint4 a0 = *reinterpret_cast<const uint4 *>(&As[k][ty * 4]);
            const uint4 a1 = *reinterpret_cast<const uint4 *>(&As[k][64 + ty * 4]);
            const uint4 b0 = *reinterpret_cast<const uint4 *>(&Bs[k][tx * 4]);
            const uint4 b1 = *reinterpret_cast<const uint4 *>(&Bs[k][64 + tx * 4]);
            const uint32_t a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const uint32_t b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[r][c] += a[r] * b[c];
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int64_t i = i0 + (r < 4 ? ty * 4 + r : 64 + ty * 4 + r - 4);
        if (i >= n) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t j = j0 + h * 64 + tx * 4;
            if (j >= ld) continue;
            uint32_t v[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) v[c] = (acc[r][h * 4 + c] - (i == j + c ? 1u : 0u)) * pinv32;
            *reinterpret_cast<uint4 *>(E + i * ld + j) = make_uint4(v[0], v[1], v[2], v[3]);
        }
    }
}

// ---------------------------------------------------------------------------
// 128-bit helpers.

// Balanced representative of y mod p for |y| < 2^126 (r64 = 2^64 mod p).
__device__ __forceinline__ int32_t mods128(__int128 y, const ModP &M, uint64_t r64) {
    const int64_t hi = (int64_t)(y >> 64);  // |hi| < 2^62
    const uint64_t lo = (uint64_t)y;
    // lo mod p: Barrett with m = floor((2^64 - 1) / p) leaves r < 3p
    uint64_t r = lo - __umul64hi(lo, M.m) * (uint64_t)M.p;
    if (r >= M.p) r -= M.p;
    if (r >= M.p) r -= M.p;
    return red_bal((int64_t)red_bal(hi, M) * (int64_t)r64 + (int64_t)r, M);
}

__device__ __forceinline__ __int128 warp_sum128(__int128 v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const uint64_t lo = __shfl_xor_sync(0xffffffffu, (unsigned long long)(uint64_t)v, o);
        const int64_t hi = __shfl_xor_sync(0xffffffffu, (long long)(int64_t)(v >> 64), o);
        v += (__int128)(((unsigned __int128)(uint64_t)hi << 64) | lo);
    }
    return v;
}

// y_0 = C b exactly, x_0 = y_0 mods p: one warp per row.
template <int NR>
__global__ void k_lift_e_init(LiftArgs a, int64_t ld, __int128 *__restrict__ ybuf,
                              int32_t *__restrict__ xbuf, uint64_t r64) {
    const int64_t n = a.n;
    const int lane = threadIdx.x & 31;
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= n) return;
    const int32_t *crow = a.Cinv + row * ld;
    const int64_t *bs[2] = {a.b, a.b2};
    int32_t *dg[2] = {a.digits, a.digits2};
    int64_t *zp[2] = {a.zproj, a.zproj2};
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        __int128 acc = 0;
        for (int64_t k = lane; k < n; k += 32) acc += (__int128)crow[k] * (__int128)bs[r][k];
        acc = warp_sum128(acc);
        if (lane == 0) {
            const int32_t x = mods128(acc, a.mod, r64);
            ybuf[r * n + row] = acc;
            xbuf[r * ld + row] = x;
            if (dg[r]) dg[r][row] = x;
            if (zp[r] && a.u && x)
                atomicAdd((unsigned long long *)&zp[r][0], (unsigned long long)((int64_t)a.u[row] * x));
        }
    }
}

// r_{i+1} = (r_i - A x_i) / p from given digits (wrapping 64-bit arithmetic,
// the true value is below 2^62): the residual the textbook iteration would
// carry, for callers that ask for it. One warp per row.
template <class TA>
__global__ void k_residual_step(const TA *__restrict__ A, int64_t n, int64_t ld,
                                const int32_t *__restrict__ x, uint64_t pinv,
                                int64_t *__restrict__ r) {
    const int lane = threadIdx.x & 31;
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= n) return;
    uint64_t acc = 0;
    for (int64_t k = lane; k < n; k += 32)
        acc += (uint64_t)((int64_t)A[row * ld + k] * (int64_t)x[k]);
    acc = (uint64_t)warp_sum64((int64_t)acc);
    if (lane == 0) r[row] = (int64_t)(((uint64_t)r[row] - acc) * pinv);
}

// ---------------------------------------------------------------------------
// The step kernel.

constexpr int kThreads = 1024;  // 32 warps, a row each at a time
constexpr int kWarps = kThreads / 32;

struct EGeom {
    int64_t ld;   // row length (multiple of 16)
    int64_t rpc;  // rows per CTA
    int cE;       // rows of E resident in shared memory per CTA
    int pad[3];
    uint64_t pinv_lo, pinv_hi;  // p^{-1} mod 2^128
    uint64_t r64;               // 2^64 mod p
};

// E_row . x_r for the NR staged vectors: sums of four products (each below
// 2^61 in magnitude, the sum below 2^63) folded into 128-bit accumulators,
// then a warp reduction. GLOBAL: the row is read from L2 (ld.global.cg,
// four 16-byte loads in flight per lane); else from shared memory.
template <int NR, bool GLOBAL>
__device__ __forceinline__ void dot_e(const int4 *__restrict__ erow, const int4 *__restrict__ xs,
                                      int64_t nq, int lane, __int128 (&acc)[NR]) {
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = 0;
#pragma unroll 4
    for (int64_t q = lane; q < nq; q += 32) {
        const int4 e = GLOBAL ? __ldcg(erow + q) : erow[q];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int4 v = xs[r * nq + q];
            const int64_t t = (int64_t)e.x * v.x + (int64_t)e.y * v.y + (int64_t)e.z * v.z +
                              (int64_t)e.w * v.w;
            acc[r] += t;
        }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = warp_sum128(acc[r]);
}

template <int NR>
__global__ void __launch_bounds__(kThreads, 1)
k_lift_e(LiftArgs a, const int32_t *__restrict__ E, EGeom g, __int128 *__restrict__ ybuf,
         int32_t *__restrict__ xbuf, GridBar *gb, long long limit) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int64_t s_z[NR][kWarps];
    const int64_t n = a.n, ld = g.ld, nq = ld / 4;
    const ModP M = a.mod;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * g.rpc;
    const int64_t r1 = min(n, r0 + g.rpc);
    const int nrows = r1 > r0 ? (int)(r1 - r0) : 0;
    int4 *xs = reinterpret_cast<int4 *>(smem);                        // NR x ld int32
    __int128 *sy = reinterpret_cast<__int128 *>(smem + 4 * ld * NR);  // rpc x NR
    int32_t *cE = reinterpret_cast<int32_t *>(smem + 4 * ld * NR + 16 * g.rpc * NR);
    const int kc = min(g.cE, nrows);
    const int steps = a.m - 1;
    const unsigned G = gridDim.x;
    const unsigned __int128 pinv = ((unsigned __int128)g.pinv_hi << 64) | g.pinv_lo;
    int32_t *dg[2] = {a.digits, a.digits2};
    int64_t *zp[2] = {a.zproj, a.zproj2};

    // resident rows and the rows' y
    {
        const int4 *src = reinterpret_cast<const int4 *>(E + r0 * ld);
        int4 *dst = reinterpret_cast<int4 *>(cE);
        for (int64_t e = tid; e < (int64_t)kc * nq; e += kThreads) dst[e] = __ldg(src + e);
        for (int e = tid; e < nrows * NR; e += kThreads)
            sy[e] = ybuf[(int64_t)(e % NR) * n + r0 + e / NR];
    }
    __syncthreads();

    unsigned bar = 0;
    for (int it = 0; it < steps; ++it) {
        const int32_t *xin = xbuf + (int64_t)(it & 1) * NR * ld;
        int32_t *xout = xbuf + (int64_t)((it + 1) & 1) * NR * ld;
        {
            const int4 *src = reinterpret_cast<const int4 *>(xin);
            for (int64_t q = tid; q < NR * nq; q += kThreads) xs[q] = __ldcg(src + q);
        }
        __syncthreads();
        int64_t zpart[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) zpart[r] = 0;
        for (int lr = warp; lr < nrows; lr += kWarps) {
            __int128 acc[NR];
            if (lr < kc)
                dot_e<NR, false>(reinterpret_cast<const int4 *>(cE + (int64_t)lr * ld), xs, nq,
                                 lane, acc);
            else
                dot_e<NR, true>(reinterpret_cast<const int4 *>(E + (r0 + lr) * ld), xs, nq, lane,
                                acc);
            if (lane == 0) {
                const int64_t row = r0 + lr;
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const int32_t xi = reinterpret_cast<const int32_t *>(xs)[r * ld + row];
                    // (y - x_i) is divisible by p: exact division
                    const unsigned __int128 d = (unsigned __int128)(sy[lr * NR + r] - xi);
                    const __int128 y = (__int128)(d * pinv) - acc[r];
                    sy[lr * NR + r] = y;
                    const int32_t xn = mods128(y, M, g.r64);
                    xout[r * ld + row] = xn;
                    if (dg[r]) dg[r][(int64_t)(it + 1) * n + row] = xn;
                    if (a.u) zpart[r] += (int64_t)a.u[row] * xn;
                }
            }
        }
        if (a.u) {
#pragma unroll
            for (int r = 0; r < NR; ++r)
                if (lane == 0) s_z[r][warp] = zpart[r];
            __syncthreads();
            if (tid < NR && zp[tid]) {
                int64_t t = 0;
                for (int k = 0; k < kWarps; ++k) t += s_z[tid][k];
                if (t) atomicAdd((unsigned long long *)&zp[tid][it + 1], (unsigned long long)t);
            }
        }
        if (!grid_sync<kThreads>(gb, (++bar) * G, limit)) return;
    }
}

unsigned __int128 inv_mod_2_128(uint64_t p) {
    unsigned __int128 x = p;  // p * p = 1 mod 8
    for (int i = 0; i < 7; ++i) x *= 2 - (unsigned __int128)p * x;
    return x;
}

template <class TA>
int launch_lift_e_t(const LiftArgs &a, const TA *A, int64_t ld, Workspace &ws, int *timed_out,
                    float *ms, LiftInfo *info) {
    cudaStream_t s = ws.stream();
    const int64_t n = a.n;
    const int NR = a.nrhs == 2 ? 2 : 1;
    const uint32_t p = a.mod.p;
    int32_t *E = nullptr, *xbuf = nullptr;
    __int128 *ybuf = nullptr;
    GridBar *gb = nullptr;
    IDET_TRY(ws.alloc_n(&E, (size_t)n * ld));
    IDET_TRY(ws.alloc_n(&xbuf, 2 * (size_t)NR * ld));
    IDET_TRY(ws.alloc_n(&ybuf, (size_t)NR * n));
    IDET_TRY(ws.alloc_n(&gb, 1));
    IDET_CUDA_TRY(cudaMemsetAsync(xbuf, 0, sizeof(int32_t) * 2 * NR * ld, s));
    IDET_CUDA_TRY(cudaMemsetAsync(gb, 0, sizeof(GridBar), s));
    if (a.zproj) IDET_CUDA_TRY(cudaMemsetAsync(a.zproj, 0, sizeof(int64_t) * a.m, s));
    if (NR == 2 && a.zproj2) IDET_CUDA_TRY(cudaMemsetAsync(a.zproj2, 0, sizeof(int64_t) * a.m, s));
    EventPair ev0, ev1;
    if (ms || info) {
        IDET_CUDA_TRY(cudaEventCreate(&ev0.a));
        IDET_CUDA_TRY(cudaEventCreate(&ev0.b));
        IDET_CUDA_TRY(cudaEventCreate(&ev1.b));
        IDET_CUDA_TRY(cudaEventRecord(ev0.a, s));
    }
    const unsigned __int128 pinv = inv_mod_2_128(p);
    {
        dim3 grid((unsigned)((ld + kGT - 1) / kGT), (unsigned)((n + kGT - 1) / kGT));
        k_e_gemm<TA><<<grid, kGThreads, 0, s>>>(a.Cinv, A, n, ld, (uint32_t)pinv, E);
        count_launch();
        IDET_CUDA_TRY(cudaGetLastError());
    }
    const uint64_t r64 = (uint64_t)(((unsigned __int128)1 << 64) % p);
    {
        const unsigned blocks = (unsigned)((n * 32 + 255) / 256);
        if (NR == 2)
            k_lift_e_init<2><<<blocks, 256, 0, s>>>(a, ld, ybuf, xbuf, r64);
        else
            k_lift_e_init<1><<<blocks, 256, 0, s>>>(a, ld, ybuf, xbuf, r64);
        count_launch();
        IDET_CUDA_TRY(cudaGetLastError());
    }
    if (ms || info) IDET_CUDA_TRY(cudaEventRecord(ev0.b, s));

    int dev = 0, sms = 0, smem_max = 0;
    IDET_CUDA_TRY(cudaGetDevice(&dev));
    IDET_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    IDET_CUDA_TRY(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int64_t row = 4 * ld;
    EGeom g{};
    g.ld = ld;
    g.pinv_lo = (uint64_t)pinv;
    g.pinv_hi = (uint64_t)(pinv >> 64);
    g.r64 = r64;
    // Fewest CTAs with one row per warp, if all their rows then fit in shared
    // memory (fewer CTAs make the grid barrier cheaper); otherwise all SMs,
    // as many rows resident as fit, the others read from L2 every step.
    int64_t G = std::min<int64_t>(sms, (n + kWarps - 1) / kWarps);
    if (G < 1) G = 1;
    g.rpc = (n + G - 1) / G;
    auto fixed = [&](int64_t rpc) { return 4 * ld * NR + 16 * rpc * NR + 2048; };
    if (g.rpc * row + fixed(g.rpc) > smem_max) {
        G = sms;
        g.rpc = (n + G - 1) / G;
    }
    if (fixed(g.rpc) > smem_max) {
        set_last_error("lift: the vector does not fit in shared memory (n too large)");
        return IDET_ERR_ARG;
    }
    g.cE = (int)std::min<int64_t>(g.rpc, ((int64_t)smem_max - fixed(g.rpc)) / row);
    const size_t smem = (size_t)(4 * ld * NR + 16 * g.rpc * NR + (int64_t)g.cE * row);
    const void *kern = NR == 2 ? (const void *)k_lift_e<2> : (const void *)k_lift_e<1>;
    IDET_TRY(allow_max_smem(kern));
    int occ = 0;
    IDET_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem));
    if (occ < 1) {
        set_last_error("lift kernel does not fit on an SM");
        return IDET_ERR_INTERNAL;
    }
    float step_ms = 0;
    GridBar hb{};
    if (a.m >= 2) {
        long long limit = lift_wait_cycles();
        LiftArgs ak = a;
        void *args[] = {(void *)&ak, (void *)&E, (void *)&g, (void *)&ybuf,
                        (void *)&xbuf, (void *)&gb, (void *)&limit};
        // one grid-synchronised lift at a time in the process (held until
        // the kernel has finished: the stream is synchronised below)
        std::unique_lock<std::mutex> coop(g_coop_mu);
        IDET_CUDA_TRY(cudaLaunchCooperativeKernel(kern, dim3((unsigned)G), dim3(kThreads), args,
                                                  smem, s));
        count_launch();
        if (ms || info) IDET_CUDA_TRY(cudaEventRecord(ev1.b, s));
        IDET_CUDA_TRY(cudaMemcpyAsync(&hb, gb, sizeof(GridBar), cudaMemcpyDeviceToHost, s));
        IDET_CUDA_TRY(cudaStreamSynchronize(s));
        if (ms || info) IDET_CUDA_TRY(cudaEventElapsedTime(&step_ms, ev0.b, ev1.b));
    } else {
        IDET_CUDA_TRY(cudaStreamSynchronize(s));
    }
    float setup_ms = 0;
    if (ms || info) IDET_CUDA_TRY(cudaEventElapsedTime(&setup_ms, ev0.a, ev0.b));
    if (ms) *ms = setup_ms + step_ms;
    if (info) {
        info->path = 1;
        info->ms_setup = setup_ms;
        info->ms_steps = step_ms;
        info->steps = std::max(0, a.m - 1);
        info->bytes = (double)info->steps * 4.0 * (double)n * (double)n;
    }
    if (timed_out) *timed_out = hb.err;
    if (hb.err) {
        set_last_error("lift: a bounded wait gave up (code %d, block %d; grid %d, cE %d, rpc %d)",
                       hb.err, hb.info[0], (int)G, g.cE, (int)g.rpc);
        return IDET_ERR_TIMEOUT;
    }
    // the residuals r_m, when asked for, from the digits
    const int64_t *bs[2] = {a.b, a.b2};
    int32_t *dgs[2] = {a.digits, a.digits2};
    int64_t *rs[2] = {a.r, a.r2};
    for (int r = 0; r < NR; ++r) {
        if (!rs[r] || (a.m > 0 && !dgs[r])) continue;
        IDET_CUDA_TRY(cudaMemcpyAsync(rs[r], bs[r], sizeof(int64_t) * n, cudaMemcpyDeviceToDevice, s));
        const uint64_t pinv64 = (uint64_t)pinv;
        for (int i = 0; i < a.m; ++i) {
            k_residual_step<TA><<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(
                A, n, ld, dgs[r] + (int64_t)i * n, pinv64, rs[r]);
            count_launch();
            IDET_CUDA_TRY(cudaGetLastError());
        }
    }
    IDET_CUDA_TRY(cudaStreamSynchronize(s));
    return IDET_OK;
}

}  // namespace

bool lift_e_applies(int64_t n, uint64_t amax) {
    if (amax == 0) return false;
    if (const char *e = getenv("IDET_LIFT_PATH"))
        if (e[0] == 'c') return false;  // "classic": the two-product kernel
    return (double)n * (double)amax < 4294967294.0;
}

int launch_lift_e(const LiftArgs &a, const void *Anar, int abytes, int64_t ld, Workspace &ws,
                  int *timed_out, float *ms, LiftInfo *info) {
    if (ld % 16 != 0) {
        set_last_error("lift: leading dimension must be a multiple of 16");
        return IDET_ERR_INTERNAL;
    }
    if (abytes == 1)
        return launch_lift_e_t<int8_t>(a, (const int8_t *)Anar, ld, ws, timed_out, ms, info);
    if (abytes == 2)
        return launch_lift_e_t<int16_t>(a, (const int16_t *)Anar, ld, ws, timed_out, ms, info);
    return launch_lift_e_t<int32_t>(a, (const int32_t *)Anar, ld, ws, timed_out, ms, info);
}

}  // namespace idet
