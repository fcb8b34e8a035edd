// Dixon p-adic lifting (Section 2.2: "The cost of solving using Dixon p-adic
// lifting is O(n^3 log^2(n||A||) + n log^2(||b||))"), one persistent
// cooperative kernel for all m iterations:
//
//   r_0 = b;  for i < m:  x_i = C (r_i mod p) mod p   (balanced digits)
//                         r_{i+1} = (r_i - A x_i) / p  (exact)
//
// with C = A^{-1} mod p precomputed from the LU of A mod p. Each iteration is
// two matrix-vector products separated by grid-wide barriers.
//
// Layout: one CTA per SM (32 warps, one row per warp at a time); CTA b owns a
// contiguous block of rows of C and A.
// As many of its rows as fit are copied to shared memory once and stay there
// for all m iterations; the rest are streamed from global memory (L2 when
// the streamed part fits in it). A is stored in the narrowest of
// int8/int16/int32 that holds its entries; rows are zero padded to a
// multiple of 16 elements. The vector operand (r mod p, then x) is staged in
// shared memory at the start of each phase.
//
// Exactness:
//  * x_i: |C_jk| < 2^30 and r mod p is split as hi * 2^16 + lo with
//    0 <= lo < 2^16, |hi| < 2^14, so both partial sums stay below
//    n 2^46 < 2^62 for n < 2^16, in int64.
//  * r_{i+1}: the true value is an integer of magnitude below
//    |r_i|/p + n ||A|| < 2^62, equal to (r_i - A x_i) p^{-1} modulo 2^64; so
//    products and sums are taken modulo 2^64 (wrapping) and multiplied by
//    the inverse of p modulo 2^64 (exact division).
#include <algorithm>

#include "idet_internal.cuh"

namespace idet {

namespace {

constexpr int kLiftThreads = 1024;
constexpr int kLiftWarps = kLiftThreads / 32;
constexpr long long kSpinLimit = 1ll << 26;

struct GridBar {
    unsigned int count;  // arrivals, monotone within one launch
    int err;
    int pad[2];
};

// Grid-wide barrier: the b-th barrier of the launch completes when
// count reaches b * gridDim.x. Bounded wait: after kSpinLimit polls the
// block records err = 1 and every block leaves at its next barrier.
__device__ __forceinline__ bool grid_sync(GridBar *gb, unsigned target) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&gb->count, 1u);
        volatile unsigned int *vc = &gb->count;
        volatile int *ve = &gb->err;
        long long spins = 0;
        while (*vc < target) {
            if (*ve) break;
            if (++spins > kSpinLimit) {
                atomicExch(&gb->err, 1);
                break;
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *((volatile int *)&gb->err) == 0;
}

__device__ __forceinline__ int64_t warp_sum64(int64_t v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Four consecutive elements of a row of A.
template <class TA> struct Quad;
template <> struct Quad<int8_t> {
    using V = char4;
};
template <> struct Quad<int16_t> {
    using V = short4;
};
template <> struct Quad<int32_t> {
    using V = int4;
};

struct LiftGeom {
    int64_t ld;   // padded row length (multiple of 16)
    int64_t rpc;  // rows per CTA
    int cC, cA;   // rows of C / A kept in shared memory per CTA
};

// Row products, one warp per row. The vector operand is staged in shared
// memory once per phase; for the x phase it is pre-split into
// lo = (r mod p) & 0xffff and hi = (r mod p) >> 16 so that the inner loop is
// two 32x32->64-bit multiply-adds per element.
template <bool SMEM>
__device__ __forceinline__ int32_t dot_c(const int4 *__restrict__ crow,
                                         const int4 *__restrict__ vlo,
                                         const int4 *__restrict__ vhi, int64_t nq, int lane,
                                         const ModP &M) {
    int64_t lo = 0, hi = 0;
#pragma unroll 8
    for (int64_t q = lane; q < nq; q += 32) {
        const int4 c = SMEM ? crow[q] : __ldg(crow + q);
        const int4 l = vlo[q], h = vhi[q];
        lo += (int64_t)c.x * l.x;
        lo += (int64_t)c.y * l.y;
        lo += (int64_t)c.z * l.z;
        lo += (int64_t)c.w * l.w;
        hi += (int64_t)c.x * h.x;
        hi += (int64_t)c.y * h.y;
        hi += (int64_t)c.z * h.z;
        hi += (int64_t)c.w * h.w;
    }
    lo = warp_sum64(lo);
    hi = warp_sum64(hi);
    return red_bal((int64_t)red_bal(hi, M) * 65536 + red_bal(lo, M), M);
}

template <class TA, bool SMEM>
__device__ __forceinline__ uint64_t dot_a(const typename Quad<TA>::V *__restrict__ arow,
                                          const int4 *__restrict__ v, int64_t nq, int lane) {
    uint64_t acc = 0;
#pragma unroll 8
    for (int64_t q = lane; q < nq; q += 32) {
        const typename Quad<TA>::V a = SMEM ? arow[q] : __ldg(arow + q);
        const int4 x = v[q];
        acc += (uint64_t)((int64_t)a.x * x.x);
        acc += (uint64_t)((int64_t)a.y * x.y);
        acc += (uint64_t)((int64_t)a.z * x.z);
        acc += (uint64_t)((int64_t)a.w * x.w);
    }
    return (uint64_t)warp_sum64((int64_t)acc);
}

template <class TA>
__global__ void __launch_bounds__(kLiftThreads, 1)
k_lift(LiftArgs a, const TA *__restrict__ Anar, LiftGeom g, int32_t *__restrict__ rm,
       int32_t *__restrict__ xcur, GridBar *gb) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int64_t n = a.n, ld = g.ld, nq = ld / 4;
    const ModP M = a.mod;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * g.rpc;
    const int64_t r1 = min(n, r0 + g.rpc);
    const int nrows = r1 > r0 ? (int)(r1 - r0) : 0;
    int4 *vlo = reinterpret_cast<int4 *>(smem);                          // ld int32
    int4 *vhi = reinterpret_cast<int4 *>(smem + 4 * ld);                 // ld int32
    int32_t *cC = reinterpret_cast<int32_t *>(smem + 8 * ld);            // g.cC rows
    TA *cA = reinterpret_cast<TA *>(smem + 8 * ld + 4 * ld * g.cC);      // g.cA rows
    __shared__ int64_t s_z[kLiftWarps];
    unsigned bar = 0;
    const unsigned G = gridDim.x;
    const int kc = min(g.cC, nrows), ka = min(g.cA, nrows);

    // resident rows
    {
        const int4 *src = reinterpret_cast<const int4 *>(a.Cinv + r0 * ld);
        int4 *dst = reinterpret_cast<int4 *>(cC);
        for (int64_t e = tid; e < (int64_t)kc * nq; e += kLiftThreads) dst[e] = __ldg(src + e);
        const int4 *srcA = reinterpret_cast<const int4 *>(Anar + r0 * ld);
        int4 *dstA = reinterpret_cast<int4 *>(cA);
        const int64_t qa = ld * (int64_t)sizeof(TA) / 16;
        for (int64_t e = tid; e < (int64_t)ka * qa; e += kLiftThreads) dstA[e] = __ldg(srcA + e);
    }
    for (int64_t i = r0 + tid; i < r1; i += kLiftThreads) {
        int64_t bi = a.b[i];
        a.r[i] = bi;
        rm[i] = red_bal(bi, M);
    }
    if (!grid_sync(gb, (++bar) * G)) return;

    using V = typename Quad<TA>::V;
    for (int it = 0; it < a.m; ++it) {
        // Phase 1: x = C (r mod p) mod p on this CTA's rows.
        {
            const int4 *src = reinterpret_cast<const int4 *>(rm);
            for (int64_t q = tid; q < nq; q += kLiftThreads) {
                const int4 v = __ldcg(src + q);
                vlo[q] = make_int4(v.x & 0xffff, v.y & 0xffff, v.z & 0xffff, v.w & 0xffff);
                vhi[q] = make_int4(v.x >> 16, v.y >> 16, v.z >> 16, v.w >> 16);
            }
        }
        __syncthreads();
        int64_t zpart = 0;
        for (int lr = warp; lr < nrows; lr += kLiftWarps) {
            const int64_t row = r0 + lr;
            const int32_t x =
                lr < kc ? dot_c<true>(reinterpret_cast<const int4 *>(cC + (int64_t)lr * ld), vlo,
                                      vhi, nq, lane, M)
                        : dot_c<false>(reinterpret_cast<const int4 *>(a.Cinv + row * ld), vlo,
                                       vhi, nq, lane, M);
            if (lane == 0) {
                xcur[row] = x;
                if (a.digits) a.digits[(int64_t)it * n + row] = x;
                if (a.u) zpart += (int64_t)a.u[row] * x;
            }
        }
        if (a.zproj) {
            if (lane == 0) s_z[warp] = zpart;
            __syncthreads();
            if (tid == 0) {
                int64_t t = 0;
                for (int k = 0; k < kLiftWarps; ++k) t += s_z[k];
                if (t) atomicAdd((unsigned long long *)&a.zproj[it], (unsigned long long)t);
            }
        }
        if (!grid_sync(gb, (++bar) * G)) return;

        // Phase 2: r <- (r - A x) / p on this CTA's rows.
        {
            const int4 *src = reinterpret_cast<const int4 *>(xcur);
            for (int64_t q = tid; q < nq; q += kLiftThreads) vlo[q] = __ldcg(src + q);
        }
        __syncthreads();
        for (int lr = warp; lr < nrows; lr += kLiftWarps) {
            const int64_t row = r0 + lr;
            const uint64_t acc =
                lr < ka ? dot_a<TA, true>(reinterpret_cast<const V *>(cA + (int64_t)lr * ld), vlo,
                                          nq, lane)
                        : dot_a<TA, false>(reinterpret_cast<const V *>(Anar + row * ld), vlo, nq,
                                           lane);
            if (lane == 0) {
                uint64_t diff = (uint64_t)__ldcg(a.r + row) - acc;
                int64_t rn = (int64_t)(diff * a.pinv);
                a.r[row] = rn;
                rm[row] = red_bal(rn, M);
            }
        }
        if (!grid_sync(gb, (++bar) * G)) return;
    }
}

template <class TA>
int launch_lift_t(const LiftArgs &a0, const void *Anar, int64_t ld, Workspace &ws,
                  int *timed_out, float *ms) {
    cudaStream_t s = ws.stream();
    LiftArgs a = a0;
    const int64_t n = a.n;
    int32_t *rm = nullptr, *xcur = nullptr;
    GridBar *gb = nullptr;
    IDET_TRY(ws.alloc_n(&rm, ld));
    IDET_TRY(ws.alloc_n(&xcur, ld));
    IDET_TRY(ws.alloc_n(&gb, 1));
    IDET_CUDA_TRY(cudaMemsetAsync(rm, 0, sizeof(int32_t) * ld, s));
    IDET_CUDA_TRY(cudaMemsetAsync(xcur, 0, sizeof(int32_t) * ld, s));
    IDET_CUDA_TRY(cudaMemsetAsync(gb, 0, sizeof(GridBar), s));
    if (a.zproj) IDET_CUDA_TRY(cudaMemsetAsync(a.zproj, 0, sizeof(int64_t) * a.m, s));

    int dev = 0, sms = 0, smem_max = 0;
    IDET_CUDA_TRY(cudaGetDevice(&dev));
    IDET_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    IDET_CUDA_TRY(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    // CTAs: one per SM, but no more than needed for one warp per row.
    int64_t G = sms;
    const int64_t need = (n + kLiftWarps - 1) / kLiftWarps;
    if (G > need) G = need < 1 ? 1 : need;
    LiftGeom g;
    g.ld = ld;
    g.rpc = (n + G - 1) / G;
    const int64_t budget = (int64_t)smem_max - 8 * ld - 2048;
    const int64_t crow = 4 * ld, arow = (int64_t)sizeof(TA) * ld;
    const int64_t cC = budget > 0 ? std::min<int64_t>(g.rpc, budget / crow) : 0;
    const int64_t rest = budget - cC * crow;
    const int64_t cA = rest > 0 ? std::min<int64_t>(g.rpc, rest / arow) : 0;
    g.cC = (int)cC;
    g.cA = (int)cA;
    const size_t smem = (size_t)(8 * ld + cC * crow + cA * arow);
    IDET_CUDA_TRY(cudaFuncSetAttribute(k_lift<TA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    int occ = 0;
    IDET_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_lift<TA>, kLiftThreads,
                                                                smem));
    if (occ < 1) {
        set_last_error("lift kernel does not fit on an SM");
        return IDET_ERR_INTERNAL;
    }
    const TA *Ap = (const TA *)Anar;
    void *args[] = {(void *)&a, (void *)&Ap, (void *)&g, (void *)&rm, (void *)&xcur, (void *)&gb};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ms) {
        IDET_CUDA_TRY(cudaEventCreate(&e0));
        IDET_CUDA_TRY(cudaEventCreate(&e1));
        IDET_CUDA_TRY(cudaEventRecord(e0, s));
    }
    IDET_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)k_lift<TA>, dim3((unsigned)G),
                                              dim3(kLiftThreads), args, smem, s));
    count_launch();
    if (ms) {
        IDET_CUDA_TRY(cudaEventRecord(e1, s));
        IDET_CUDA_TRY(cudaEventSynchronize(e1));
        IDET_CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    int err = 0;
    IDET_CUDA_TRY(cudaMemcpyAsync(&err, &gb->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaStreamSynchronize(s));
    if (timed_out) *timed_out = err;
    if (err) {
        set_last_error("lift: a grid barrier wait exceeded its limit");
        return IDET_ERR_TIMEOUT;
    }
    return IDET_OK;
}

}  // namespace

int launch_lift(const LiftArgs &a, const void *Anar, int abytes, int64_t ld, Workspace &ws,
                int *timed_out, float *ms) {
    if (ld % 16 != 0) {
        set_last_error("lift: leading dimension must be a multiple of 16");
        return IDET_ERR_INTERNAL;
    }
    if (abytes == 1) return launch_lift_t<int8_t>(a, Anar, ld, ws, timed_out, ms);
    if (abytes == 2) return launch_lift_t<int16_t>(a, Anar, ld, ws, timed_out, ms);
    return launch_lift_t<int32_t>(a, Anar, ld, ws, timed_out, ms);
}

}  // namespace idet
