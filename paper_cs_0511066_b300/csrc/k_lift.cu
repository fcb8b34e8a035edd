// Dixon p-adic lifting (Section 2.2: "The cost of solving using Dixon p-adic
// lifting is O(n^3 log^2(n||A||) + n log^2(||b||))"), one persistent
// cooperative kernel for all m iterations:
//
//   r_0 = b;  for i < m:  x_i = C (r_i mod p) mod p   (balanced digits)
//                         r_{i+1} = (r_i - A x_i) / p  (exact)
//
// with C = A^{-1} mod p precomputed from the LU of A mod p. Each iteration is
// two matrix-vector products separated by grid-wide barriers; rows are
// distributed over all warps of the grid. Both products stream an n x n int32
// matrix, so the kernel is bound by memory bandwidth (HBM, or L2 when the two
// matrices fit).
//
// Exactness:
//  * x_i: |C_jk| < 2^30 and r mod p is split as hi * 2^16 + lo with
//    0 <= lo < 2^16, |hi| < 2^14, so both partial sums stay below
//    n 2^46 < 2^58 (n <= 4096) in int64.
//  * r_{i+1}: the true value is an integer of magnitude below
//    |r_i|/p + n ||A|| < 2^62, and it equals (r_i - A x_i) times p^{-1} modulo
//    2^64; so the products and the sum are taken modulo 2^64 (wrapping) and
//    multiplied by the inverse of p modulo 2^64 (exact division).
#include "idet_internal.cuh"

namespace idet {

namespace {

constexpr int kLiftThreads = 256;
constexpr long long kSpinLimit = 1ll << 24;

struct GridBar {
    unsigned int count;
    unsigned int gen;
    int err;
    int pad;
};

// Grid-wide barrier with a bounded wait: after kSpinLimit polls the waiting
// block records err = 1 and returns; callers then leave the kernel.
__device__ bool grid_sync(GridBar *gb, unsigned nblocks) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *vgen = &gb->gen;
        volatile int *verr = &gb->err;
        unsigned int g = *vgen;
        __threadfence();
        unsigned int arrived = atomicAdd(&gb->count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(&gb->count, 0u);
            __threadfence();
            atomicAdd(&gb->gen, 1u);
        } else {
            long long spins = 0;
            while (*vgen == g && *verr == 0) {
                if (++spins > kSpinLimit) {
                    atomicExch(&gb->err, 1);
                    break;
                }
                __nanosleep(32);
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

// ld: leading dimension (multiple of 4) of A32 and Cinv; columns n..ld-1 are
// zero, as are rm[n..ld) and xcur[n..ld).
__global__ void __launch_bounds__(kLiftThreads)
k_lift(LiftArgs a, int64_t ld, int32_t *__restrict__ rm, int32_t *__restrict__ xcur,
       GridBar *gb) {
    const unsigned nblocks = gridDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = kLiftThreads / 32;
    const int64_t gwarp = (int64_t)blockIdx.x * nwarps + warp;
    const int64_t twarps = (int64_t)nblocks * nwarps;
    const int64_t n = a.n;
    const ModP M = a.mod;
    __shared__ int64_t s_z[kLiftThreads / 32];

    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)nblocks * blockDim.x) {
        int64_t bi = a.b[i];
        a.r[i] = bi;
        rm[i] = red_bal(bi, M);
    }
    if (!grid_sync(gb, nblocks)) return;

    for (int it = 0; it < a.m; ++it) {
        // Phase 1: x = C rm mod p.
        int64_t zpart = 0;
        for (int64_t row = gwarp; row < n; row += twarps) {
            const int4 *crow = reinterpret_cast<const int4 *>(a.Cinv + row * ld);
            const int4 *rv = reinterpret_cast<const int4 *>(rm);
            int64_t lo = 0, hi = 0;
            for (int64_t q = lane; q < ld / 4; q += 32) {
                int4 c = __ldg(crow + q);
                int4 v = __ldcg(rv + q);  // written by other blocks: bypass L1
                lo += (int64_t)c.x * (v.x & 0xffff) + (int64_t)c.y * (v.y & 0xffff) +
                      (int64_t)c.z * (v.z & 0xffff) + (int64_t)c.w * (v.w & 0xffff);
                hi += (int64_t)c.x * (v.x >> 16) + (int64_t)c.y * (v.y >> 16) +
                      (int64_t)c.z * (v.z >> 16) + (int64_t)c.w * (v.w >> 16);
            }
            lo = warp_sum64(lo);
            hi = warp_sum64(hi);
            if (lane == 0) {
                int32_t x = red_bal((int64_t)red_bal(hi, M) * 65536 + lo, M);
                xcur[row] = x;
                if (a.digits) a.digits[(int64_t)it * n + row] = x;
                if (a.u) zpart += (int64_t)a.u[row] * x;
            }
        }
        if (a.zproj) {
            if (lane == 0) s_z[warp] = zpart;
            __syncthreads();
            if (threadIdx.x == 0) {
                int64_t t = 0;
                for (int k = 0; k < nwarps; ++k) t += s_z[k];
                if (t) atomicAdd((unsigned long long *)&a.zproj[it], (unsigned long long)t);
            }
        }
        if (!grid_sync(gb, nblocks)) return;

        // Phase 2: r <- (r - A x) / p.
        for (int64_t row = gwarp; row < n; row += twarps) {
            const int4 *arow = reinterpret_cast<const int4 *>(a.A32 + row * ld);
            const int4 *xv = reinterpret_cast<const int4 *>(xcur);
            uint64_t acc = 0;
            for (int64_t q = lane; q < ld / 4; q += 32) {
                int4 av = __ldg(arow + q);
                int4 x = __ldcg(xv + q);
                acc += (uint64_t)((int64_t)av.x * x.x) + (uint64_t)((int64_t)av.y * x.y) +
                       (uint64_t)((int64_t)av.z * x.z) + (uint64_t)((int64_t)av.w * x.w);
            }
            acc = (uint64_t)warp_sum64((int64_t)acc);
            if (lane == 0) {
                uint64_t diff = (uint64_t)__ldcg(a.r + row) - acc;
                int64_t rn = (int64_t)(diff * a.pinv);
                a.r[row] = rn;
                rm[row] = red_bal(rn, M);
            }
        }
        if (!grid_sync(gb, nblocks)) return;
    }
}

}  // namespace

int launch_lift(const LiftArgs &a0, Workspace &ws, int *timed_out, float *ms) {
    cudaStream_t s = ws.stream();
    LiftArgs a = a0;
    const int64_t n = a.n;
    const int64_t ld = (n + 3) / 4 * 4;
    int32_t *rm = nullptr, *xcur = nullptr;
    GridBar *gb = nullptr;
    IDET_TRY(ws.alloc_n(&rm, ld));
    IDET_TRY(ws.alloc_n(&xcur, ld));
    IDET_TRY(ws.alloc_n(&gb, 1));
    IDET_CUDA_TRY(cudaMemsetAsync(rm, 0, sizeof(int32_t) * ld, s));
    IDET_CUDA_TRY(cudaMemsetAsync(xcur, 0, sizeof(int32_t) * ld, s));
    IDET_CUDA_TRY(cudaMemsetAsync(gb, 0, sizeof(GridBar), s));
    if (a.zproj) IDET_CUDA_TRY(cudaMemsetAsync(a.zproj, 0, sizeof(int64_t) * a.m, s));

    int dev = 0, sms = 0, occ = 0;
    IDET_CUDA_TRY(cudaGetDevice(&dev));
    IDET_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    IDET_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_lift,
                                                                kLiftThreads, 0));
    if (occ < 1) occ = 1;
    if (occ > 4) occ = 4;
    int64_t need = (n * 32 + kLiftThreads - 1) / kLiftThreads;  // one warp per row
    int64_t nblk = (int64_t)sms * occ;
    if (nblk > need) nblk = need < 1 ? 1 : need;
    int64_t ldv = ld;
    void *args[] = {(void *)&a, (void *)&ldv, (void *)&rm, (void *)&xcur, (void *)&gb};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ms) {
        IDET_CUDA_TRY(cudaEventCreate(&e0));
        IDET_CUDA_TRY(cudaEventCreate(&e1));
        IDET_CUDA_TRY(cudaEventRecord(e0, s));
    }
    IDET_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)k_lift, dim3((unsigned)nblk),
                                              dim3(kLiftThreads), args, 0, s));
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

}  // namespace idet
