// Residue reduction A -> A mod p_k for a batch of primes, and row statistics
// for the Hadamard bound.
//
// The reduction is the n^2 log||A|| term of the per-prime cost (Section 2.1,
// "Its complexity is O(n^omega + n^2 log(||A||))"). It is a streaming
// kernel: each int64 entry is read once per batch of W primes and W int32
// residues are written, so it is bound by HBM bandwidth.
#include "idet_internal.cuh"

namespace idet {

namespace {

constexpr int kThreads = 256;

// One thread per entry, grid-stride. The primes of the batch sit in shared
// memory; each entry is reduced for all of them.
__global__ void k_reduce(const int64_t *__restrict__ A, int64_t n, int64_t lda,
                         const ModP *__restrict__ mods, int W,
                         int32_t *__restrict__ R) {
    extern __shared__ ModP sm_mods[];
    for (int w = threadIdx.x; w < W; w += blockDim.x) sm_mods[w] = mods[w];
    __syncthreads();
    const int64_t total = n * n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += stride) {
        int64_t i = e / n, j = e - i * n;
        int64_t a = A[i * lda + j];
        for (int w = 0; w < W; ++w) R[(int64_t)w * total + e] = red_bal(a, sm_mods[w]);
    }
}

// Zigzag code of an entry, 2a for a >= 0 and -2a - 1 for a < 0: its maximum
// over a matrix tells both the largest magnitude and whether every entry
// lies in the int32 range [-2^31, 2^31 - 1] (maximum <= 2^32 - 1).
__device__ __forceinline__ unsigned long long zigzag(int64_t a) {
    return ((unsigned long long)a << 1) ^ (unsigned long long)(a >> 63);
}

// One block per row: sum of squares (double) and the maximum zigzag code.
__global__ void k_row_stats(const int64_t *__restrict__ A, int64_t n, int64_t lda,
                            double *__restrict__ rowsq,
                            unsigned long long *__restrict__ amax) {
    __shared__ double s_sum[kThreads / 32];
    __shared__ unsigned long long s_max[kThreads / 32];
    const int64_t i = blockIdx.x;
    double acc = 0.0;
    unsigned long long mx = 0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        int64_t a = A[i * lda + j];
        unsigned long long m = zigzag(a);
        double d = (double)a;
        acc += d * d;
        mx = m > mx ? m : mx;
    }
    for (int o = 16; o; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = t > mx ? t : mx;
    }
    if ((threadIdx.x & 31) == 0) {
        s_sum[threadIdx.x >> 5] = acc;
        s_max[threadIdx.x >> 5] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        unsigned long long m = 0;
        for (int k = 0; k < kThreads / 32; ++k) {
            t += s_sum[k];
            m = s_max[k] > m ? s_max[k] : m;
        }
        // Upper bound: every product and addition above is rounded to
        // nearest, relative error < (n + 2) 2^-53 < 2^-30 for n < 2^20.
        rowsq[i] = t * (1.0 + 0x1p-30);  // upward margin >> rounding error
        atomicMax(amax, m);
    }
}

// Column sums of squares (double, same upward margin as the rows): one
// thread per column, rows streamed (coalesced across the warp).
__global__ void k_col_stats(const int64_t *__restrict__ A, int64_t n, int64_t lda,
                            double *__restrict__ colsq) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double acc = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double d = (double)A[i * lda + j];
        acc += d * d;
    }
    colsq[j] = acc * (1.0 + 0x1p-30);
}

// Row and column sums of squares and max |a_ij| for a batch of matrices,
// one CTA per matrix (rows by warps, columns by threads; same upward margin
// as the single-matrix kernels).
__global__ void k_stats_multi(const StatJob *__restrict__ jobs) {
    const StatJob J = jobs[blockIdx.x];
    const int64_t n = J.n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long mx = 0;
    for (int64_t i = warp; i < n; i += kThreads / 32) {
        double acc = 0.0;
        for (int64_t j = lane; j < n; j += 32) {
            const int64_t a = J.A[i * n + j];
            const unsigned long long m = zigzag(a);
            const double d = (double)a;
            acc += d * d;
            mx = m > mx ? m : mx;
        }
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) J.rowsq[i] = acc * (1.0 + 0x1p-30);
    }
    for (int o = 16; o; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = t > mx ? t : mx;
    }
    if (lane == 0) atomicMax(J.amax, mx);
    for (int64_t j = threadIdx.x; j < n; j += kThreads) {
        double acc = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            const double d = (double)J.A[i * n + j];
            acc += d * d;
        }
        J.colsq[j] = acc * (1.0 + 0x1p-30);
    }
}

__global__ void k_to_int32(const int64_t *__restrict__ A, int64_t n, int64_t lda,
                           int32_t *__restrict__ A32) {
    const int64_t total = n * n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += stride) {
        int64_t i = e / n, j = e - i * n;
        A32[e] = (int32_t)A[i * lda + j];
    }
}

template <class T>
__global__ void k_narrow(const int64_t *__restrict__ A, int64_t n, int64_t lda, T *__restrict__ out,
                         int64_t ldo) {
    const int64_t total = n * ldo;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        int64_t i = e / ldo, j = e - i * ldo;
        out[e] = j < n ? (T)A[i * lda + j] : (T)0;
    }
}

int grid_for(int64_t total) {
    int64_t g = (total + kThreads - 1) / kThreads;
    if (g > 148 * 16) g = 148 * 16;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

int launch_row_stats(const int64_t *A, int64_t n, int64_t lda, double *rowsq,
                     unsigned long long *amax, cudaStream_t s) {
    IDET_CUDA_TRY(cudaMemsetAsync(amax, 0, sizeof(unsigned long long), s));
    k_row_stats<<<(unsigned)n, kThreads, 0, s>>>(A, n, lda, rowsq, amax);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

int launch_stats_multi(const StatJob *jobs_dev, int count, cudaStream_t s) {
    if (count <= 0) return IDET_OK;
    k_stats_multi<<<count, kThreads, 0, s>>>(jobs_dev);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

int launch_col_stats(const int64_t *A, int64_t n, int64_t lda, double *colsq, cudaStream_t s) {
    k_col_stats<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(A, n, lda, colsq);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

int launch_to_int32(const int64_t *A, int64_t n, int64_t lda, int32_t *A32,
                    cudaStream_t s) {
    k_to_int32<<<grid_for(n * n), kThreads, 0, s>>>(A, n, lda, A32);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

int launch_narrow(const int64_t *A, int64_t n, int64_t lda, void *out, int64_t ldo, int bytes,
                  cudaStream_t s) {
    const int g = grid_for(n * ldo);
    if (bytes == 1)
        k_narrow<int8_t><<<g, kThreads, 0, s>>>(A, n, lda, (int8_t *)out, ldo);
    else if (bytes == 2)
        k_narrow<int16_t><<<g, kThreads, 0, s>>>(A, n, lda, (int16_t *)out, ldo);
    else
        k_narrow<int32_t><<<g, kThreads, 0, s>>>(A, n, lda, (int32_t *)out, ldo);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

int launch_reduce(const int64_t *A, int64_t n, int64_t lda, const ModP *mods,
                  int W, int32_t *R, cudaStream_t s) {
    if (W <= 0) return IDET_OK;
    k_reduce<<<grid_for(n * n), kThreads, sizeof(ModP) * W, s>>>(A, n, lda, mods,
                                                                 W, R);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

}  // namespace idet
