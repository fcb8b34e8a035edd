// det(A) mod p_k for small matrices without any device memory allocation.
//
// Some callers cannot allocate device memory: plugins hosted by a framework
// that owns all device memory through its own pool, or processes whose
// allocator is locked down (for determinism, or while a context is being
// set up). This entry point serves them by using a fixed scratch area that
// lives in the library image itself: a file-scope __device__ array, present
// on every GPU that loads the library until the process exits. It has no
// counterpart in the paper; it is the same computation as
// idet_det_mod_primes restricted to small sizes. Every call shares the one
// area, so calls whose GPU work overlaps race; each call writes every
// scratch byte it reads, and returns only after its work has finished.
//
// Limits: n <= kMaxN = 128 and at most kMaxW = 32 primes per call, so the
// scratch is 32 * 128 * 128 * 4 bytes of residues (2 MiB) plus the staged
// matrix (128 KiB), per-prime parameters and the row statistics that check
// the entries' size.
//
// In host code the array's name only stands for it; the device address is
// obtained once per device with cudaGetSymbolAddress, with that device
// current, by the first call made on it, which should therefore come before
// any stream capture.
#include <cstring>
#include <mutex>

#include "idet_internal.cuh"

namespace idet {

namespace {

constexpr int kMaxN = 128;
constexpr int kMaxW = 32;
constexpr size_t kResBytes = sizeof(int32_t) * kMaxW * kMaxN * kMaxN;
constexpr size_t kMatBytes = sizeof(int64_t) * kMaxN * kMaxN;
constexpr size_t kModOff = kResBytes + kMatBytes;
constexpr size_t kStateOff = kModOff + 1024;
constexpr size_t kDetOff = kStateOff + 1024;
constexpr size_t kStatOff = kDetOff + 1024;  // row sums of squares, then the zigzag max
constexpr size_t kScratchBytes = kStatOff + sizeof(double) * kMaxN + 256;
static_assert(sizeof(ModP) * kMaxW <= 1024, "parameter area");
static_assert(sizeof(LUState) * kMaxW <= 1024, "state area");

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {};

// Device address of the scratch on the current device (set up on first use).
int scratch_address(unsigned char **out) {
    int dev = 0;
    IDET_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_last_error("device ordinal %d out of range", dev);
        return IDET_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_last_error("cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
            return IDET_ERR_CUDA;
        }
        g_addr[dev] = (unsigned char *)p;
    }
    *out = g_addr[dev];
    return IDET_OK;
}

// A prime of the class (2^30, 2^31) when wide, else (2^20, 2^21).
bool prime_ok(uint32_t p, bool wide) {
    if (!(p & 1)) return false;
    if (wide ? !(p > (1u << 30) && p < (1u << 31)) : !(p > (1u << 20) && p < (1u << 21)))
        return false;
    for (uint32_t d = 3; (uint64_t)d * d <= p; d += 2)
        if (p % d == 0) return false;
    return true;
}

}  // namespace

}  // namespace idet

using namespace idet;

extern "C" int idet_det_mod_primes_noalloc(const int64_t *A, int64_t n, int64_t lda,
                                           int32_t on_device, const uint32_t *primes,
                                           int32_t nprimes, void *stream, uint32_t *det_mod) {
    if (n < 1 || n > kMaxN || lda < n || !A || !primes || !det_mod || nprimes < 1 ||
        nprimes > kMaxW) {
        set_last_error("idet_det_mod_primes_noalloc: need 1 <= n <= %d, 1 <= nprimes <= %d, "
                       "lda >= n and non-null pointers",
                       kMaxN, kMaxW);
        return IDET_ERR_ARG;
    }
    ModP mods[kMaxW];
    const bool wide = primes[0] > (1u << 30);
    for (int i = 0; i < nprimes; ++i) {
        if (!prime_ok(primes[i], wide)) {
            set_last_error("primes must be primes of one class: all in (2^20, 2^21) or all in "
                           "(2^30, 2^31)");
            return IDET_ERR_ARG;
        }
        mods[i] = make_mod(primes[i]);
    }
    // the residue reduction needs |a_ij| < 2^62; host input is checked here,
    // device input by the statistics kernel below (before any result is
    // written)
    if (!on_device) {
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = 0; j < n; ++j) {
                const int64_t v = A[i * lda + j];
                if (v >= (1ll << 62) || v <= -(1ll << 62)) {
                    set_last_error("idet_det_mod_primes_noalloc: entries must satisfy "
                                   "|a_ij| < 2^62");
                    return IDET_ERR_ARG;
                }
            }
    }
    unsigned char *base = nullptr;
    IDET_TRY(scratch_address(&base));
    cudaStream_t s = (cudaStream_t)stream;
    int32_t *R = (int32_t *)base;
    int64_t *Ad = (int64_t *)(base + kResBytes);
    ModP *md = (ModP *)(base + kModOff);
    LUState *st = (LUState *)(base + kStateOff);
    uint32_t *dd = (uint32_t *)(base + kDetOff);
    double *rowsq = (double *)(base + kStatOff);
    unsigned long long *zz = (unsigned long long *)(base + kStatOff + sizeof(double) * kMaxN);
    // stage A (compact, ld = n) and the prime parameters; every scratch byte
    // read below is written first in this call
    IDET_CUDA_TRY(cudaMemcpy2DAsync(Ad, sizeof(int64_t) * n, A, sizeof(int64_t) * lda,
                                    sizeof(int64_t) * n, n,
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                    s));
    IDET_CUDA_TRY(cudaMemcpyAsync(md, mods, sizeof(ModP) * nprimes, cudaMemcpyHostToDevice, s));
    IDET_TRY(launch_row_stats(Ad, n, n, rowsq, zz, s));
    IDET_TRY(launch_reduce(Ad, n, n, md, nprimes, R, s));
    IDET_TRY(lu_small_into(R, (int)n, md, nprimes, st, dd, s));
    uint32_t res[kMaxW];
    unsigned long long hz = 0;
    IDET_CUDA_TRY(cudaMemcpyAsync(res, dd, sizeof(uint32_t) * nprimes, cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaMemcpyAsync(&hz, zz, sizeof(hz), cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaStreamSynchronize(s));
    // zigzag code 2|a| or 2|a| - 1: |a| < 2^62 iff the code is below 2^63 - 1
    if (hz >= (1ull << 63) - 1) {
        set_last_error("idet_det_mod_primes_noalloc: entries must satisfy |a_ij| < 2^62");
        return IDET_ERR_ARG;
    }
    memcpy(det_mod, res, sizeof(uint32_t) * nprimes);
    return IDET_OK;
}
