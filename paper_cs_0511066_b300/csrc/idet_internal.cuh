// Internal declarations shared by the CUDA translation units of libidet.
//
// Residues are stored "balanced": an element of Z/p is kept as the int32 in
// [-(p-1)/2, (p-1)/2] (p odd). Two prime classes are used:
//   * CRA primes, 2^20 < p < 2^21: |residue| < 2^20, products < 2^40, so
//     thousands of products can be summed exactly in int64 before a
//     reduction (delayed reduction);
//   * the lift prime, 2^30 < p < 2^31: |residue| < 2^30, products < 2^60,
//     so at most 4 products are summed before a fold.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <atomic>
#include <functional>
#include <mutex>
#include <vector>

#include "../../include/idet.h"

namespace idet {

// ---------------------------------------------------------------------------
// Modular arithmetic (device and host)

struct ModP {
    uint32_t p;      // odd prime, p < 2^31
    uint32_t half;   // (p - 1) / 2
    uint64_t m;      // floor((2^64 - 1) / p): Barrett multiplier
    int64_t off;     // a multiple of p with off >= 2^62
};

inline ModP make_mod(uint32_t p) {
    ModP M;
    M.p = p;
    M.half = (p - 1) / 2;
    M.m = ~0ull / p;
    M.off = (int64_t)(((1ull << 62) / p + 1) * p);
    return M;
}

// Balanced representative of s mod p, for |s| < 2^62.
// u = s + off lies in [0, 2^63 + p); Barrett with m = floor((2^64-1)/p)
// gives q in {floor(u/p) - 1, floor(u/p)}, so u - q p lies in [0, 2p).
__device__ __forceinline__ int32_t red_bal(int64_t s, const ModP &M) {
    uint64_t u = (uint64_t)(s + M.off);
    uint64_t q = __umul64hi(u, M.m);
    uint64_t r = u - q * (uint64_t)M.p;
    if (r >= M.p) r -= M.p;
    return (r > M.half) ? (int32_t)((int64_t)r - (int64_t)M.p) : (int32_t)r;
}

// Non-negative representative in [0, p).
__device__ __forceinline__ uint32_t red_pos(int64_t s, const ModP &M) {
    uint64_t u = (uint64_t)(s + M.off);
    uint64_t q = __umul64hi(u, M.m);
    uint64_t r = u - q * (uint64_t)M.p;
    if (r >= M.p) r -= M.p;
    return (uint32_t)r;
}

__device__ __forceinline__ int32_t mul_bal(int32_t a, int32_t b, const ModP &M) {
    return red_bal((int64_t)a * (int64_t)b, M);
}

// Inverse of a (nonzero mod p) by the extended Euclidean algorithm;
// returns the balanced representative.
__host__ __device__ inline int32_t inv_bal(int64_t a, uint32_t p) {
    int64_t r0 = (int64_t)p, r1 = a % (int64_t)p;
    if (r1 < 0) r1 += p;
    int64_t t0 = 0, t1 = 1;
    while (r1 != 0) {
        int64_t q = r0 / r1, t;
        t = r0 - q * r1; r0 = r1; r1 = t;
        t = t0 - q * t1; t0 = t1; t1 = t;
    }
    t0 %= (int64_t)p;
    if (t0 < 0) t0 += p;
    if (t0 > (int64_t)(p - 1) / 2) t0 -= p;
    return (int32_t)t0;
}

// ---------------------------------------------------------------------------
// Error plumbing

struct Status {
    int code = IDET_OK;
    const char *what = nullptr;
};

void set_last_error(const char *fmt, ...);

#define IDET_CUDA_TRY(expr)                                                   \
    do {                                                                      \
        cudaError_t _e = (expr);                                              \
        if (_e != cudaSuccess) {                                              \
            ::idet::set_last_error("%s:%d %s: %s", __FILE__, __LINE__, #expr, \
                                   cudaGetErrorString(_e));                   \
            return IDET_ERR_CUDA;                                             \
        }                                                                     \
    } while (0)

#define IDET_TRY(expr)                  \
    do {                                \
        int _rc = (expr);               \
        if (_rc != IDET_OK) return _rc; \
    } while (0)

// Raises a kernel's dynamic shared-memory limit to the most the device
// allows (opt-in limit less the kernel's static shared memory). It is always
// the same value, so host threads launching concurrently cannot lower it
// under one another's launches, as per-call sizes would. Defined in api.cu.
int allow_max_smem(const void *kernel);

// ---------------------------------------------------------------------------
// Device workspace: allocations made through the user-installed allocator
// (or cudaMallocAsync on the call's stream), released in LIFO order when the
// Workspace goes out of scope.

// Set by threads that must not call a user allocator (the serving
// workers): their workspaces use cudaMallocAsync on their own stream.
extern thread_local bool t_native_alloc;
// SMs that persistent kernels launched from this thread leave free (one
// while a single-CTA reconstruction runs beside them on another stream).
extern thread_local int t_reserve_sms;

class Workspace {
  public:
    explicit Workspace(cudaStream_t s);
    ~Workspace();
    // Returns IDET_OK or IDET_ERR_NOMEM; *ptr is 256-byte aligned.
    int alloc(void **ptr, size_t bytes);
    template <class T> int alloc_n(T **ptr, size_t count) {
        return alloc((void **)ptr, count * sizeof(T) + 16);
    }
    cudaStream_t stream() const { return stream_; }

  private:
    int raw_alloc(void **ptr, size_t bytes);
    cudaStream_t stream_;
    bool native_;
    std::vector<void *> ptrs_;
    // requests below kDirect are carved from chunks of kChunk bytes (one
    // allocator call per chunk instead of one per request)
    static constexpr size_t kDirect = (size_t)4 << 20, kChunk = (size_t)32 << 20;
    char *chunk_ = nullptr;
    size_t chunk_left_ = 0;
};

// Counter of kernel launches made by this library (for the benchmark's
// launch accounting); incremented by every launcher.
extern std::atomic<unsigned long long> g_launches;
inline void count_launch(unsigned k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// ---------------------------------------------------------------------------
// Kernel launchers (defined in the .cu files)

// k_reduce.cu ---------------------------------------------------------------
// Entries accepted by the int64 entry points: the int32 range
// [-2^31, 2^31 - 1]. zz is the maximum zigzag code reported by the
// statistics kernels; on success *amax = max |a_ij| (at most 2^31).
inline bool entry_range(unsigned long long zz, unsigned long long *amax) {
    *amax = (zz + 1) >> 1;
    return zz <= 0xffffffffull;
}
// Row statistics of an int64 matrix: rowsq[i] = sum_j A_ij^2 (double,
// rounded upward by a relative 2^-30 margin), amax[0] = the maximum zigzag
// code of the entries (2a for a >= 0, -2a - 1 for a < 0); decode it with
// entry_range above.
int launch_row_stats(const int64_t *A, int64_t n, int64_t lda, double *rowsq,
                     unsigned long long *amax, cudaStream_t s);
// colsq[j] = sum_i A_ij^2 (double, rounded upward).
int launch_col_stats(const int64_t *A, int64_t n, int64_t lda, double *colsq, cudaStream_t s);
// A -> int8/int16/int32 copy (bytes = 1, 2, 4) with leading dimension ldo
// >= n, zero padded; entries must fit the type.
int launch_narrow(const int64_t *A, int64_t n, int64_t lda, void *out, int64_t ldo, int bytes,
                  cudaStream_t s);
// A (int64, entries in the int32 range) -> int32 copy with leading dimension n.
int launch_to_int32(const int64_t *A, int64_t n, int64_t lda, int32_t *A32,
                    cudaStream_t s);
// R[w] = A mod mods[w] (balanced), w < W; R has W * n * n entries (ld n).
int launch_reduce(const int64_t *A, int64_t n, int64_t lda, const ModP *mods,
                  int W, int32_t *R, cudaStream_t s);

// k_lu.cu -----------------------------------------------------------------
struct LUState {
    uint32_t det;    // running product of pivots mod p, in [0, p)
    int32_t neg;     // parity of row swaps
    int32_t dead;    // 1 once a column had no pivot: det = 0 mod p
    int32_t pad;
};
// A (matrix, prime) job of the batched small LU.
struct LUSmallJob {
    int32_t *R;      // n x n residues, ld n, factored in place; or null:
    const int64_t *A64;  // the int64 entries (n x n, ld n), reduced on load
    int32_t n, pad;
    ModP mod;
    LUState *st;
    uint32_t *det;   // out: det mod p in [0, p)
};
// Batched whole-matrix LU in shared memory, one CTA per job (n <= 192).
int lu_small_multi(const LUSmallJob *jobs_dev, int count, int max_n, cudaStream_t s);
// Jobs of the batched Chinese remaindering and rational reconstruction.
struct CraJob {
    const uint32_t *primes, *residues;
    int32_t *digits;
    int32_t count, pad;
};
struct RRJob {
    const int64_t *z;
    int32_t m, hN, hD, den_cap;
    uint32_t *den;
    int32_t *info;
    uint32_t p, pad;
};
int launch_cra_multi(const CraJob *jobs_dev, int count, cudaStream_t s);
// k_batch.cu: one CTA per lifting job.
struct LiftJob {
    const int32_t *A, *C;   // n rows of ld int32 entries (zero padded)
    const int64_t *b;
    const int32_t *u;       // projection vector (may be null)
    int64_t *r;             // out: r_m
    int64_t *z;             // out: m projections u . x_i (may be null)
    int32_t *digits;        // out: m x n digits (may be null)
    int32_t n, ld, m, pad;
    ModP mod;
    uint64_t pinv;
};
int launch_lift_multi(const LiftJob *jobs_dev, int count, int max_ld, cudaStream_t s);
// Whole-matrix elimination by an 8-CTA cluster per job: mode 0 det mod p,
// mode 1 A^{-1} mod p (det = 1 on success, 0 if singular mod p).
struct ElimJob {
    const int64_t *A;     // n x n, leading dimension lda (int64 entries)
    int64_t lda;
    int32_t n, ld;        // ld: row length of Cinv (mode 1)
    ModP mod;
    int32_t *Cinv;        // mode 1 output
    uint32_t *det;        // det mod p (mode 0) or invertibility flag (mode 1)
    int32_t *A32;         // mode 1, optional: A as int32, n rows of ld (zero padded)
};
int launch_elim_cluster(const ElimJob *jobs_dev, int count, int max_n, int mode, cudaStream_t s);
bool elim_cluster_fits(int n);

// CUDA-graph replay of a batched phase (graph.cu): the job arrays (blobs)
// are copied into a fixed device buffer and record(device pointers, stream)
// issues the phase's launches; the sequence is captured per (key, blob
// sizes) on the second occurrence and replayed afterwards.
struct JobBlob {
    const void *data;
    size_t bytes;
};
int run_phase_graph(cudaStream_t s, uint64_t key, const std::vector<JobBlob> &blobs,
                    const std::function<int(const std::vector<const void *> &, cudaStream_t)> &record);
// Row and column statistics of many int64 matrices in one launch (one CTA
// per matrix): rowsq/colsq/amax as in launch_row_stats / launch_col_stats.
struct StatJob {
    const int64_t *A;  // n x n, ld n
    int64_t n;
    double *rowsq, *colsq;
    unsigned long long *amax;
};
int launch_stats_multi(const StatJob *jobs_dev, int count, cudaStream_t s);

// Autotuner table (tune.cu): the tuned choice for order n and prime class.
bool tuned_lookup(int64_t n, int prime_bits, idet_tuned *out);

// Multi-word entries (k_mp.cu): sign x magnitude of L base-2^32 limbs.
int launch_reduce_mp(const uint32_t *mag, const int8_t *sgn, int64_t n, int L, const ModP *mods,
                     int W, int32_t *R, cudaStream_t s);
int launch_mp_stats(const uint32_t *mag, const int8_t *sgn, int64_t n, int L, double *E,
                    double *rowl2, double *coll2, unsigned int *maxbits, cudaStream_t s);
int launch_mp_planes(const uint32_t *mag, const int8_t *sgn, int64_t n, int L, int T, int64_t ldp,
                     int16_t *planes, cudaStream_t s);
struct MpLiftArgs {
    const int32_t *C;        // A^{-1} mod p, n rows of ldc
    int64_t ldc, n;
    const int16_t *planes;   // T x n x ldp signed base-2^15 digits of A
    int T;
    int64_t ldp;
    const int32_t *u;        // projection vector
    int32_t *x, *rm, *rd;    // x_i; r mod p; residual digits n x len
    int len;
    int32_t *digits;         // lifting digits, row it = x_it
    int64_t *z;              // z[it] = u . x_it (zeroed by the caller)
    int32_t *info;
    ModP mod;
    uint32_t pinv15;         // p^{-1} mod 2^15
};
int launch_mp_step(const MpLiftArgs &a, int it, cudaStream_t s);
int launch_ratrecon_multi(const RRJob *jobs_dev, int count, int max_m, cudaStream_t s);
// Factor W residue matrices R[w] (n x n, ld n) in place: PA = LU mod p_w with
// the first-nonzero pivot rule. perm (W*n, may be null) receives the row
// permutation; det_out[w] = det mod p_w in [0, p_w). wide = the primes are
// of the 31-bit class.
int lu_factor_batched(int32_t *R, int64_t n, const ModP *mods_dev,
                      const ModP *mods_host, int W, bool wide, int nb,
                      int32_t *perm, uint32_t *det_out, int update_path,
                      Workspace &ws);
// Inverse of A mod p from its LU (R, perm as produced above with W = 1):
// out (n rows of ld_out >= n, columns n .. ld_out - 1 zeroed) receives
// A^{-1} mod p, balanced; Y (n x n) is scratch and must not overlap out.
int lu_inverse(const int32_t *R, const int32_t *perm, int64_t n,
               const ModP &mod_host, const ModP *mod_dev, bool wide, int nb,
               int32_t *Y, int32_t *out, int64_t ld_out, Workspace &ws);

// k_gemm_tc.cu: C <- C - A B mod p on the tensor cores (21-bit primes,
// K <= 32), path = IDET_PATH_I8, IDET_PATH_BF16 or IDET_PATH_F64.
// tcgen05 bf16-limb trailing update (k_gemm_tc05.cu); scratch holds
// tc05_scratch_bytes(n, W) bytes for any M, N <= n. tc05_check_error
// synchronises s and reports a bounded wait that gave up.
// L = 3 limbs for 21-bit primes, 5 for 31-bit primes.
size_t tc05_scratch_bytes(int64_t n, int W, int L);
int gemm_sub_tc05(const int32_t *A, int64_t lda, int64_t sA, const int32_t *B, int64_t ldb,
                  int64_t sB, int32_t *C, int64_t ldc, int64_t sC, int M, int N, int K,
                  const ModP *mods, const LUState *st, int W, void *scratch, cudaStream_t s,
                  int L);
int tc05_check_error(cudaStream_t s);
// scratch: tc_scratch_bytes(n, W, path) bytes (the packed limb tiles of A and
// B^T for any M, N <= n, K <= 128); tc_check_error synchronises s and
// reports a bounded wait for a tile copy that gave up.
size_t tc_scratch_bytes(int64_t n, int W, int path);
int tc_check_error(cudaStream_t s);
int gemm_sub_tc(int path, const int32_t *A, int64_t lda, int64_t sA, const int32_t *B, int64_t ldb,
                int64_t sB, int32_t *C, int64_t ldc, int64_t sC, int M, int N, int K,
                const ModP *mods, const LUState *st, int W, void *scratch, cudaStream_t s);

// k_lift.cu ---------------------------------------------------------------
// Held while a grid-synchronised lifting kernel runs: two of them on
// different streams could each hold part of the SMs and wait for the other.
extern std::mutex g_coop_mu;
// Two timing events destroyed with the scope, also on error returns.
struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    EventPair() = default;
    EventPair(const EventPair &) = delete;
    EventPair &operator=(const EventPair &) = delete;
    ~EventPair() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

struct LiftArgs {
    const int32_t *Cinv;   // A^{-1} mod p, balanced, n rows of ld entries
    const int64_t *b;      // right-hand side, n
    const int32_t *u;      // projection vector, n (may be null)
    int64_t n;
    int32_t m;             // number of digits to produce (per right-hand side)
    ModP mod;
    uint64_t pinv;         // p^{-1} mod 2^64
    int32_t *digits;       // m x n (row i = digit vector x_i), may be null
    int64_t *zproj;        // m projections u . x_i, may be null
    int64_t *r;            // n: residual r_m (the two-product kernel always
                           // writes it; the one-product kernel only when the
                           // digits are kept), may be null then
    uint64_t amax;         // max |a_ij|; 0 = unknown (two-product kernel)
    int32_t nrhs;          // right-hand sides lifted together: 1 (0 reads as
                           // 1) or 2, the second given by b2/digits2/...
    const int64_t *b2;
    int32_t *digits2;
    int64_t *zproj2;
    int64_t *r2;
};
// What a lift ran: path 0 the two-product kernel (k_lift.cu), 1 the
// one-product kernel (k_lifte.cu); setup = forming E and y_0; steps = the
// persistent kernel's launch, its steps and algorithmic bytes (E, or C and A,
// once per step).
struct LiftInfo {
    int path, steps;
    float ms_setup, ms_steps;
    double bytes;
};
// Anar: A as int8/int16/int32 (abytes = 1, 2, 4), n rows of ld entries;
// Cinv rows also have ld entries; ld must be a multiple of 16. Chooses the
// one-product kernel when n a.amax < 2^32 - 2 (lift_e_applies).
int launch_lift(const LiftArgs &a, const void *Anar, int abytes, int64_t ld, Workspace &ws,
                int *timed_out, float *ms = nullptr, LiftInfo *info = nullptr);
// k_lifte.cu: the one-product lift (x_i = y_i mods p, y_{i+1} = (y_i - x_i)/p
// - E x_i with E = (C A - I)/p); applies when n amax < 2^32 - 2.
bool lift_e_applies(int64_t n, uint64_t amax);
int launch_lift_e(const LiftArgs &a, const void *Anar, int abytes, int64_t ld, Workspace &ws,
                  int *timed_out, float *ms, LiftInfo *info);

// k_bignum.cu ---------------------------------------------------------------
// Device big integers: little-endian uint32 limbs with an explicit length.
struct BigDev {
    uint32_t *w;
    int32_t cap;
};
// Garner mixed-radix digits with balanced digits (symmetric range) for a
// wave of new primes appended after `count` existing ones; see k_bignum.cu.
int launch_cra_append(const uint32_t *primes, const uint32_t *residues,
                      int32_t *digits, int start, int count, int32_t *info,
                      cudaStream_t s);
// residues_out[k] = res_in[k] * K^{-1} mod primes[k] (K as limbs); skip[k]=1
// where K = 0 mod primes[k].
int launch_div_by_K(const uint32_t *Klimbs, int Klen, const uint32_t *primes,
                    const uint32_t *res_in, uint32_t *res_out, int32_t *skip,
                    int count, cudaStream_t s);
// Mixed radix (balanced digits) -> two's complement limbs, then times K.
int launch_mixed_to_int(const uint32_t *primes, const int32_t *digits,
                        int count, const uint32_t *Klimbs, int Klen,
                        uint32_t *out, int out_cap, int32_t *out_info,
                        cudaStream_t s);
// Rational reconstruction of the p-adic number with base-p lifting sums z
// (int64, m of them, |z_i| < 2^59): numerator below p^hN, denominator below
// p^hD; den receives the denominator's base-p digits. info[0]: 0 ok,
// 1 no fraction within the bounds, 2/4 capacity; info[1]: digits of den.
// With ainit (alen digits) the first operand is ainit instead of p^m; with
// hN = 0 the extended Euclid then runs to the zero remainder and den receives
// |cofactor of b| = ainit / gcd(ainit, b).
int launch_ratrecon(const int64_t *z, int m, uint32_t p, int hN, int hD, uint32_t *den,
                    int den_cap, int32_t *info, Workspace &ws, const uint32_t *ainit = nullptr,
                    int alen = 0);
// The same reconstruction (without ainit) with the denominator in binary:
// den receives its 32-bit limbs; info[0] as above, info[1]: limbs of den,
// info[2]: its bit length, info[3]: its leading 31 bits. 2^30 < p < 2^31.
// The numbers live in shared memory: callers check ratrecon_bin_fits first
// (about m <= 9,000 base-p digits) and use launch_ratrecon otherwise.
bool ratrecon_bin_fits(int m, int hN, int hD);
int launch_ratrecon_bin(const int64_t *z, int m, uint32_t p, int hN, int hD, uint32_t *den,
                        int den_cap, int32_t *info, Workspace &ws);
// k_lif.cu: exact lcm of denominators (see there).
int launch_lif_check(const int32_t *digits, int64_t n, int m, const uint32_t *D, int dlen,
                     uint32_t p, int h, int32_t *flag, cudaStream_t s);
int launch_mul_radix(const uint32_t *a, int la, const uint32_t *b, int lb, uint32_t p,
                     uint32_t *out, int cap, int32_t *out_len, cudaStream_t s);
int launch_gather_col(const int32_t *digits, int64_t n, int m, int64_t j, int64_t *z,
                      cudaStream_t s);
// k_bonus.cu: lcm of two radix-p numbers (digits in [0, p)) into workspace;
// and the extended bonus pi~_2 = s~^2 / gcd(det(R N), s~^2) of Section 3.2
// from the digits of two lifted solutions (dig: [2][m][n]), R (2 x n int64,
// device) and s~ (radix-p digits), with p^m > 2 |det(R N)|.
int lcm_radix(const uint32_t *a, int la, const uint32_t *b, int lb, uint32_t p, Workspace &ws,
              uint32_t **out, int *lout);
int bonus_pi2(const int32_t *dig, int64_t n, int m, uint32_t p, const int64_t *R,
              const uint32_t *sdig, int slen, Workspace &ws, uint32_t **pi, int *plen);
// Base-p digits -> base-2^32 limbs (out_len receives the limb count).
int launch_radix_to_binary(const uint32_t *dig, int len, uint32_t p, uint32_t *out, int cap,
                           int32_t *out_len, cudaStream_t s);

}  // namespace idet

namespace idet {
// Whole-matrix LU (n <= 192) writing only into the given buffers.
int lu_small_into(int32_t *R, int n, const ModP *mods_dev, int W, LUState *st,
                  uint32_t *det_out, cudaStream_t s);
}  // namespace idet
