/*
 * idet.h -- C ABI of libidet, a CUDA (sm_103a) implementation of the
 * data-parallel path of Dumas & Urbanska, "An introspective algorithm for
 * the integer determinant": multi-prime LU over Z/p (Section 2.1, Alg. 2.1),
 * Dixon p-adic lifting for the largest invariant factor s_n (Section 2.2),
 * and Chinese remaindering of det(A)/s_n with early termination (Alg. 2.1,
 * Alg. 4.1 with i_max = 1, as run in Section 5.1).
 *
 * Conventions shared by every entry point:
 *   - Matrices are dense, row-major, n x n, with leading dimension lda >= n
 *     (in elements). Entries are int64 values in the int32 range
 *     -2^31 <= a_ij <= 2^31 - 1.
 *     Orders above IDET_MAX_ORDER (65536) are rejected with IDET_ERR_ARG
 *     before any device work (their sizes would overflow the byte counts).
 *   - on_device = 0: pointers are host memory; the library copies them.
 *     on_device = 1: pointers are device memory of the current device.
 *   - stream is a cudaStream_t (passed as void*; NULL = legacy default
 *     stream). Calls are synchronous with respect to the host: they return
 *     after their results are written.
 *   - Inputs are never modified. Output buffers are owned by the caller.
 *   - Device workspace is allocated per call with the allocator installed by
 *     idet_set_allocator, or cudaMallocAsync/cudaFreeAsync on the stream.
 *   - Return value: IDET_OK (0) or one of the IDET_ERR_* codes below;
 *     idet_last_error() gives a message for the calling thread's last error.
 *   - Results are exact integers. int_det is correct with probability at
 *     least 1 - 2^log2_epsilon (Alg. 2.1 ensures 1 - epsilon), or always when
 *     certify = 1 (reconstruction past twice the Hadamard bound, Lemma 2.1(i)).
 *     A reconstruction stopped by the bound runs 40 bits past 2H and checks
 *     |r| <= H; a violation means a modular determinant was wrong and the
 *     call returns IDET_ERR_INTERNAL instead of a value.
 */
#ifndef IDET_H
#define IDET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define IDET_OK 0
#define IDET_MAX_ORDER 65536  /* largest accepted n, every entry point */
#define IDET_ERR_ARG 1        /* n < 0, null pointer, lda < n, entry too large */
#define IDET_ERR_BUFFER 2     /* output capacity too small; nlimbs = needed  */
#define IDET_ERR_SINGULAR 3   /* det(A) = 0 where a nonsingular A is needed  */
#define IDET_ERR_NOMEM 4      /* device workspace could not be allocated     */
#define IDET_ERR_TIMEOUT 5    /* a bounded device wait gave up               */
#define IDET_ERR_CUDA 6       /* a CUDA call failed                          */
#define IDET_ERR_INTERNAL 7   /* a reconstruction failed its own check       */

/* Trailing-update (Schur complement) arithmetic of the LU over Z/p. */
#define IDET_PATH_AUTO 0      /* TC05 for 21-bit primes, INT64 for 31-bit    */
#define IDET_PATH_INT64 1     /* CUDA cores, int64 delayed reduction         */
#define IDET_PATH_I8 2        /* signed 7-bit int8 limbs, int32 accumulation */
#define IDET_PATH_F64 3       /* FP64 with delayed reduction below 2^53      */
#define IDET_PATH_BF16 4      /* 7-bit limbs exact in bf16, mma.sync        */
#define IDET_PATH_TC05 5      /* 7-bit limbs exact in bf16, tcgen05.mma with
                                 accumulators in tensor memory                */

/* Big integer: sign in {-1, 0, +1}, magnitude in little-endian base-2^32
 * limbs. The caller provides limbs[0..cap). On IDET_ERR_BUFFER, nlimbs is set
 * to the number of limbs needed and nothing else is written. */
typedef struct {
    int32_t sign;
    uint32_t nlimbs;
    uint32_t cap;
    uint32_t *limbs;
} idet_int;

typedef struct {
    double log2_epsilon;   /* error tolerance epsilon = 2^log2_epsilon (-64) */
    uint64_t seed;         /* seeds the prime sampling and the random b, u   */
    int32_t certify;       /* 1: no early termination; stop at prod p >= 2H  */
    int32_t update_path;   /* IDET_PATH_*                                    */
    int32_t nb;            /* LU panel width, 0 = default                    */
    int32_t wave;          /* primes factored per batch, 0 = default         */
    int32_t lif;           /* 1 (default): Alg. 4.1 with i_max = 1; 0: CRA
                              only (Alg. 2.1 on det(A)); 2 (idet_int_det
                              only, else as 1): solve first, then Alg. 2.1
                              on det(A)/K without early termination, up to
                              prod p >= 2H/K (the LIF method of Fig. 2)      */
    int32_t prime_bits;    /* CRA prime class: 21 (primes in (2^20, 2^21)) or
                              31 (primes in (2^30, 2^31)); 0 = default: 21
                              for idet_int_det, 31 for idet_int_det_mp      */
    int32_t inject_fault;  /* failure-detection tests only (0 = off): k > 0
                              adds 1 to det(A) mod p for the k-th CRA prime
                              factored (idet_int_det, idet_int_det_mp), a
                              wrong modular determinant made on the host    */
    int32_t i_max;         /* idet_int_det, lif = 1: solves of Alg. 4.1's
                              inner loop. 0 or 1: one solve (K = s~_n);
                              2: two solves in one block lift and the
                              extended bonus of Section 3.2, K = lcm(s~_n,
                              pi~_2) (the i_max = 2 column of Table 1)    */
    int32_t reserved[4];
} idet_opts;

typedef struct {
    int32_t primes_used;       /* CRA primes factored (det mod p computed)   */
    int32_t primes_in_cra;     /* primes the final reconstruction used      */
    int32_t et_stop;           /* 1 early termination, 2 bound, 0 neither   */
    int32_t lift_iters;        /* Dixon iterations (0 when no solve ran)    */
    int32_t lift_timed_out;
    int32_t log2_K;            /* bits of the factor K = s~_n found          */
    double log2_H;             /* log2 of the Hadamard bound used           */
    double ms_lu;              /* device time of the multi-prime LU         */
    double ms_lift;            /* wall time of the solve: lift and
                                  reconstruction (and, in the speculative
                                  order, the first CRA wave beside the
                                  reconstruction)                           */
    double ms_cra;             /* device time of reconstruction steps       */
    double ms_total;
    uint64_t launches;         /* kernels launched by the call              */
    double ms_lift_kernel;     /* device time of the lifting kernel alone   */
    double lift_bytes;         /* its algorithmic bytes: the matrices it
                                  reads once per step (E: 4 n^2 per step;
                                  C and A: (4 + bytes(a_ij)) n^2)           */
    double lu_macs;            /* (2/3) n^3 per factored CRA prime: the
                                  modular MACs of the work timed by ms_lu   */
    double ms_inverse;         /* LU + inverse mod the lifting prime        */
    double ms_rr;              /* rational reconstruction kernel(s) (with the
                                  speculative order the first CRA wave, in
                                  ms_lu, runs beside it; idet_int_det_batch:
                                  included in ms_lift_kernel)                */
    double inverse_macs;       /* modular MACs timed by ms_inverse: the LU
                                  (2n^3/3) and the triangular solves (n^3/6
                                  forward, the inverse of L being lower
                                  triangular, n^3/2 backward) per lifting
                                  prime; 2n^3 per system in batches        */
    double ms_lift_setup;      /* forming E = (C A - I)/p and y_0 = C b for
                                  the one-product lift (0 otherwise)        */
    int32_t lift_path;         /* 1: one-product lift (E), 0: C and A       */
    int32_t pad_;
} idet_stats;

/* Fill *opts with the defaults. */
void idet_default_opts(idet_opts *opts);

/* Message for the calling thread's last error (never NULL). */
const char *idet_last_error(void);

/* Optional device allocator used for all workspace (e.g. a framework's
 * caching allocator). alloc returns NULL on failure. Pass NULLs to restore
 * the cudaMallocAsync default. Not thread-safe with concurrent calls. */
typedef void *(*idet_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*idet_free_fn)(void *ptr, void *stream, void *ctx);
void idet_set_allocator(idet_alloc_fn alloc, idet_free_fn free_, void *ctx);

/* Kernels launched by this library since load (monotone counter). */
uint64_t idet_launch_count(void);

/* Failure-detection tests: the cycle limit of every bounded wait in the
 * lifting kernels (grid-wide barriers, copy-ring waits). cycles <= 0
 * restores the default (about two seconds of SM clock). A wait that runs out
 * ends the kernel cleanly (its copies drained) and the call returns
 * IDET_ERR_TIMEOUT with stats->lift_timed_out set; later calls are
 * unaffected. Process-wide; not for use while lifts are running. */
void idet_set_wait_limit(int64_t cycles);

/*
 * det(A): "computing the determinant of an integer matrix A" (Abstract,
 * Section 1), by Alg. 4.1 with i_max = 1 (Section 5.1): Alg. 2.1 on det(A)
 * for the Lemma 2.1(iv) number of primes, then one Dixon solve giving a
 * factor K of s_n (Section 2.2), then Alg. 2.1 on det(A)/K reusing the
 * residues already computed (Section 4). opts may be NULL (defaults), stats
 * may be NULL. det receives the exact determinant.
 * Order of the steps: for n < 500 (and with certify, lif != 1, i_max = 2 or
 * 31-bit CRA primes) the first CRA wave comes first and the solve follows
 * only without early termination (from n = 1500 the LU and inverse mod the
 * lifting prime run beside the wave on a second stream). From n = 500 on the
 * order is speculative: inverse and lift first, then the first wave on a
 * second stream while the rational reconstruction (one CTA) runs; the wave's
 * early-termination verdict still wins (its determinant is returned, K is
 * not used). Set the environment variable IDET_ET_FIRST to keep the wave
 * first at every n. The result does not depend on the order.
 * Order limit of the solve: the lifting kernel stages its vector in shared
 * memory (4 n bytes per right-hand side when n max|a_ij| < 2^32, else the
 * vector and one row of A^{-1} mod p, 12 n bytes), so with lif = 1 or 2 n is
 * at most about 50,000 (25,000 with i_max = 2), or 19,000 for the largest
 * entries, on a GPU with 227 KB of shared memory per block; larger n return
 * IDET_ERR_ARG. lif = 0 (Alg. 2.1 alone) has no such limit.
 */
int idet_int_det(const int64_t *A, int64_t n, int64_t lda, int32_t on_device,
                 const idet_opts *opts, void *stream, idet_int *det,
                 idet_stats *stats);

/*
 * det(A) for entries of many words: a_ij = A_sign[i n + j] * sum_l
 * A_limbs[(i n + j) L + l] 2^(32 l), A_sign in {-1, 0, 1} (0 only with a zero
 * magnitude), 1 <= L <= 64 limbs, n <= 65536, both arrays row-major without
 * padding, on the host or (on_device) the device. Same method as
 * idet_int_det (Alg. 4.1 with i_max = 1), CRA primes of opts->prime_bits
 * (default 31: for entries this large log_l H approaches the 21-bit pool),
 * and an output-sensitive Dixon lift: it stops at the first length m at
 * which a reconstructed denominator D passes the certificate (every
 * D x_j mod p^m small, and the Hadamard-free bound n max|a| p^h + D max|b| <
 * p^m / 2 making A y = D b hold over Z), so m follows the size of s~_n and of
 * the numerators, not H. Errors as idet_int_det; stats->lift_iters is m and
 * stats->log2_K the bits of the factor s~_n found.
 */
int idet_int_det_mp(const uint32_t *A_limbs, const int8_t *A_sign, int64_t n, int32_t L,
                    int32_t on_device, const idet_opts *opts, void *stream, idet_int *det,
                    idet_stats *stats);

/*
 * s~_n for the right-hand side b: the lcm of the denominators of the entries
 * of A^{-1} b, computed by Dixon p-adic lifting and rational reconstruction
 * (Section 2.2, LargestInvariantFactor with one solve). b has n int64
 * entries with |b_i| < 2^62 (on_device applies to b too). The value is exact
 * and deterministic given (A, b). IDET_ERR_SINGULAR if A is singular.
 */
int idet_largest_invariant_factor(const int64_t *A, int64_t n, int64_t lda,
                                  const int64_t *b, int32_t on_device,
                                  const idet_opts *opts, void *stream,
                                  idet_int *s);

/*
 * det(A) mod p_k for a list of primes (the modular step of Alg. 2.1, "compute
 * det(A) mod p_i using the LU factorization modulo p_i", Section 2.1).
 * primes: host array of nprimes odd primes, each with 2^20 < p < 2^21 or
 * 2^30 < p < 2^31 (all of one class). det_mod: host array receiving the
 * residues in [0, p_k). The pivot is the first nonzero entry at or below the
 * diagonal.
 */
int idet_det_mod_primes(const int64_t *A, int64_t n, int64_t lda,
                        int32_t on_device, const uint32_t *primes,
                        int32_t nprimes, const idet_opts *opts, void *stream,
                        uint32_t *det_mod);

/*
 * LU over Z/p of one prime: factors (host, n*n int32 in [0, p): strict lower
 * part L with unit diagonal, upper part U) and perm (host, n int32: row of A
 * now at position i) with PA = LU. Returns IDET_ERR_SINGULAR (factors then
 * partial) when a column has no nonzero pivot. Same prime classes as above.
 */
int idet_lu_mod_prime(const int64_t *A, int64_t n, int64_t lda,
                      int32_t on_device, uint32_t p, const idet_opts *opts,
                      void *stream, uint32_t *lu, int32_t *perm);

/*
 * The Dixon p-adic lifting iteration of Section 2.2 for one prime p with
 * 2^30 < p < 2^31: C = A^{-1} mod p; r_0 = b; x_i = C r_i mod p in the
 * balanced range [-(p-1)/2, (p-1)/2]; r_{i+1} = (r_i - A x_i)/p. Writes the m
 * digit vectors to digits (host, m*n int32, row i = x_i) and r_m to
 * residual (host, n int64). |b_i| < 2^62 (IDET_ERR_ARG otherwise).
 * IDET_ERR_SINGULAR if A is singular mod p.
 */
int idet_dixon_digits(const int64_t *A, int64_t n, int64_t lda,
                      const int64_t *b, uint32_t p, int32_t m,
                      int32_t on_device, void *stream, int32_t *digits,
                      int64_t *residual);

/*
 * The block form of the same iteration: nrhs = 1 or 2 right-hand sides
 * lifted together, so that each step reads the lifting matrix once for all
 * of them (Section 6: grouping the solvings into block iterations;
 * Theorem 2.2(ii) and (iii) take r = 2 solves). B holds the right-hand sides
 * as nrhs consecutive vectors of n int64 (|b_i| < 2^62; device memory when
 * on_device). digits (host, nrhs * m * n int32) receives the digit vectors
 * [k][i][j] = x_i of right-hand side k; residual (host, nrhs * n int64) the
 * r_m. stats (may be NULL): lift_iters = m, lift_path, ms_lift_kernel (the
 * stepping kernel), ms_lift_setup and lift_bytes (the bytes of the lifting
 * matrices read by the stepping kernel, counted once per step).
 */
int idet_dixon_digits_block(const int64_t *A, int64_t n, int64_t lda,
                            const int64_t *B, int32_t nrhs, uint32_t p, int32_t m,
                            int32_t on_device, void *stream, int32_t *digits,
                            int64_t *residual, idet_stats *stats);

/*
 * Chinese remaindering in the symmetric range (Section 2.1): the unique r
 * with r = residues[k] mod primes[k] for all k and
 * -floor(M/2) <= r < ceil(M/2), M = prod primes (odd primes, pairwise
 * distinct, < 2^31). Host arrays. trailing (may be NULL) receives the
 * number k of early-termination agreements r_{t-k} = ... = r_t at the end of
 * the sequence (Alg. 2.1).
 */
int idet_crt_symmetric(const uint32_t *residues, const uint32_t *primes,
                       int32_t count, void *stream, idet_int *r,
                       int32_t *trailing);

/*
 * The extended bonus of Section 3.2 for k = 2 right-hand sides: with
 * X = A^{-1} B, s~ the lcm of the denominators of the entries of X (Section
 * 2.2), N = s~ X and a 2 x n matrix R,
 *     pi~_2 = s~^2 / gcd(det(R N), s~^2),
 * a factor of s_n s_{n-1}, the product of the two largest invariant factors
 * of A (Lemma 3.5). B and R are host arrays of two rows of n int64 each
 * (|b|, |r| < 2^62); A follows the conventions (on_device applies to A
 * only). Both solves run as one block lift; det(R N) comes from the p-adic
 * digits, the lift being long enough that p^m > 2 |det(R N)|. pi receives
 * pi~_2 and s_tilde receives s~. IDET_ERR_SINGULAR if A is singular.
 */
int idet_extended_bonus(const int64_t *A, int64_t n, int64_t lda, const int64_t *B,
                        const int64_t *R, int32_t on_device, const idet_opts *opts, void *stream,
                        idet_int *pi, idet_int *s_tilde);

/*
 * Alg. 2.1's loop (Section 2.1) run over a given stream of modular
 * determinants: residues[k] = det mod primes[k] for k = 0 .. count-1 in the
 * order the primes were drawn (odd, distinct, < 2^31; host arrays). The
 * mixed-radix digits of r_0, r_1, ... are formed on the device; the loop
 * stops at the first k where the on-the-fly bound of Lemma 2.1(iii), with
 * |P| = pool_size and l = 2^log2_l, falls below epsilon = 2^log2_epsilon
 * (not with certify = 1), or where prod p reaches 2H 2^40 with
 * H = 2^log2_H. *stop_index receives k (-1: no stop within the stream) and
 * *reason 1 (early termination), 2 (bound) or 3 (bound reached, but
 * |r| > H: a residue is wrong), 0 if no stop. r receives the value
 * reconstructed from the residues up to the stop (all of them if none), in
 * the symmetric range. This is the rule idet_int_det applies to its own
 * residues.
 */
int idet_cra_early_termination(const uint32_t *residues, const uint32_t *primes, int32_t count,
                               double log2_H, double log2_epsilon, double log2_l,
                               double pool_size, int32_t certify, void *stream, idet_int *r,
                               int32_t *stop_index, int32_t *reason);

/*
 * det(A_i) for a batch of independent matrices of possibly different orders:
 * the same method as idet_int_det (Alg. 4.1 with i_max = 1), with the
 * batch's work fused across matrices -- the LUs of all (matrix, prime) pairs
 * with n_i <= 192 in one launch, one launch for all the Dixon solves (one
 * CTA per matrix), one for all reconstructions and one per round of Chinese
 * remaindering -- in the spirit of Section 6's remark that the LUs of a CRA
 * step and several p-adic liftings are independent and can run in parallel.
 * A[i] (n[i] x n[i], leading dimension lda[i]) follow the conventions above;
 * dets[i] receives det(A_i) (IDET_ERR_BUFFER if any dets[i].cap is too
 * small: that entry's nlimbs is set and the call fails). stats (may be NULL)
 * receives totals over the batch.
 */
int idet_int_det_batch(int32_t count, const int64_t *const *A, const int64_t *n,
                       const int64_t *lda, int32_t on_device, const idet_opts *opts,
                       void *stream, idet_int *dets, idet_stats *stats);

/*
 * det(A) mod p_k for small matrices WITHOUT allocating device memory. The
 * paper has no counterpart: this serves callers that cannot call cudaMalloc
 * or any allocator -- for instance code that runs where a framework owns all
 * device memory through its own pool, or a context that forbids allocation
 * while it is being set up. The result equals idet_det_mod_primes on the
 * same arguments.
 *
 * Limits: 1 <= n <= 128, 1 <= nprimes <= 32, |a_ij| < 2^62; primes as for
 * idet_det_mod_primes (all in (2^20, 2^21) or all in (2^30, 2^31)); sizes,
 * entries or primes beyond the limits return IDET_ERR_ARG with a message
 * (for device input the entries are checked on the device, and det_mod is
 * then left unwritten). A (n x n, leading
 * dimension lda) is host memory when on_device = 0, device memory when 1;
 * primes and det_mod are host arrays of nprimes entries.
 *
 * Scratch: a fixed area of about 2.2 MiB that lives in the library image as
 * a __device__ array; every GPU that loads the library holds it until the
 * process exits. The first call on a device looks up the area's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture. All calls share the one area and it keeps
 * the last call's contents (each call writes everything it reads): calls
 * whose GPU work overlaps -- on different streams or host threads -- race
 * and must be serialised by the caller. The call is synchronous.
 */
int idet_det_mod_primes_noalloc(const int64_t *A, int64_t n, int64_t lda,
                                int32_t on_device, const uint32_t *primes,
                                int32_t nprimes, void *stream, uint32_t *det_mod);

/* ------------------------------------------------------------------------
 * Serving with continuous batching. A server owns `slots` worker threads,
 * each with its own CUDA stream on the current device. idet_submit copies
 * the matrix (host memory, entries in [-2^31, 2^31 - 1]) and queues the job; workers
 * admit queued jobs first-in first-out whenever a slot and device memory are
 * free: each job is charged an estimate of its device footprint against
 * hbm_budget (0 = 80% of the free memory at creation); a job that does not
 * fit lets later ones that fit go ahead, until it has been overtaken
 * 2 slots + 2 times, after which it waits for the memory. A worker taking a
 * job with n <= small_n also takes the other queued jobs with n <= small_n
 * that fit (max_batch in all) and runs them as one batch
 * (idet_int_det_batch); larger jobs run alone (idet_int_det). Jobs on
 * different workers overlap on the device. Each result is the value
 * idet_int_det returns for that matrix with the server's opts.
 */
typedef struct idet_server idet_server;

typedef struct {
    int32_t status;        /* the job's result code (IDET_*)                 */
    int32_t batched;       /* jobs in the group it ran in (1 = alone)        */
    int32_t worker;        /* worker (stream) that ran it                    */
    int32_t pad;
    double ms_queue;       /* submit -> start, host clock                   */
    double ms_run;         /* start -> end                                  */
    double ms_latency;     /* submit -> end                                 */
    double t_start_ms;     /* start and end on a monotonic host clock       */
    double t_end_ms;
    idet_stats stats;      /* of its run (of the whole group when batched)  */
} idet_job_info;

typedef struct {
    int32_t queued, running, max_running, pad;
    uint64_t bytes_in_use, budget, admitted, completed, groups;
} idet_server_stats;

/* NULL on error (idet_last_error). opts may be NULL. hbm_budget = 0: 80 %
 * of the device memory free at creation. The workers allocate from the
 * device's default stream-ordered memory pool, whose release threshold is
 * raised so that freed workspace is kept for the next job (a per-process
 * setting of that pool). */
idet_server *idet_server_create(size_t hbm_budget, int32_t slots, int32_t small_n,
                                int32_t max_batch, const idet_opts *opts);
/* IDET_ERR_NOMEM if the job alone exceeds the budget. */
int idet_submit(idet_server *srv, const int64_t *A, int64_t n, int64_t lda, uint64_t *ticket);
/* Waits up to timeout_ms (< 0: no limit) for the job. IDET_OK: det written,
 * ticket released. IDET_ERR_TIMEOUT: not finished yet. IDET_ERR_BUFFER:
 * det->nlimbs set to the size needed, job kept. A job error is returned as
 * its code (ticket released). info may be NULL. Several threads may poll
 * the same ticket: one collects the result, the others then get
 * IDET_ERR_ARG (ticket already collected). */
int idet_poll(idet_server *srv, uint64_t ticket, int32_t timeout_ms, idet_int *det,
              idet_job_info *info);
void idet_server_info(idet_server *srv, idet_server_stats *out);
/* Finishes the submitted jobs, then stops the workers and frees the server
 * with any results not collected. No other call on srv may be in progress
 * (a thread blocked in idet_poll included) or follow. */
void idet_server_destroy(idet_server *srv);

/* ------------------------------------------------------------------------
 * Autotuner for the multi-prime LU. idet_autotune times, for order n and
 * the prime class prime_bits (21 or 31), the reduction plus LU of W primes
 * on a random matrix with entries of entry_bits bits (2..32) generated on the
 * device, for every update path of the class (21-bit: TC05, INT64, BF16,
 * I8; 31-bit: TC05, INT64), panel width nb in {16, 32} and W in {4, 8, 16}, and
 * records the fastest per prime in a process-wide table keyed by (n bucket
 * of a quarter octave, prime bits). Calls with update_path = AUTO, nb = 0
 * or wave = 0 then use the entry of the nearest bucket within one octave
 * (else the built-in defaults). out may be NULL. The table is saved to and
 * loaded from JSON files (idet_tuning_load merges). Not thread-safe with
 * concurrent idet_autotune calls on the same stream.
 */
typedef struct {
    int32_t update_path;   /* IDET_PATH_* of the winner                     */
    int32_t nb;            /* panel width                                   */
    int32_t wave;          /* primes per wave                               */
    int32_t pad;
    double ms_per_prime;   /* reduction + LU time per prime of the winner   */
} idet_tuned;

int idet_autotune(int64_t n, int32_t prime_bits, int32_t entry_bits, void *stream,
                  idet_tuned *out);
int idet_tuning_save(const char *path);
int idet_tuning_load(const char *path);
void idet_tuning_clear(void);

#ifdef __cplusplus
}
#endif

#endif /* IDET_H */
