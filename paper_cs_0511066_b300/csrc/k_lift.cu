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
// Layout and schedule. One CTA per SM owns a contiguous block of rows of C
// and of A. As many of those rows as fit stay in shared memory for the whole
// launch ("resident"); the others are streamed every iteration. Streaming is
// warp-specialised: warp 31 of each CTA is a producer that copies streamed
// rows with bulk asynchronous copies (cp.async.bulk) into a ring of shared
// memory slots guarded by full/empty mbarriers; warps 0..30 consume resident
// rows and ring slots. The streamed data does not depend on the iteration's
// vector, so the producer runs ahead across phases and across the grid
// barriers, keeping memory busy while the consumers wait. The vector operand
// (r mod p, pre-split into 16-bit halves, then x) is staged in shared memory
// at the start of each phase. A is stored in the narrowest of
// int8/int16/int32 that holds its entries; rows are zero padded to a
// multiple of 16 elements.
//
// Exactness:
//  * x_i: |C_jk| < 2^30 and r mod p is split as hi * 2^16 + lo with
//    0 <= lo < 2^16, |hi| < 2^14, so both partial sums stay below
//    n 2^46 < 2^62 for n < 2^16, in int64.
//  * r_{i+1}: the true value is an integer of magnitude below
//    |r_i|/p + n ||A|| < 2^62, equal to (r_i - A x_i) p^{-1} modulo 2^64; so
//    products and sums are taken modulo 2^64 (wrapping) and multiplied by
//    the inverse of p modulo 2^64 (exact division).
//
// Every wait is bounded (lift_common.cuh): a grid barrier or an mbarrier
// that does not complete sets err, all warps leave, and the producer first
// waits for the copies it has issued.
#include <algorithm>
#include <cstdlib>

#include <atomic>
#include <mutex>

#include "idet_internal.cuh"
#include "lift_common.cuh"

namespace idet {

namespace {

constexpr int kLiftThreads = 1024;
constexpr int kConsumers = 31;  // warps 0..30
constexpr int kConsThreads = kConsumers * 32;
constexpr int kProducer = 31;   // warp 31
constexpr int kRingMax = 16;
struct LiftGeom {
    int64_t ld;   // padded row length (multiple of 16)
    int64_t rpc;  // rows per CTA
    int cC, cA;   // rows of C / A resident in shared memory per CTA
    int S;        // ring slots (0: no streaming)
    int keep;     // streamed rows per iteration copied with an L2 evict_last hint
};

using namespace lift;

__device__ __forceinline__ void cons_sync() { lift::cons_sync<kConsThreads>(); }

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

// x phase: sum_k C[row][k] v[k] mod p; the row is in shared memory and v is
// staged as 16-bit halves lo, hi (two 32x32->64 multiply-adds per element).
__device__ __forceinline__ int32_t dot_c(const int4 *__restrict__ crow,
                                         const int4 *__restrict__ vlo,
                                         const int4 *__restrict__ vhi, int64_t nq, int lane,
                                         const ModP &M) {
    int64_t lo = 0, hi = 0;
#pragma unroll 4
    for (int64_t q = lane; q < nq; q += 32) {
        const int4 c = crow[q];
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

// r phase: sum_k A[row][k] x[k] modulo 2^64; the row is in shared memory.
template <class TA>
__device__ __forceinline__ uint64_t dot_a(const typename Quad<TA>::V *__restrict__ arow,
                                          const int4 *__restrict__ v, int64_t nq, int lane) {
    uint64_t acc = 0;
#pragma unroll 4
    for (int64_t q = lane; q < nq; q += 32) {
        const typename Quad<TA>::V a = arow[q];
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
       int32_t *__restrict__ xcur, GridBar *gb, long long limit) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[kRingMax], empty[kRingMax];
    __shared__ int64_t s_z[kConsumers];
    __shared__ volatile unsigned int s_issued;  // copies issued so far
    using V = typename Quad<TA>::V;
    const int64_t n = a.n, ld = g.ld, nq = ld / 4;
    const ModP M = a.mod;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * g.rpc;
    const int64_t r1 = min(n, r0 + g.rpc);
    const int nrows = r1 > r0 ? (int)(r1 - r0) : 0;
    const int64_t slotB = 4 * ld;
    int4 *vlo = reinterpret_cast<int4 *>(smem);
    int4 *vhi = reinterpret_cast<int4 *>(smem + 4 * ld);
    unsigned char *ring = smem + 8 * ld;
    int32_t *cC = reinterpret_cast<int32_t *>(ring + g.S * slotB);
    TA *cA = reinterpret_cast<TA *>(ring + g.S * slotB + 4 * ld * g.cC);
    const int kc = min(g.cC, nrows), ka = min(g.cA, nrows);
    const int nsC = nrows - kc, nsA = nrows - ka;  // streamed rows per phase
    const int per_it = nsC + nsA;
    const unsigned G = gridDim.x;

    if (tid == 0) {
        s_issued = 0;
        for (int s = 0; s < g.S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // resident rows (all warps)
    {
        const int4 *src = reinterpret_cast<const int4 *>(a.Cinv + r0 * ld);
        int4 *dst = reinterpret_cast<int4 *>(cC);
        for (int64_t e = tid; e < (int64_t)kc * nq; e += kLiftThreads) dst[e] = __ldg(src + e);
        const int4 *srcA = reinterpret_cast<const int4 *>(Anar + r0 * ld);
        int4 *dstA = reinterpret_cast<int4 *>(cA);
        const int64_t qa = ld * (int64_t)sizeof(TA) / 16;
        for (int64_t e = tid; e < (int64_t)ka * qa; e += kLiftThreads) dstA[e] = __ldg(srcA + e);
    }
    __syncthreads();

    if (warp == kProducer) {
        // ---- producer: stream rows kc.. of C and ka.. of A, every iteration
        if (lane == 0 && per_it > 0 && g.S > 0) {
            // The first g.keep streamed rows of every iteration are marked to
            // stay in L2 (evict_last), the others to leave it first, so that a
            // fixed subset of the streamed bytes is served by L2 each time
            // instead of the whole set cycling through it.
            const uint64_t pol_keep = policy_evict_last(), pol_pass = policy_evict_first();
            long long seq = 0;
            bool ok = true;
            for (int it = 0; it < a.m && ok; ++it) {
                for (int k = 0; k < per_it; ++k, ++seq) {
                    const int slot = (int)(seq % g.S);
                    const unsigned par = (unsigned)((seq / g.S) & 1) ^ 1u;
                    if (!mbar_wait(&empty[slot], par, gb, limit, seq, slot, it)) {
                        ok = false;
                        break;
                    }
                    const void *src;
                    unsigned bytes;
                    if (k < nsC) {
                        src = a.Cinv + (r0 + kc + k) * ld;
                        bytes = (unsigned)(4 * ld);
                    } else {
                        src = Anar + (r0 + ka + (k - nsC)) * ld;
                        bytes = (unsigned)(sizeof(TA) * ld);
                    }
                    mbar_expect_tx(&full[slot], bytes);
                    bulk_g2s(ring + slot * slotB, src, bytes, &full[slot],
                             k < g.keep ? pol_keep : pol_pass);
                    s_issued = (unsigned int)(seq + 1);
                }
            }
            // no copy may be in flight when the CTA exits
            drain_ring(full, g.S, seq);
        }
        return;
    }

    // ---- consumers (warps 0..30)
    for (int64_t i = r0 + tid; i < r1; i += kConsThreads) {
        int64_t bi = a.b[i];
        a.r[i] = bi;
        rm[i] = red_bal(bi, M);
    }
    unsigned bar = 0;
    if (!grid_sync<kConsThreads>(gb, (++bar) * G, limit)) return;
    long long seq_base = 0;
    bool fail = false;

    for (int it = 0; it < a.m; ++it) {
        // Phase 1: x = C (r mod p) mod p on this CTA's rows.
        {
            const int4 *src = reinterpret_cast<const int4 *>(rm);
            for (int64_t q = tid; q < nq; q += kConsThreads) {
                const int4 v = __ldcg(src + q);
                vlo[q] = make_int4(v.x & 0xffff, v.y & 0xffff, v.z & 0xffff, v.w & 0xffff);
                vhi[q] = make_int4(v.x >> 16, v.y >> 16, v.z >> 16, v.w >> 16);
            }
        }
        cons_sync();
        int64_t zpart = 0;
        for (int lr = warp; lr < nrows; lr += kConsumers) {
            const int64_t row = r0 + lr;
            int32_t x = 0;
            if (lr < kc) {
                x = dot_c(reinterpret_cast<const int4 *>(cC + (int64_t)lr * ld), vlo, vhi, nq,
                          lane, M);
            } else {
                const long long seq = seq_base + (lr - kc);
                const int slot = (int)(seq % g.S);
                if (!wait_issued(&s_issued, seq, gb, limit, slot, it) ||
                    !mbar_wait(&full[slot], (unsigned)((seq / g.S) & 1), gb, limit, seq, slot, it)) {
                    fail = true;
                    break;
                }
                x = dot_c(reinterpret_cast<const int4 *>(ring + slot * slotB), vlo, vhi, nq, lane,
                          M);
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[slot]);
            }
            if (lane == 0) {
                xcur[row] = x;
                if (a.digits) a.digits[(int64_t)it * n + row] = x;
                if (a.u) zpart += (int64_t)a.u[row] * x;
            }
        }
        seq_base += nsC;
        if (a.zproj) {
            if (lane == 0) s_z[warp] = zpart;
            cons_sync();
            if (tid == 0) {
                int64_t t = 0;
                for (int k = 0; k < kConsumers; ++k) t += s_z[k];
                if (t) atomicAdd((unsigned long long *)&a.zproj[it], (unsigned long long)t);
            }
        }
        if (fail) fail_once(gb, 3, 0, -1, -1, 0, it);
        if (!grid_sync<kConsThreads>(gb, (++bar) * G, limit)) return;

        // Phase 2: r <- (r - A x) / p on this CTA's rows.
        {
            const int4 *src = reinterpret_cast<const int4 *>(xcur);
            for (int64_t q = tid; q < nq; q += kConsThreads) vlo[q] = __ldcg(src + q);
        }
        cons_sync();
        for (int lr = warp; lr < nrows; lr += kConsumers) {
            const int64_t row = r0 + lr;
            uint64_t acc = 0;
            if (lr < ka) {
                acc = dot_a<TA>(reinterpret_cast<const V *>(cA + (int64_t)lr * ld), vlo, nq, lane);
            } else {
                const long long seq = seq_base + (lr - ka);
                const int slot = (int)(seq % g.S);
                if (!wait_issued(&s_issued, seq, gb, limit, slot, it) ||
                    !mbar_wait(&full[slot], (unsigned)((seq / g.S) & 1), gb, limit, seq, slot, it)) {
                    fail = true;
                    break;
                }
                acc = dot_a<TA>(reinterpret_cast<const V *>(ring + slot * slotB), vlo, nq, lane);
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[slot]);
            }
            if (lane == 0) {
                uint64_t diff = (uint64_t)__ldcg(a.r + row) - acc;
                int64_t rn = (int64_t)(diff * a.pinv);
                a.r[row] = rn;
                rm[row] = red_bal(rn, M);
            }
        }
        seq_base += nsA;
        if (fail) fail_once(gb, 3, 0, -1, -1, 0, it);
        if (!grid_sync<kConsThreads>(gb, (++bar) * G, limit)) return;
    }
}

std::atomic<long long> g_wait_cycles{0};


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
    const int64_t crow = 4 * ld, arow = (int64_t)sizeof(TA) * ld;
    const int64_t avail = (int64_t)smem_max - 8 * ld - 4096;
    LiftGeom g{};
    g.ld = ld;
    // Fewest CTAs with one row per consumer warp, if everything then fits in
    // shared memory (fewer CTAs make the grid barrier cheaper); otherwise all
    // SMs, a ring of streaming slots, and as many resident rows as fit.
    int64_t G = std::min<int64_t>(sms, (n + kConsumers - 1) / kConsumers);
    if (G < 1) G = 1;
    g.rpc = (n + G - 1) / G;
    if (g.rpc * (crow + arow) <= avail) {
        g.S = 0;
        g.cC = (int)g.rpc;
        g.cA = (int)g.rpc;
    } else {
        G = sms;
        g.rpc = (n + G - 1) / G;
        // ring depth: bytes in flight per SM; IDET_LIFT_SLOTS overrides (tuning)
        int want = 8;
        if (const char *e = getenv("IDET_LIFT_SLOTS")) want = atoi(e);
        g.S = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)kRingMax, (int64_t)want,
                                                           avail / crow}));
        const int64_t left = avail - g.S * crow;
        const int64_t cC = left > 0 ? std::min<int64_t>(g.rpc, left / crow) : 0;
        const int64_t cA = std::min<int64_t>(g.rpc, std::max<int64_t>(0, left - cC * crow) / arow);
        g.cC = (int)cC;
        g.cA = (int)cA;
        if (g.S * crow > avail) {
            set_last_error("lift: a row does not fit in shared memory (n too large)");
            return IDET_ERR_ARG;
        }
    }
    // L2 budget for the rows kept across iterations (IDET_LIFT_L2_MB, tuning)
    {
        double l2mb = 72.0;
        if (const char *e = getenv("IDET_LIFT_L2_MB")) l2mb = atof(e);
        const int64_t per_it = std::max<int64_t>(0, g.rpc - g.cC) + std::max<int64_t>(0, g.rpc - g.cA);
        const double row_bytes = (double)(crow + arow) / 2;
        const double total = (double)G * per_it * row_bytes;
        const double frac = total > 0 ? std::min(1.0, l2mb * 1048576.0 / total) : 0.0;
        g.keep = (int)(frac * per_it);
    }
    const size_t smem = (size_t)(8 * ld + g.S * crow + (int64_t)g.cC * crow + (int64_t)g.cA * arow);
    IDET_TRY(allow_max_smem((const void *)k_lift<TA>));
    int occ = 0;
    IDET_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_lift<TA>, kLiftThreads,
                                                                smem));
    if (occ < 1) {
        set_last_error("lift kernel does not fit on an SM");
        return IDET_ERR_INTERNAL;
    }
    const TA *Ap = (const TA *)Anar;
    long long limit = lift_wait_cycles();
    void *args[] = {(void *)&a,    (void *)&Ap, (void *)&g,    (void *)&rm,
                    (void *)&xcur, (void *)&gb, (void *)&limit};
    EventPair ev;
    if (ms) {
        IDET_CUDA_TRY(cudaEventCreate(&ev.a));
        IDET_CUDA_TRY(cudaEventCreate(&ev.b));
        IDET_CUDA_TRY(cudaEventRecord(ev.a, s));
    }
    // One grid-synchronised lift at a time in the process: two of them on
    // different streams could each hold part of the SMs and wait for the
    // other's. Held until the kernel has finished (stream synchronised below).
    std::unique_lock<std::mutex> coop(g_coop_mu);
    IDET_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)k_lift<TA>, dim3((unsigned)G),
                                              dim3(kLiftThreads), args, smem, s));
    count_launch();
    if (ms) {
        IDET_CUDA_TRY(cudaEventRecord(ev.b, s));
        IDET_CUDA_TRY(cudaEventSynchronize(ev.b));
        IDET_CUDA_TRY(cudaEventElapsedTime(ms, ev.a, ev.b));
    }
    GridBar hb{};
    IDET_CUDA_TRY(cudaMemcpyAsync(&hb, gb, sizeof(GridBar), cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaStreamSynchronize(s));
    if (timed_out) *timed_out = hb.err;
    if (hb.err) {
        set_last_error("lift: a bounded wait gave up (code %d, block %d warp %d seq %d slot %d "
                       "parity %d iteration %d; grid %d, S %d, cC %d, cA %d, rpc %d)",
                       hb.err, hb.info[0], hb.info[1], hb.info[2], hb.info[3], hb.info[4],
                       hb.info[5], (int)G, g.S, g.cC, g.cA, (int)g.rpc);
        return IDET_ERR_TIMEOUT;
    }
    return IDET_OK;
}

}  // namespace

std::mutex g_coop_mu;

long long lift_wait_cycles() {
    const long long v = g_wait_cycles.load(std::memory_order_relaxed);
    return v > 0 ? v : lift::kDefaultWaitCycles;
}

static int launch_lift_classic(const LiftArgs &a, const void *Anar, int abytes, int64_t ld,
                               Workspace &ws, int *timed_out, float *ms) {
    if (abytes == 1) return launch_lift_t<int8_t>(a, Anar, ld, ws, timed_out, ms);
    if (abytes == 2) return launch_lift_t<int16_t>(a, Anar, ld, ws, timed_out, ms);
    return launch_lift_t<int32_t>(a, Anar, ld, ws, timed_out, ms);
}

int launch_lift(const LiftArgs &a, const void *Anar, int abytes, int64_t ld, Workspace &ws,
                int *timed_out, float *ms, LiftInfo *info) {
    if (ld % 16 != 0) {
        set_last_error("lift: leading dimension must be a multiple of 16");
        return IDET_ERR_INTERNAL;
    }
    if (lift_e_applies(a.n, a.amax)) return launch_lift_e(a, Anar, abytes, ld, ws, timed_out, ms, info);
    // the two-product kernel, once per right-hand side
    float t0 = 0, t1 = 0;
    int to0 = 0, to1 = 0;
    int64_t *r_tmp = nullptr;
    LiftArgs a0 = a;
    if (!a0.r) {
        IDET_TRY(ws.alloc_n(&r_tmp, a.n));
        a0.r = r_tmp;
    }
    IDET_TRY(launch_lift_classic(a0, Anar, abytes, ld, ws, &to0, ms || info ? &t0 : nullptr));
    if (a.nrhs == 2 && to0 == 0) {
        LiftArgs a1 = a;
        a1.b = a.b2;
        a1.digits = a.digits2;
        a1.zproj = a.zproj2;
        a1.r = a.r2 ? a.r2 : r_tmp;
        if (!a1.r) {
            IDET_TRY(ws.alloc_n(&r_tmp, a.n));
            a1.r = r_tmp;
        }
        IDET_TRY(launch_lift_classic(a1, Anar, abytes, ld, ws, &to1, ms || info ? &t1 : nullptr));
    }
    if (timed_out) *timed_out = to0 ? to0 : to1;
    if (ms) *ms = t0 + t1;
    if (info) {
        info->path = 0;
        info->steps = a.m * (a.nrhs == 2 ? 2 : 1);
        info->ms_setup = 0;
        info->ms_steps = t0 + t1;
        info->bytes = (double)info->steps * (4.0 + abytes) * (double)a.n * (double)a.n;
    }
    return IDET_OK;
}

}  // namespace idet

extern "C" void idet_set_wait_limit(int64_t cycles) {
    idet::g_wait_cycles.store(cycles > 0 ? (long long)cycles : 0, std::memory_order_relaxed);
}
