// Multi-word integer steps of the path, on one CTA each:
//
//  * k_cra_append -- Chinese remaindering in the symmetric range (Section
//    2.1) by Garner's mixed-radix scheme with BALANCED digits: with
//    r = sum_i v_i prod_{j<i} p_j and every |v_i| <= (p_i - 1)/2, r lies in
//    [-(M-1)/2, (M-1)/2], M = prod p_i, which is the symmetric range of
//    Lemma 2.1 for odd M. Adding p_t gives
//        v_t = (d_t - r mod p_t) (M mod p_t)^{-1} mod p_t,
//    and r_t = r_{t-1} exactly when v_t = 0, which is the early-termination
//    agreement test of Alg. 2.1.
//  * k_div_by_K   -- d_k K^{-1} mod p_k, the residues of det(A)/K
//    (Section 2.3, "reconstruct only det(A)/s_n"), skipping p_k | K.
//  * k_mixed_to_int -- r from its mixed-radix digits, times K.
//  * k_ratrecon   -- rational reconstruction of a p-adic number (Section 2.2,
//    via Dixon's method): extended Euclid on (p^m, X) with Lehmer's
//    multi-step quotients, stopped at the first remainder below the
//    numerator bound; the cofactor is the denominator.
#include <climits>

#include "idet_internal.cuh"

namespace idet {

namespace {

// ---------------------------------------------------------------------------
// Garner CRT

constexpr int kCraThreads = 256;

__device__ __forceinline__ uint32_t mod_u64(uint64_t v, uint32_t p, uint64_t m) {
    uint64_t q = __umul64hi(v, m);
    uint64_t r = v - q * p;
    return (uint32_t)(r >= p ? r - p : r);
}

__device__ void cra_append_body(const uint32_t *__restrict__ primes,
                                const uint32_t *__restrict__ residues,
                                int32_t *__restrict__ digits, int start, int count) {
    __shared__ uint32_t s_sum[kCraThreads];
    __shared__ uint32_t s_prod[kCraThreads];
    const int tid = threadIdx.x;
    for (int t = start; t < start + count; ++t) {
        const uint32_t pt = primes[t];
        const uint64_t mt = ~0ull / pt;
        // chunk [beg, end) of the previous digits
        const int per = (t + kCraThreads - 1) / kCraThreads;
        const int beg = min(t, tid * per), end = min(t, beg + per);
        uint64_t acc = 0, prod = 1 % pt;
        for (int i = end - 1; i >= beg; --i) {
            const uint32_t pi = primes[i] % pt;
            int32_t v = digits[i];
            uint32_t vm = v >= 0 ? (uint32_t)v % pt : (pt - (uint32_t)(-(int64_t)v % pt)) % pt;
            acc = mod_u64((uint64_t)vm + (uint64_t)pi * acc, pt, mt);
            prod = mod_u64(prod * pi, pt, mt);
        }
        s_sum[tid] = (uint32_t)acc;
        s_prod[tid] = (uint32_t)prod;
        __syncthreads();
        if (tid == 0) {
            uint64_t r = 0, M = 1 % pt;
            for (int c = 0; c < kCraThreads; ++c) {
                r = mod_u64(r + (uint64_t)s_sum[c] * M, pt, mt);
                M = mod_u64(M * s_prod[c], pt, mt);
            }
            uint64_t d = residues[t] % pt;
            uint64_t diff = (d + pt - r) % pt;
            int32_t inv = inv_bal((int64_t)M, pt);
            uint64_t invp = inv < 0 ? (uint64_t)(inv + (int64_t)pt) : (uint64_t)inv;
            uint32_t v = mod_u64(diff * invp, pt, mt);
            digits[t] = v > (pt - 1) / 2 ? (int32_t)((int64_t)v - pt) : (int32_t)v;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kCraThreads)
k_cra_append(const uint32_t *__restrict__ primes, const uint32_t *__restrict__ residues,
             int32_t *__restrict__ digits, int start, int count) {
    cra_append_body(primes, residues, digits, start, count);
}

// One CTA per job of a batch: digits of residues mod primes, from scratch.
__global__ void __launch_bounds__(kCraThreads) k_cra_multi(const CraJob *__restrict__ jobs) {
    const CraJob j = jobs[blockIdx.x];
    cra_append_body(j.primes, j.residues, j.digits, 0, j.count);
}

// K mod p_k by Horner over the base-2^32 limbs, then d_k K^{-1}.
__global__ void k_div_by_K(const uint32_t *__restrict__ K, int Klen,
                           const uint32_t *__restrict__ primes,
                           const uint32_t *__restrict__ res_in, uint32_t *__restrict__ res_out,
                           int32_t *__restrict__ skip, int count) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const uint32_t p = primes[k];
    const uint64_t m = ~0ull / p;
    uint64_t acc = 0;
    for (int i = Klen - 1; i >= 0; --i) acc = mod_u64((acc << 32) | K[i], p, m);
    if (acc == 0) {
        skip[k] = 1;
        res_out[k] = 0;
        return;
    }
    skip[k] = 0;
    int32_t inv = inv_bal((int64_t)acc, p);
    uint64_t invp = inv < 0 ? (uint64_t)(inv + (int64_t)p) : (uint64_t)inv;
    res_out[k] = mod_u64((uint64_t)(res_in[k] % p) * invp, p, m);
}

// out (two's complement, out_cap limbs) = K * sum_i v_i prod_{j<i} p_j.
// info[0] = sign of the result, info[1] = limbs of |result|, info[2] = error.
// Single thread: used on the short digit sequences left after early
// termination, and once per certified reconstruction.
__global__ void k_mixed_to_int(const uint32_t *__restrict__ primes,
                               const int32_t *__restrict__ digits, int count,
                               const uint32_t *__restrict__ K, int Klen,
                               uint32_t *__restrict__ out, int out_cap,
                               uint32_t *__restrict__ tmp, int32_t *__restrict__ info) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    // tmp: two's complement accumulator with out_cap limbs
    for (int i = 0; i < out_cap; ++i) tmp[i] = 0;
    int len = 1;  // limbs in use (plus sign extension above)
    for (int t = count - 1; t >= 0; --t) {
        const uint64_t p = primes[t];
        // tmp = tmp * p (two's complement: multiply the full width)
        uint64_t carry = 0;
        int lim = min(out_cap, len + 2);
        for (int i = 0; i < lim; ++i) {
            uint64_t v = (uint64_t)tmp[i] * p + carry;
            tmp[i] = (uint32_t)v;
            carry = v >> 32;
        }
        // sign extension of the high part: if negative, the limbs above lim
        // must stay all-ones; recompute them from tmp[lim-1]
        uint32_t ext = (tmp[lim - 1] & 0x80000000u) ? 0xffffffffu : 0u;
        for (int i = lim; i < out_cap; ++i) tmp[i] = ext;
        // + v_t (sign extended)
        int64_t c = digits[t];
        for (int i = 0; i < out_cap && c != 0; ++i) {
            int64_t v = (int64_t)tmp[i] + c;
            tmp[i] = (uint32_t)v;
            c = v >> 32;
        }
        len = min(out_cap - 2, len + 1);
        while (len > 1 && tmp[len - 1] == ext && ((tmp[len - 2] & 0x80000000u) ? 0xffffffffu : 0u) == ext) --len;
        len = max(len, 1);
    }
    int neg = (tmp[out_cap - 1] & 0x80000000u) != 0;
    if (neg) {  // magnitude
        uint64_t c = 1;
        for (int i = 0; i < out_cap; ++i) {
            uint64_t v = (uint64_t)(~tmp[i]) + c;
            tmp[i] = (uint32_t)v;
            c = v >> 32;
        }
    }
    int rl = out_cap;
    while (rl > 0 && tmp[rl - 1] == 0) --rl;
    if (rl == 0) {
        info[0] = 0;
        info[1] = 0;
        info[2] = 0;
        return;
    }
    // out = K * |r|
    int total = Klen + rl;
    if (total > out_cap) {
        info[2] = total;
        return;
    }
    for (int i = 0; i < total; ++i) out[i] = 0;
    for (int i = 0; i < Klen; ++i) {
        uint64_t carry = 0;
        for (int j = 0; j < rl; ++j) {
            uint64_t v = (uint64_t)K[i] * tmp[j] + out[i + j] + carry;
            out[i + j] = (uint32_t)v;
            carry = v >> 32;
        }
        int k = i + rl;
        while (carry) {
            uint64_t v = (uint64_t)out[k] + carry;
            out[k] = (uint32_t)v;
            carry = v >> 32;
            ++k;
        }
    }
    while (total > 0 && out[total - 1] == 0) --total;
    info[0] = neg ? -1 : 1;
    info[1] = total;
    info[2] = 0;
}

// ---------------------------------------------------------------------------
// Rational reconstruction in radix p (one CTA of kRR threads).
//
// Numbers are little-endian digit vectors in [0, p), p the lift prime
// (2^30 < p < 2^31), with explicit lengths. The p-adic value X mod p^m needs
// no conversion (its digits are the normalised lifting digits) and
// Q = p^m is the digit 1 at position m. Quotients are found Lehmer-style
// from the two leading digits (Knuth, TAOCP vol. 2, 4.5.2, Algorithm L:
// a run of single-precision Euclid steps is accepted while the quotients of
// (u + A)/(v + C) and (u + B)/(v + D) agree), and applied to the full
// numbers as one 2x2 matrix. Bounds are powers of p: the reconstruction stops
// at the first remainder with at most hN digits (value < p^hN) and accepts a
// denominator of at most hD digits; uniqueness needs m >= hN + hD + 1.
//
// Layout and synchronisation: the four numbers (a, b and the cofactor
// magnitudes ta, tb) sit in shared memory; for an update over L digits every
// thread owns one contiguous chunk of them. Every thread reads the leading
// digits and derives the same Lehmer matrix, lengths and comparisons, so no
// value is broadcast: an iteration costs one barrier after those reads and the
// two of the carry exchange (settle below). Exchanging a and b exchanges
// pointers, not digits.

constexpr int kRT = 1024;  // threads of the radix conversion
constexpr int kRR = 256;   // threads of the reconstruction

struct Radix {
    uint32_t p;
    uint32_t mu;   // floor(2^62 / p), in (2^31, 2^32) for 2^30 < p < 2^31
    int64_t kp;    // ceil(2^61 / p)
    int64_t off;   // kp * p, in [2^61, 2^61 + p)
};

__device__ __forceinline__ Radix make_radix(uint32_t p) {
    Radix R;
    R.p = p;
    R.mu = (uint32_t)((1ull << 62) / p);
    R.kp = (int64_t)(((1ull << 61) + p - 1) / p);
    R.off = R.kp * (int64_t)p;
    return R;
}

// v = carry * p + digit with 0 <= digit < p, for |v| < 2^61 - 2^31 and
// 2^30 < p < 2^31 (Barrett): u = v + off lies in [0, 2^62), the estimate
// floor((u >> 30) mu / 2^32) is at most 2 below floor(u / p), and the
// remainder is fixed by at most two subtractions. Two 32-bit multiplies.
__device__ __forceinline__ uint32_t divmod_p(int64_t v, const Radix &R, int64_t &carry) {
    const uint64_t u = (uint64_t)(v + R.off);
    uint32_t q = __umulhi((uint32_t)(u >> 30), R.mu);
    uint64_t r = u - (uint64_t)q * R.p;
    if (r >= R.p) {
        r -= R.p;
        ++q;
    }
    if (r >= R.p) {
        r -= R.p;
        ++q;
    }
    carry = (int64_t)q - R.kp;
    return (uint32_t)r;
}

__device__ __forceinline__ void chunk_of(int len, int &beg, int &end) {
    const int per = (len + kRT - 1) / kRT;
    beg = min(len, (int)threadIdx.x * per);
    end = min(len, beg + per);
}

// The reconstruction's chunks: an odd stride puts the threads' digits of one
// step in distinct shared-memory banks.
template <int T = kRR>
__device__ __forceinline__ void rr_chunk(int len, int &beg, int &end) {
    const int per = ((len + T - 1) / T) | 1;
    beg = min(len, (int)threadIdx.x * per);
    end = min(len, beg + per);
}

template <int T = kRR>
struct RRCarry {
    int64_t co[4][T];   // carry out of each chunk, computed with carry-in 0
    int64_t co2[4][T];  // carries that rippled through a whole chunk
};

// Radix 2^31: v = carry * 2^31 + digit with 0 <= digit < 2^31 (floor
// division by a shift; any int64 v).
constexpr uint32_t kM31 = 0x7fffffffu;
__device__ __forceinline__ uint32_t norm31(int64_t v, int64_t &carry) {
    carry = v >> 31;
    return (uint32_t)v & kM31;
}

template <bool BIN>
__device__ __forceinline__ uint32_t norm(int64_t v, const Radix &R, int64_t &carry) {
    return BIN ? norm31(v, carry) : divmod_p(v, R, carry);
}

// The threads' chunks of NA numbers hold digits computed with carry-in 0 and
// carry-outs c[]; add to every chunk the carry-out of the chunk below it, so
// that all digits lie in [0, radix) (radix p, or 2^31 when BIN). Carries out
// of the top chunk are dropped: the numbers fit in the chunks' digits
// (reduction mod radix^len where that is the intent). One exchange settles
// every carry whose ripple ends inside the next chunk; a ripple through a
// whole chunk (digits all radix - 1, or all 0 for a borrow) takes further
// passes, each moving it at least one chunk up.
template <int NA, bool BIN = false, int T = kRR>
__device__ __forceinline__ void settle(uint32_t *const (&w)[NA], int beg, int end,
                                       const int64_t (&c)[NA], RRCarry<T> &K, const Radix &R) {
    const int tid = threadIdx.x;
#pragma unroll
    for (int q = 0; q < NA; ++q) K.co[q][tid] = c[q];
    __syncthreads();
    bool pend = false;
#pragma unroll
    for (int q = 0; q < NA; ++q) {
        int64_t cc = tid > 0 ? K.co[q][tid - 1] : 0;
        for (int k = beg; k < end && cc != 0; ++k)
            w[q][k] = norm<BIN>((int64_t)w[q][k] + cc, R, cc);
        if (beg >= end) cc = 0;
        K.co2[q][tid] = cc;
        pend |= cc != 0;
    }
    if (!__syncthreads_or(pend && tid != T - 1)) return;
    for (int pass = 0; pass < T; ++pass) {
        int64_t cin[NA];
#pragma unroll
        for (int q = 0; q < NA; ++q) cin[q] = tid > 0 ? K.co2[q][tid - 1] : 0;
        __syncthreads();
        pend = false;
#pragma unroll
        for (int q = 0; q < NA; ++q) {
            int64_t cc = cin[q];
            for (int k = beg; k < end && cc != 0; ++k)
                w[q][k] = norm<BIN>((int64_t)w[q][k] + cc, R, cc);
            if (beg >= end) cc = 0;
            K.co2[q][tid] = cc;
            pend |= cc != 0;
        }
        if (!__syncthreads_or(pend && tid != T - 1)) return;
    }
}

// r + c for a digit r in [0, p) and a carry |c| <= 2^30 + 1: the digit in
// [0, p), and c' = floor((r + c) / p) in {-1, 0, 1} added to the carry q of
// the next position.
__device__ __forceinline__ uint32_t add_carry(uint32_t r, int64_t c, uint32_t p, int64_t &q) {
    int64_t s = (int64_t)r + c;
    if (s < 0) {
        s += p;
        --q;
    } else if (s >= (int64_t)p) {
        s -= p;
        ++q;
    }
    return (uint32_t)s;
}

// (x, y) <- (A x + B y, C x + D y) on digits [0, La) and (tx, ty) <-
// (|A| tx + |B| ty, |C| tx + |D| ty) on [0, Lt); |A|..|D| < 2^28; all results
// are >= 0 and fit in their digits. Every position is split into digit and
// carry on its own (no dependence between positions); only the carry of the
// position below, at most 2^30 + 1 in magnitude, is then added, so the
// serial chain per position is one addition and compare.
__device__ void rr_lincomb(uint32_t *__restrict__ x, uint32_t *__restrict__ y,
                           uint32_t *__restrict__ tx, uint32_t *__restrict__ ty, int La, int Lt,
                           int32_t A, int32_t B, int32_t C, int32_t D, RRCarry<> &K,
                           const Radix &R) {
    int beg, end;
    rr_chunk(max(La, Lt), beg, end);
    const uint32_t aA = A < 0 ? -A : A, aB = B < 0 ? -B : B, aC = C < 0 ? -C : C,
                   aD = D < 0 ? -D : D;
    int64_t c[4] = {0, 0, 0, 0};
    for (int k = beg; k < end; ++k) {
        if (k < La) {
            // digits below 2^31: signed 32 x 32 -> 64-bit products
            const int32_t xv = (int32_t)x[k], yv = (int32_t)y[k];
            int64_t q0, q1;
            const uint32_t r0 = divmod_p((int64_t)A * xv + (int64_t)B * yv, R, q0);
            const uint32_t r1 = divmod_p((int64_t)C * xv + (int64_t)D * yv, R, q1);
            x[k] = add_carry(r0, c[0], R.p, q0);
            y[k] = add_carry(r1, c[1], R.p, q1);
            c[0] = q0;
            c[1] = q1;
        }
        if (k < Lt) {
            const uint32_t txv = tx[k], tyv = ty[k];
            int64_t q2, q3;
            const uint32_t r2 = divmod_p((int64_t)((uint64_t)aA * txv + (uint64_t)aB * tyv), R, q2);
            const uint32_t r3 = divmod_p((int64_t)((uint64_t)aC * txv + (uint64_t)aD * tyv), R, q3);
            tx[k] = add_carry(r2, c[2], R.p, q2);
            ty[k] = add_carry(r3, c[3], R.p, q3);
            c[2] = q2;
            c[3] = q3;
        }
    }
    uint32_t *const w[4] = {x, y, tx, ty};
    settle<4>(w, beg, end, c, K, R);
}

// x <- x - q y p^sh on [0, La) and tx <- tx + q ty p^sh on [0, Lt)
// (0 < q < 2^29); the results are >= 0 and fit in their digits.
__device__ void rr_submul(uint32_t *x, const uint32_t *y, int ylen, uint32_t *tx,
                          const uint32_t *ty, int tylen, int La, int Lt, int64_t q, int sh,
                          RRCarry<> &K, const Radix &R) {
    int beg, end;
    rr_chunk(max(La, Lt), beg, end);
    const uint32_t q32 = (uint32_t)q;
    int64_t c[2] = {0, 0};
    for (int k = beg; k < end; ++k) {
        const int src = k - sh;
        if (k < La) {
            const int64_t yv = (src >= 0 && src < ylen) ? y[src] : 0;
            x[k] = divmod_p((int64_t)x[k] - (int64_t)((uint64_t)q32 * (uint32_t)yv) + c[0], R, c[0]);
        }
        if (k < Lt) {
            const int64_t tyv = (src >= 0 && src < tylen) ? ty[src] : 0;
            tx[k] = divmod_p((int64_t)tx[k] + (int64_t)((uint64_t)q32 * (uint32_t)tyv) + c[1], R, c[1]);
        }
    }
    uint32_t *const w[2] = {x, tx};
    settle<2>(w, beg, end, c, K, R);
}

// floor(n / d) for 0 < d, n < 2^63 and a quotient below 2^29: subtraction
// for the smallest quotients, else a single-precision estimate (relative
// error below 2^-21) corrected by one more estimate on the exact remainder
// and unit steps.
__device__ __forceinline__ float u64_to_float(uint64_t v) {
    return __uint2float_rn((uint32_t)(v >> 32)) * 4294967296.0f + __uint2float_rn((uint32_t)v);
}

__device__ __forceinline__ uint64_t quot29(uint64_t n, uint64_t d) {
    if (n < d) return 0;
    uint64_t r = n - d;
    if (r < d) return 1;
    r -= d;
    if (r < d) return 2;
    const float fd = u64_to_float(d);
    int64_t q = __float2int_rz(__fdividef(u64_to_float(n), fd));
    int64_t rr = (int64_t)(n - (uint64_t)q * d);
    if (rr < 0 || (uint64_t)rr >= d) {
        const float fr = rr < 0 ? -u64_to_float((uint64_t)-rr) : u64_to_float((uint64_t)rr);
        q += __float2int_rd(__fdividef(fr, fd));
        rr = (int64_t)(n - (uint64_t)q * d);
    }
    while (rr < 0) {
        --q;
        rr += (int64_t)d;
    }
    while ((uint64_t)rr >= d) {
        ++q;
        rr -= (int64_t)d;
    }
    return (uint64_t)q;
}

__device__ int trim(const uint32_t *x, int l) {
    while (l > 0 && x[l - 1] == 0) --l;
    return l;
}

// Two digits starting at position s (value < p^2 < 2^62).
__device__ uint64_t top2(const uint32_t *x, int l, int s, uint32_t p) {
    uint64_t hi = (s + 1 < l && s + 1 >= 0) ? x[s + 1] : 0;
    uint64_t lo = (s < l && s >= 0) ? x[s] : 0;
    return hi * p + lo;
}

__device__ int cmp_big(const uint32_t *x, int lx, const uint32_t *y, int ly) {
    if (lx != ly) return lx < ly ? -1 : 1;
    for (int k = lx - 1; k >= 0; --k)
        if (x[k] != y[k]) return x[k] < y[k] ? -1 : 1;
    return 0;
}

// For a >= b > 0: c in [1, 2^29) and a digit shift sh with c * b * p^sh <= a,
// removing at least a quarter of a's leading digit.
__device__ void exact_step(const uint32_t *a, int la, const uint32_t *b, int lb, uint32_t p,
                           uint64_t &q, int &sh) {
    uint64_t c;
    int s;
    if (la == 1) {  // then lb == 1
        c = a[0] / b[0];
        s = 0;
    } else if (la > lb) {
        // a >= atop p^(la-2), b < (b_top + 1) p^(lb-1)
        const uint64_t atop = top2(a, la, la - 2, p);
        const uint64_t btop = (uint64_t)b[lb - 1] + 1;
        c = atop / btop;
        s = la - 1 - lb;
        // A quotient estimate far above the clamp (a small top digit of b,
        // up to 2^61) would make the clamped subtraction remove only a
        // sliver of a: take it one digit higher, c / p (still c b p^s <= a),
        // so that every step removes at least a quarter of a's top digit.
        if (c >= (1ull << 29) && c / p >= 1) {
            c /= p;
            s += 1;
        }
    } else {  // la == lb >= 2
        const uint64_t atop = top2(a, la, la - 2, p);
        const uint64_t btop = top2(b, lb, lb - 2, p) + 1;
        c = atop / btop;
        s = 0;
    }
    if (c >= (1ull << 29)) c = (1ull << 29) - 1;
    if (c == 0) {
        c = 1;
        s = 0;
    }
    q = c;
    sh = s;
}

// The Lehmer matrix of a run of Euclid steps read off the leading parts ah,
// bh of a and b (both taken at position s: digits of radix p, or bits when
// BIN; steps = 0: no step could be certified). Runs stop short of the
// numerator bound, so that no remainder below it is skipped: a step is taken
// only while the new b keeps more than lim digits (bits), and the last steps
// are taken exactly.
template <bool BIN>
__device__ __forceinline__ int lehmer(uint64_t ah, uint64_t bh, int s, int lim, uint32_t p,
                                      int64_t &A, int64_t &B, int64_t &C, int64_t &D) {
    A = 1;
    B = 0;
    C = 0;
    D = 1;
    int steps = 0;
    while (true) {
        const int64_t d1 = (int64_t)bh + C, d2 = (int64_t)bh + D;
        if (d1 <= 0 || d2 <= 0) break;
        if ((int64_t)ah + A < 0 || (int64_t)ah + B < 0) break;
        const uint64_t n1 = (uint64_t)((int64_t)ah + A), n2 = (uint64_t)((int64_t)ah + B);
        if (d1 < (1ll << 35) && n1 >= ((uint64_t)d1 << 28)) break;  // quotient >= 2^28
        // floor(n1 / d1), and the same quotient for (n2, d2): q1 d2 <= n2 < (q1 + 1) d2
        const uint64_t q1 = quot29(n1, (uint64_t)d1);
        if (q1 >= (1ull << 28)) break;
        const unsigned __int128 p2 = (unsigned __int128)q1 * (uint64_t)d2;
        if (p2 > n2 || n2 - (uint64_t)p2 >= (uint64_t)d2) break;
        const int64_t q = (int64_t)q1;
        const int64_t nC = A - q * C, nD = B - q * D;
        if (nC >= (1ll << 28) || nC <= -(1ll << 28) || nD >= (1ll << 28) || nD <= -(1ll << 28))
            break;
        const uint64_t nbh = ah - (uint64_t)q * bh;
        const int est = BIN ? s + (64 - __clzll((long long)nbh))
                            : s + (nbh >= p ? 2 : (nbh ? 1 : 0));
        if (est <= lim) break;
        A = C;
        C = nC;
        B = D;
        D = nD;
        ah = bh;
        bh = nbh;
        ++steps;
    }
    return steps;
}

template <class T>
__device__ __forceinline__ void swap_(T &x, T &y) {
    const T t = x;
    x = y;
    y = t;
}

// zdig: m base-p digits of X (|z_i| < 2^59 each; normalised here).
// base: 4 * cap digits (a, b, ta, tb). On success info[0] = 0,
// info[1] = digits of the denominator, written to den (base p).
__device__ void ratrecon_body(const int64_t *__restrict__ z, int m, uint32_t p, int hN, int hD,
                              uint32_t *__restrict__ base, int cap, uint32_t *__restrict__ den,
                              int den_cap, int32_t *__restrict__ info,
                              const uint32_t *__restrict__ ainit, int alen) {
    __shared__ RRCarry<> K;
    uint32_t *a = base, *b = base + cap, *ta = base + 2 * cap, *tb = base + 3 * cap;
    const int tid = threadIdx.x;
    const Radix R = make_radix(p);
    for (int k = tid; k < 4 * cap; k += kRR) base[k] = 0;
    __syncthreads();
    // b = X mod p^m with digits in [0, p): the carry out of digit m - 1 is
    // dropped by settle
    {
        int beg, end;
        rr_chunk(m, beg, end);
        int64_t c[1] = {0};
        for (int k = beg; k < end; ++k) b[k] = divmod_p(z[k] + c[0], R, c[0]);
        uint32_t *const w[1] = {b};
        settle<1>(w, beg, end, c, K, R);
    }
    // a = p^m, or the given first operand (hN = 0: full extended Euclid);
    // ta = 0, tb = 1
    if (ainit) {
        for (int k = tid; k < alen; k += kRR) a[k] = ainit[k];
    } else if (tid == 0) {
        a[m] = 1;
    }
    if (tid == 0) tb[0] = 1;
    __syncthreads();
    int la = ainit ? trim(a, alen) : m + 1, lb = trim(b, m), lta = 0, ltb = 1;
    // The steps below keep a >= b; a given first operand may be the smaller
    // one: exchange the pair with its coefficients (the cofactor found at the
    // zero remainder is the same).
    if (cmp_big(a, la, b, lb) < 0) {
        swap_(a, b);
        swap_(la, lb);
        swap_(ta, tb);
        swap_(lta, ltb);
    }
    // Every pass completes at least one Euclid step or one partial quotient
    // subtraction, each removing at least one bit from a or b; the bound
    // below exceeds the total bit length of (a, b) with a wide margin (a has
    // m + 1 digits, or alen when it is given: it can be much longer than b).
    const long max_iter = 4L * 32 * ((ainit && alen > m ? alen : m) + 4) + 1000;
    int mode = 0;  // 0 running, 1 done, 2 capacity exceeded
    for (long iter = 0; iter < max_iter; ++iter) {
        if (lb <= hN) {
            mode = 1;
            break;
        }
        const int s = la >= 2 ? la - 2 : 0;
        int64_t A, B, C, D;
        const int steps = lehmer<false>(top2(a, la, s, p), top2(b, lb, s, p), s, hN + 2, p, A, B, C, D);
        if (steps > 0) {
            const int La = la, Lt = max(lta, ltb) + 2;
            if (Lt > cap) {
                mode = 2;
                break;
            }
            __syncthreads();  // every thread has read the leading digits
            rr_lincomb(a, b, ta, tb, La, Lt, (int32_t)A, (int32_t)B, (int32_t)C, (int32_t)D, K, R);
            la = trim(a, La);
            lb = trim(b, La);
            lta = trim(ta, Lt);
            ltb = trim(tb, Lt);
        } else if (cmp_big(a, la, b, lb) < 0) {
            swap_(a, b);
            swap_(la, lb);
            swap_(ta, tb);
            swap_(lta, ltb);
        } else {
            uint64_t q;
            int sh;
            exact_step(a, la, b, lb, p, q, sh);
            const int La = la, Lt = max(lta, ltb + sh) + 2;
            if (Lt > cap) {
                mode = 2;
                break;
            }
            __syncthreads();
            rr_submul(a, b, lb, ta, tb, ltb, La, Lt, (int64_t)q, sh, K, R);
            la = trim(a, La);
            lta = trim(ta, Lt);
            if (cmp_big(a, la, b, lb) < 0) {
                swap_(a, b);
                swap_(la, lb);
                swap_(ta, tb);
                swap_(lta, ltb);
            }
        }
    }
    if (mode != 1) {
        if (tid == 0) info[0] = 2;
        return;
    }
    const int ld = ltb;
    if (ld == 0 || ld > hD) {
        if (tid == 0) {
            info[0] = 1;  // no fraction within the bounds
            info[1] = ld;
        }
        return;
    }
    if (ld > den_cap) {
        if (tid == 0) {
            info[0] = 4;
            info[1] = ld;
        }
        return;
    }
    for (int k = tid; k < ld; k += kRR) den[k] = tb[k];
    if (tid == 0) {
        info[0] = 0;
        info[1] = ld;
    }
}

__global__ void __launch_bounds__(kRR)
k_ratrecon(const int64_t *__restrict__ z, int m, uint32_t p, int hN, int hD,
           uint32_t *__restrict__ gbuf, int cap, uint32_t *__restrict__ den, int den_cap,
           int32_t *__restrict__ info, const uint32_t *__restrict__ ainit, int alen) {
    extern __shared__ uint32_t dyn[];
    ratrecon_body(z, m, p, hN, hD, gbuf ? gbuf : dyn, cap, den, den_cap, info, ainit, alen);
}

// One CTA per job of a batch (numbers in shared memory, 4 * cap digits).
__global__ void __launch_bounds__(kRR) k_ratrecon_multi(const RRJob *__restrict__ jobs, int cap) {
    extern __shared__ uint32_t dyn[];
    const RRJob j = jobs[blockIdx.x];
    ratrecon_body(j.z, j.m, j.p, j.hN, j.hD, dyn, cap, j.den, j.den_cap, j.info, nullptr, 0);
}

// ---------------------------------------------------------------------------
// The same reconstruction with the numbers in radix 2^31, for the callers
// that want the denominator in binary (one CTA of kRR threads). The result is
// the one above -- the first remainder of Euclid on (p^m, X) below p^hN, and
// its cofactor as the denominator if that is below p^hD -- computed three ways
// faster: a position is split into digit and carry by a mask and a shift
// rather than a division by p; the Lehmer matrix is found by one thread and
// handed to the others through shared memory; and the denominator comes out
// in 32-bit limbs, with no conversion after it. The p-adic digits are brought
// to binary first by Horner's rule, two digits per pass (X <- X p^2 + d' p +
// d), with p^m, p^hN and p^hD formed in the same passes.

// floor(x / 2^s) for a number x of l limbs (radix 2^31) below 2^(s + 64).
__device__ __forceinline__ uint64_t bits_at(const uint32_t *x, int l, int s) {
    const int i = s / 31, o = s % 31;
    const uint64_t x0 = i < l ? x[i] : 0, x1 = i + 1 < l ? x[i + 1] : 0,
                   x2 = i + 2 < l ? x[i + 2] : 0;
    return (x0 >> o) | (x1 << (31 - o)) | (x2 << (62 - o));
}

__device__ __forceinline__ int bitlen31(const uint32_t *x, int l) {
    return l == 0 ? 0 : 31 * (l - 1) + (32 - __clz((int)x[l - 1]));
}

// 31-bit limb k of y 2^sh (sh = 31 sl + sb).
__device__ __forceinline__ uint32_t shifted31(const uint32_t *y, int ylen, int k, int sl, int sb) {
    const int i = k - sl;
    const uint32_t hi = (i >= 0 && i < ylen) ? y[i] : 0;
    const uint32_t lo = (i - 1 >= 0 && i - 1 < ylen) ? y[i - 1] : 0;
    return sb ? ((hi << sb) | (lo >> (31 - sb))) & kM31 : hi;
}

// (x, y) <- (A x + B y, C x + D y) on limbs [0, La) and (tx, ty) <-
// (|A| tx + |B| ty, |C| tx + |D| ty) on [0, Lt); |A|..|D| < 2^28, limbs below
// 2^31: every product is one signed 32 x 32 -> 64-bit multiply and
// |A x_k + B y_k + carry| < 2^61.
template <int T>
__device__ void rb_lincomb(uint32_t *__restrict__ x, uint32_t *__restrict__ y,
                           uint32_t *__restrict__ tx, uint32_t *__restrict__ ty, int La, int Lt,
                           int32_t A, int32_t B, int32_t C, int32_t D, RRCarry<T> &K,
                           const Radix &R) {
    int beg, end;
    rr_chunk<T>(max(La, Lt), beg, end);
    const int32_t aA = A < 0 ? -A : A, aB = B < 0 ? -B : B, aC = C < 0 ? -C : C,
                  aD = D < 0 ? -D : D;
    const int ea = min(end, La), et = min(end, Lt), e4 = min(ea, et);
    int64_t c[4] = {0, 0, 0, 0};
    int k = beg;
    // the next position's limbs are loaded before this position's are
    // stored (the four numbers never overlap)
    int32_t xv = 0, yv = 0, txv = 0, tyv = 0;
    if (k < e4) {
        xv = (int32_t)x[k];
        yv = (int32_t)y[k];
        txv = (int32_t)tx[k];
        tyv = (int32_t)ty[k];
    }
    for (; k < e4; ++k) {
        int32_t xn = 0, yn = 0, txn = 0, tyn = 0;
        if (k + 1 < e4) {
            xn = (int32_t)x[k + 1];
            yn = (int32_t)y[k + 1];
            txn = (int32_t)tx[k + 1];
            tyn = (int32_t)ty[k + 1];
        }
        x[k] = norm31((int64_t)A * xv + (int64_t)B * yv + c[0], c[0]);
        y[k] = norm31((int64_t)C * xv + (int64_t)D * yv + c[1], c[1]);
        tx[k] = norm31((int64_t)aA * txv + (int64_t)aB * tyv + c[2], c[2]);
        ty[k] = norm31((int64_t)aC * txv + (int64_t)aD * tyv + c[3], c[3]);
        xv = xn;
        yv = yn;
        txv = txn;
        tyv = tyn;
    }
    for (int j = k; j < ea; ++j) {
        const int32_t xv = (int32_t)x[j], yv = (int32_t)y[j];
        x[j] = norm31((int64_t)A * xv + (int64_t)B * yv + c[0], c[0]);
        y[j] = norm31((int64_t)C * xv + (int64_t)D * yv + c[1], c[1]);
    }
    for (int j = k; j < et; ++j) {
        const int32_t txv = (int32_t)tx[j], tyv = (int32_t)ty[j];
        tx[j] = norm31((int64_t)aA * txv + (int64_t)aB * tyv + c[2], c[2]);
        ty[j] = norm31((int64_t)aC * txv + (int64_t)aD * tyv + c[3], c[3]);
    }
    uint32_t *const w[4] = {x, y, tx, ty};
    settle<4, true, T>(w, beg, end, c, K, R);
}

// x <- x - q y 2^sh on [0, La) and tx <- tx + q ty 2^sh on [0, Lt)
// (0 < q < 2^29); the results are >= 0 and fit in their limbs.
template <int T>
__device__ void rb_submul(uint32_t *__restrict__ x, const uint32_t *__restrict__ y, int ylen,
                          uint32_t *__restrict__ tx, const uint32_t *__restrict__ ty, int tylen,
                          int La, int Lt, uint32_t q, int sh, RRCarry<T> &K, const Radix &R) {
    int beg, end;
    rr_chunk<T>(max(La, Lt), beg, end);
    const int sl = sh / 31, sb = sh % 31;
    int64_t c[2] = {0, 0};
    for (int k = beg; k < end; ++k) {
        if (k < La)
            x[k] = norm31((int64_t)x[k] - (int64_t)((uint64_t)q * shifted31(y, ylen, k, sl, sb)) +
                              c[0],
                          c[0]);
        if (k < Lt)
            tx[k] = norm31((int64_t)tx[k] + (int64_t)((uint64_t)q * shifted31(ty, tylen, k, sl, sb)) +
                               c[1],
                           c[1]);
    }
    uint32_t *const w[2] = {x, tx};
    settle<2, true, T>(w, beg, end, c, K, R);
}

// For a >= b > 0 (bit lengths abits, bbits): c in [1, 2^29) and a bit shift
// sh with c b 2^sh <= a, c >= 2^27 whenever sh > 0.
__device__ void rb_exact_step(const uint32_t *a, int la, int abits, const uint32_t *b, int lb,
                              int bbits, uint32_t &q, int &sh) {
    uint64_t c;
    int s = 0;
    if (abits <= 62) {
        // exact quotient; above the clamp, its leading 29 bits at a shift
        c = bits_at(a, la, 0) / bits_at(b, lb, 0);
        if (c >= (1ull << 29)) {
            s = (64 - __clzll((long long)c)) - 29;
            c >>= s;
        }
    } else {
        // a >= atop 2^(abits - 62); b < bt 2^sb
        const uint64_t atop = bits_at(a, la, abits - 62);
        const int sb = bbits > 32 ? bbits - 32 : 0;
        const uint64_t bt = bits_at(b, lb, sb) + 1;
        s = abits - bbits - 28;
        if (s < 0) s = 0;
        const int e = (abits - 62) - (sb + s);  // in [-30, -2]
        c = (atop / bt) >> (-e);
    }
    if (c >= (1ull << 29)) c = (1ull << 29) - 1;
    if (c == 0) c = 1;
    q = (uint32_t)c;
    sh = s;
}

// A run of Euclid steps on the leading parts ah >= bh of a and b, both taken
// at bit s (a = ah 2^s + a', b = bh 2^s + b', 0 <= a', b' < 2^s), with
// r_0 = ah, r_1 = bh and cofactors r_i = u_i ah + v_i bh. The same quotients
// applied to (a, b) give R_i = r_i 2^s + e_i with e_i = u_i a' + v_i b'; the
// signs alternate (u_i >= 0 >= v_i for even i, u_i <= 0 <= v_i for odd i), so
// -|v_i| 2^s < e_i < |u_i| 2^s for even i and -|u_i| 2^s < e_i < |v_i| 2^s
// for odd i, up to equality when a cofactor is 0. The quotient q_i of
// r_(i-1) by r_i is therefore that of R_(i-1) by R_i (0 <= R_(i+1) < R_i)
// whenever
//     r_(i+1) >= |v_(i+1)| and r_i - r_(i+1) >= |u_(i+1) - u_i|   (i+1 even),
//     r_(i+1) >= |u_(i+1)| and r_i - r_(i+1) >= |v_(i+1) - v_i|   (i+1 odd).
// One division per step, no second quotient: a single-precision estimate of
// r_(i-1) / r_i (relative error below 2^-21), one unit correction either way,
// and the exact test 0 <= r_(i+1) < r_i, which fails (and ends the run) in
// the rare case of a larger error. The run stops at the first step that fails
// a test, whose quotient or cofactors reach 2^28, or whose remainder keeps at
// most lim bits (so that no remainder below the numerator bound is skipped;
// the last steps are taken exactly); the tests of a step are combined into
// one branch. On return (a, b) <- (A a + B b, C a + D b) applies the
// accepted steps.
__device__ __forceinline__ int lehmer_bin(uint64_t ah, uint64_t bh, int s, int lim, int64_t &A,
                                          int64_t &B, int64_t &C, int64_t &D) {
    int64_t u0 = 1, v0 = 0, u1 = 0, v1 = 1;
    uint64_t r0 = ah, r1 = bh;
    int steps = 0;
    bool even = true;  // parity of the index of the next remainder (2 first)
    while (r1 > 0) {
        float fq = __fdividef(u64_to_float(r0), u64_to_float(r1));
        fq = fminf(fq, 268435456.0f);  // 2^28: larger quotients end the run
        int64_t q = (int64_t)__float2uint_rz(fq);
        int64_t r2 = (int64_t)(r0 - (uint64_t)q * r1);
        if (r2 < 0) {
            --q;
            r2 += (int64_t)r1;
        } else if ((uint64_t)r2 >= r1) {
            ++q;
            r2 -= (int64_t)r1;
        }
        const int64_t u2 = u0 - q * u1, v2 = v0 - q * v1;
        const int64_t au2 = u2 < 0 ? -u2 : u2, av2 = v2 < 0 ? -v2 : v2;
        const int64_t du = u2 - u1, dv = v2 - v1;
        const int64_t need1 = even ? av2 : au2;
        const int64_t need2 = even ? (du < 0 ? -du : du) : (dv < 0 ? -dv : dv);
        const bool ok = r2 >= 0 && (uint64_t)r2 < r1 && q < (1ll << 28) &&
                        au2 < (1ll << 28) && av2 < (1ll << 28) && r2 >= need1 &&
                        (int64_t)r1 - r2 >= need2 &&
                        s + (64 - __clzll(r2)) > lim;
        if (!ok) break;
        u0 = u1;
        v0 = v1;
        u1 = u2;
        v1 = v2;
        r0 = r1;
        r1 = (uint64_t)r2;
        even = !even;
        ++steps;
    }
    A = u0;
    B = v0;
    C = u1;
    D = v1;
    return steps;
}

struct RBShared {
    int64_t A, B, C, D;
    int steps;  // > 0: Lehmer matrix; 0: exact step (q, sh)
    int sh;
    uint32_t q;
};

// z: m base-p digits of X (|z_i| < 2^59 each). base: 5 * cap + 2 * bcap
// limbs (cap >= m + 4 for a, b, ta, tb and the digits; bcap >= max(hN, hD) + 4
// for the bounds). On success info[0] = 0, info[1] = 32-bit limbs of the
// denominator written to den, info[2] = its bit length, info[3] = its
// leading 31 bits; info[0] = 1: no fraction within the bounds, 2: capacity.
template <int T>
__device__ void ratrecon_bin_body(const int64_t *__restrict__ z, int m, uint32_t p, int hN,
                                  int hD, uint32_t *__restrict__ base, int cap, int bcap,
                                  uint32_t *__restrict__ den, int den_cap,
                                  int32_t *__restrict__ info) {
    __shared__ RRCarry<T> K;
    __shared__ RBShared S;
    uint32_t *a = base, *b = base + cap, *ta = base + 2 * cap, *tb = base + 3 * cap,
             *dg = base + 4 * cap, *NB = base + 5 * cap, *DB = base + 5 * cap + bcap;
    const int tid = threadIdx.x;
    const Radix R = make_radix(p);
    for (int k = tid; k < 5 * cap + 2 * bcap; k += T) base[k] = 0;
    __syncthreads();
    // the digits of X mod p^m in [0, p)
    {
        int beg, end;
        rr_chunk<T>(m, beg, end);
        int64_t c[1] = {0};
        for (int k = beg; k < end; ++k) dg[k] = divmod_p(z[k] + c[0], R, c[0]);
        uint32_t *const w[1] = {dg};
        settle<1, false, T>(w, beg, end, c, K, R);
    }
    // Horner: b <- X, a <- p^e with e = m at the end; NB = p^hN, DB = p^hD.
    // p^2 = P1 2^31 + P0; limb k of v p^2 is x_k P0 + x_(k-1) P1 + carry.
    const uint64_t p2 = (uint64_t)p * p;
    const uint32_t P0 = (uint32_t)(p2 & kM31), P1 = (uint32_t)(p2 >> 31);
    int L = 0, e = m & 1;  // limbs in use (an upper bound), exponent of a
    if (tid == 0) {
        a[0] = e ? p : 1;
        b[0] = (m & 1) ? dg[m - 1] : 0;
    }
    L = 1;
    __syncthreads();
    auto capture = [&](uint32_t *dst, int want) {
        // dst = p^want (< 2^(31 want): at most want <= bcap - 4 limbs) from
        // a = p^e, e in {want, want - 1}
        const int Lc = min(L + 1, bcap);
        for (int k = tid; k < Lc; k += T) dst[k] = k < L ? a[k] : 0;
        __syncthreads();
        if (e == want - 1 && tid == 0) {
            uint64_t c = 0;
            for (int k = 0; k < Lc; ++k) {
                const uint64_t v = (uint64_t)dst[k] * p + c;
                dst[k] = (uint32_t)v & kM31;
                c = v >> 31;
            }
        }
        __syncthreads();
    };
    if (hN == 0) {
        if (tid == 0) NB[0] = 1;
    } else if (e == hN || e == hN - 1) {
        capture(NB, hN);
    }
    if (hD == 0) {
        if (tid == 0) DB[0] = 1;
    } else if (e == hD || e == hD - 1) {
        capture(DB, hD);
    }
    __syncthreads();
    for (int i = m - 2 - (m & 1); i >= 0; i -= 2) {
        // a p^2 = p^(e+2) and b p^2 + v < p^(e+2) < 2^(31 (e+2)): e + 2 limbs
        L = min(cap, e + 3);
        int beg, end;
        rr_chunk<T>(L, beg, end);
        int64_t c[2] = {0, 0};
        if (beg == 0 && end > 0) c[1] = (int64_t)((uint64_t)dg[i + 1] * p + dg[i]);
        uint64_t ha = 0, hb = 0;
        uint32_t av = beg < end ? a[beg] : 0, bv = beg < end ? b[beg] : 0;
        for (int k = beg; k < end; ++k) {
            // next limbs loaded before this position is stored
            const uint32_t an = k + 1 < end ? a[k + 1] : 0, bn = k + 1 < end ? b[k + 1] : 0;
            const uint64_t va = (uint64_t)av * P0 + ha + (uint64_t)c[0];
            const uint64_t vb = (uint64_t)bv * P0 + hb + (uint64_t)c[1];
            a[k] = (uint32_t)va & kM31;
            b[k] = (uint32_t)vb & kM31;
            c[0] = (int64_t)(va >> 31);
            c[1] = (int64_t)(vb >> 31);
            ha = (uint64_t)av * P1;
            hb = (uint64_t)bv * P1;
            av = an;
            bv = bn;
        }
        c[0] += (int64_t)ha;
        c[1] += (int64_t)hb;
        uint32_t *const w[2] = {a, b};
        settle<2, true, T>(w, beg, end, c, K, R);
        e += 2;
        if (e == hN || e == hN - 1) capture(NB, hN);
        if (e == hD || e == hD - 1) capture(DB, hD);
    }
    // the digits' space becomes tb's scratch: clear ta and tb, tb = 1
    for (int k = tid; k < 2 * cap; k += T) ta[k] = 0;
    __syncthreads();
    if (tid == 0) tb[0] = 1;
    int la = trim(a, L), lb = trim(b, L), lta = 0, ltb = 1;
    const int lnb = trim(NB, bcap), ldb = trim(DB, bcap);
    const int nbbits = bitlen31(NB, lnb);
    __syncthreads();
    // a = p^m > X = b: no exchange needed
    const long max_iter = 4L * 32 * (m + 4) + 1000;
    int mode = 0;  // 0 running, 1 done, 2 capacity exceeded
    for (long iter = 0; iter < max_iter; ++iter) {
        if (cmp_big(b, lb, NB, lnb) < 0) {
            mode = 1;
            break;
        }
        const bool swap_only = cmp_big(a, la, b, lb) < 0;
        if (!swap_only && tid == 0) {
            const int abits = bitlen31(a, la), bbits = bitlen31(b, lb);
            const int s = abits > 62 ? abits - 62 : 0;
            int64_t A, B, C, D;
            const int steps =
                lehmer_bin(bits_at(a, la, s), bits_at(b, lb, s), s, nbbits + 64, A, B, C, D);
            S.steps = steps;
            S.A = A;
            S.B = B;
            S.C = C;
            S.D = D;
            if (steps == 0) {
                uint32_t q;
                int sh;
                rb_exact_step(a, la, abits, b, lb, bbits, q, sh);
                S.q = q;
                S.sh = sh;
            }
        }
        if (swap_only) {
            swap_(a, b);
            swap_(la, lb);
            swap_(ta, tb);
            swap_(lta, ltb);
            continue;
        }
        __syncthreads();  // the step is published; every thread has read the lengths
        const int steps = S.steps;
        if (steps > 0) {
            const int La = la, Lt = max(lta, ltb) + 2;
            if (Lt > cap) {
                mode = 2;
                break;
            }
            rb_lincomb(a, b, ta, tb, La, Lt, (int32_t)S.A, (int32_t)S.B, (int32_t)S.C,
                       (int32_t)S.D, K, R);
            la = trim(a, La);
            lb = trim(b, La);
            lta = trim(ta, Lt);
            ltb = trim(tb, Lt);
        } else {
            const uint32_t q = S.q;
            const int sh = S.sh;
            const int La = la, Lt = max(lta, ltb + sh / 31 + 1) + 2;
            if (Lt > cap) {
                mode = 2;
                break;
            }
            rb_submul(a, b, lb, ta, tb, ltb, La, Lt, q, sh, K, R);
            la = trim(a, La);
            lta = trim(ta, Lt);
        }
    }
    if (mode != 1) {
        if (tid == 0) info[0] = 2;
        return;
    }
    // the denominator tb, if 0 < tb < p^hD, in 32-bit limbs
    if (ltb == 0 || cmp_big(tb, ltb, DB, ldb) >= 0) {
        if (tid == 0) {
            info[0] = 1;
            info[1] = ltb;
        }
        return;
    }
    const int bits = bitlen31(tb, ltb);
    const int l32 = (bits + 31) / 32;
    if (l32 > den_cap) {
        if (tid == 0) {
            info[0] = 4;
            info[1] = l32;
        }
        return;
    }
    for (int j = tid; j < l32; j += T) {
        const int i = j + j / 31, o = j % 31;
        const uint64_t lo = tb[i], hi = i + 1 < ltb ? tb[i + 1] : 0;
        den[j] = (uint32_t)((lo >> o) | (hi << (31 - o)));
    }
    if (tid == 0) {
        info[0] = 0;
        info[1] = l32;
        info[2] = bits;
        info[3] = (int32_t)bits_at(tb, ltb, bits > 31 ? bits - 31 : 0);
    }
}

// The numbers always in shared memory (ratrecon_bin_fits). More threads
// than the base-p kernel: one thread finds the Lehmer matrix while the others
// wait, so the extra warps cost no issue slots and halve every vector pass.
constexpr int kRB = 512;

__global__ void __launch_bounds__(kRB)
k_ratrecon_bin(const int64_t *__restrict__ z, int m, uint32_t p, int hN, int hD, int cap,
               int bcap, uint32_t *__restrict__ den, int den_cap, int32_t *__restrict__ info) {
    extern __shared__ uint32_t dyn[];
    ratrecon_bin_body<kRB>(z, m, p, hN, hD, dyn, cap, bcap, den, den_cap, info);
}

// Base-p digits (len of them) -> base-2^32 limbs, Horner on one CTA:
// x <- x * p + d, from the top digit down. out has cap limbs.
__global__ void __launch_bounds__(kRT)
k_radix_to_binary(const uint32_t *__restrict__ dig, int len, uint32_t p,
                  uint32_t *__restrict__ out, int cap, int32_t *__restrict__ out_len) {
    __shared__ int64_t s_co[kRT];
    __shared__ int s_len;
    for (int k = threadIdx.x; k < cap; k += kRT) out[k] = 0;
    if (threadIdx.x == 0) s_len = 0;
    __syncthreads();
    for (int i = len - 1; i >= 0; --i) {
        const int L = min(cap, s_len + 1);
        int beg, end;
        chunk_of(L, beg, end);
        uint64_t c = (threadIdx.x == 0) ? dig[i] : 0;
        for (int k = beg; k < end; ++k) {
            uint64_t v = (uint64_t)out[k] * p + c;
            out[k] = (uint32_t)v;
            c = v >> 32;
        }
        // unsigned carries: propagate
        s_co[threadIdx.x] = (int64_t)c;
        __syncthreads();
        int64_t cin = threadIdx.x > 0 ? s_co[threadIdx.x - 1] : 0;
        __syncthreads();
        for (int pass = 0; pass <= kRT; ++pass) {
            uint64_t cc = (uint64_t)cin;
            for (int k = beg; k < end && cc != 0; ++k) {
                uint64_t v = (uint64_t)out[k] + cc;
                out[k] = (uint32_t)v;
                cc = v >> 32;
            }
            if (beg >= end) cc = 0;  // past the top limb: nothing to carry into
            s_co[threadIdx.x] = (int64_t)cc;
            int any = __syncthreads_or(cc != 0 && threadIdx.x != kRT - 1);
            if (!any) break;
            cin = threadIdx.x > 0 ? s_co[threadIdx.x - 1] : 0;
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            int l = L;
            while (l > 0 && out[l - 1] == 0) --l;
            s_len = l;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out_len = s_len;
}

}  // namespace

int launch_cra_append(const uint32_t *primes, const uint32_t *residues, int32_t *digits,
                      int start, int count, int32_t *info, cudaStream_t s) {
    (void)info;
    if (count <= 0) return IDET_OK;
    k_cra_append<<<1, kCraThreads, 0, s>>>(primes, residues, digits, start, count);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

int launch_div_by_K(const uint32_t *Klimbs, int Klen, const uint32_t *primes,
                    const uint32_t *res_in, uint32_t *res_out, int32_t *skip, int count,
                    cudaStream_t s) {
    if (count <= 0) return IDET_OK;
    k_div_by_K<<<(count + 127) / 128, 128, 0, s>>>(Klimbs, Klen, primes, res_in, res_out,
                                                     skip, count);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

int launch_mixed_to_int(const uint32_t *primes, const int32_t *digits, int count,
                        const uint32_t *Klimbs, int Klen, uint32_t *out, int out_cap,
                        int32_t *out_info, cudaStream_t s) {
    // out_cap limbs of scratch follow `out` in the same allocation
    k_mixed_to_int<<<1, 32, 0, s>>>(primes, digits, count, Klimbs, Klen, out, out_cap,
                                    out + out_cap, out_info);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

int launch_ratrecon(const int64_t *z, int m, uint32_t p, int hN, int hD, uint32_t *den,
                    int den_cap, int32_t *info, Workspace &ws, const uint32_t *ainit, int alen) {
    cudaStream_t s = ws.stream();
    if (p <= (1u << 30) || p >= (1u << 31)) {
        set_last_error("rational reconstruction: p = %u is outside (2^30, 2^31)", p);
        return IDET_ERR_ARG;
    }
    const int cap = (m > alen ? m : alen) + 4;
    uint32_t *gbuf = nullptr;
    size_t smem = sizeof(uint32_t) * 4 * (size_t)cap;
    if (smem > 190 * 1024) {
        IDET_TRY(ws.alloc_n(&gbuf, 4 * (size_t)cap));
        smem = 0;
    } else {
        IDET_TRY(allow_max_smem((const void *)k_ratrecon));
    }
    k_ratrecon<<<1, kRR, smem, s>>>(z, m, p, hN, hD, gbuf, cap, den, den_cap, info, ainit, alen);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

static size_t ratrecon_bin_smem(int m, int hN, int hD) {
    const size_t cap = (size_t)m + 4, bcap = (size_t)(hN > hD ? hN : hD) + 4;
    return sizeof(uint32_t) * (5 * cap + 2 * bcap);
}

bool ratrecon_bin_fits(int m, int hN, int hD) {
    return m >= 1 && ratrecon_bin_smem(m, hN, hD) <= 190 * 1024;
}

int launch_ratrecon_bin(const int64_t *z, int m, uint32_t p, int hN, int hD, uint32_t *den,
                        int den_cap, int32_t *info, Workspace &ws) {
    cudaStream_t s = ws.stream();
    if (p <= (1u << 30) || p >= (1u << 31)) {
        set_last_error("rational reconstruction: p = %u is outside (2^30, 2^31)", p);
        return IDET_ERR_ARG;
    }
    if (m < 1 || hN < 0 || hD < 0 || hN > m || hD > m || !ratrecon_bin_fits(m, hN, hD)) {
        set_last_error("rational reconstruction: bad bounds or too long (m %d, hN %d, hD %d)", m,
                       hN, hD);
        return IDET_ERR_ARG;
    }
    const int cap = m + 4, bcap = (hN > hD ? hN : hD) + 4;
    IDET_TRY(allow_max_smem((const void *)k_ratrecon_bin));
    k_ratrecon_bin<<<1, kRB, ratrecon_bin_smem(m, hN, hD), s>>>(z, m, p, hN, hD, cap, bcap, den,
                                                                 den_cap, info);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

int launch_ratrecon_multi(const RRJob *jobs_dev, int count, int max_m, cudaStream_t s) {
    if (count <= 0) return IDET_OK;
    const int cap = max_m + 4;
    const size_t smem = sizeof(uint32_t) * 4 * (size_t)cap;
    if (smem > 190 * 1024) {
        set_last_error("batched reconstruction: lift too long");
        return IDET_ERR_ARG;
    }
    IDET_TRY(allow_max_smem((const void *)k_ratrecon_multi));
    k_ratrecon_multi<<<count, kRR, smem, s>>>(jobs_dev, cap);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

int launch_cra_multi(const CraJob *jobs_dev, int count, cudaStream_t s) {
    if (count <= 0) return IDET_OK;
    k_cra_multi<<<count, kCraThreads, 0, s>>>(jobs_dev);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

int launch_radix_to_binary(const uint32_t *dig, int len, uint32_t p, uint32_t *out, int cap,
                           int32_t *out_len, cudaStream_t s) {
    k_radix_to_binary<<<1, kRT, 0, s>>>(dig, len, p, out, cap, out_len);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

}  // namespace idet
