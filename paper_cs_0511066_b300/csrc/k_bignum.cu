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
// Rational reconstruction in radix p (single CTA, kRT threads).
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

constexpr int kRT = 1024;

struct RRShared {
    int64_t co[4][kRT];
    int la, lb, lta, ltb;
    int64_t A, B, C, D;
    int steps;
    int mode;  // 0 running, 1 done, 2 capacity exceeded
    uint64_t q;
    int sh;
    int flag;
};

struct Radix {
    uint32_t p;
    uint64_t m;    // floor((2^64-1)/p)
    int64_t kp;    // ceil(2^62 / p)
    int64_t off;   // kp * p >= 2^62
};

__device__ __forceinline__ Radix make_radix(uint32_t p) {
    Radix R;
    R.p = p;
    R.m = ~0ull / p;
    R.kp = (int64_t)(((1ull << 62) + p - 1) / p);
    R.off = R.kp * (int64_t)p;
    return R;
}

// v = carry * p + digit with 0 <= digit < p, for |v| < 2^62.
__device__ __forceinline__ uint32_t divmod_p(int64_t v, const Radix &R, int64_t &carry) {
    uint64_t u = (uint64_t)(v + R.off);
    uint64_t q = __umul64hi(u, R.m);
    uint64_t r = u - q * R.p;
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

// Each thread has written its digits [beg, end) of NA arrays with carry-in
// 0 and carry-outs co[]; propagate the (signed) carries across the chunks.
// Each pass moves every pending carry at least one chunk up, so at most kRT
// passes are needed.
template <int NA>
__device__ void resolve_p(uint32_t *const *w, int beg, int end, const int64_t *co,
                          RRShared &S, const Radix &R) {
    const int tid = threadIdx.x;
#pragma unroll
    for (int q = 0; q < NA; ++q) S.co[q][tid] = co[q];
    __syncthreads();
    int64_t cin[NA];
#pragma unroll
    for (int q = 0; q < NA; ++q) cin[q] = tid > 0 ? S.co[q][tid - 1] : 0;
    __syncthreads();
    for (int pass = 0; pass <= kRT; ++pass) {
        bool pend = false;
#pragma unroll
        for (int q = 0; q < NA; ++q) {
            int64_t c = cin[q];
            for (int k = beg; k < end && c != 0; ++k) w[q][k] = divmod_p((int64_t)w[q][k] + c, R, c);
            // a chunk past the top digit drops its carry: the result fits in
            // the digits below, so carries beyond them cancel
            if (beg >= end) c = 0;
            S.co[q][tid] = c;
            pend |= (c != 0);
        }
        int any = __syncthreads_or(pend && tid != kRT - 1);
        if (!any) break;
#pragma unroll
        for (int q = 0; q < NA; ++q) cin[q] = tid > 0 ? S.co[q][tid - 1] : 0;
        __syncthreads();
    }
    __syncthreads();
}

// (x, y) <- (A x + B y, C x + D y) and (tx, ty) <- (|A| tx + |B| ty,
// |C| tx + |D| ty) in one pass over L digits; |A|..|D| < 2^28; all results
// are >= 0 and fit in L digits.
__device__ void lincomb4_p(uint32_t *x, uint32_t *y, uint32_t *tx, uint32_t *ty, int La,
                           int Lt, int64_t A, int64_t B, int64_t C, int64_t D, RRShared &S,
                           const Radix &R) {
    // x, y use digits [0, La), tx, ty digits [0, Lt); both are zero above
    // their ranges, so one chunking of [0, max(La, Lt)) serves all four.
    const int L = max(La, Lt);
    int beg, end;
    chunk_of(L, beg, end);
    const int64_t aA = A < 0 ? -A : A, aB = B < 0 ? -B : B, aC = C < 0 ? -C : C,
                  aD = D < 0 ? -D : D;
    int64_t c[4] = {0, 0, 0, 0};
    for (int k = beg; k < end; ++k) {
        if (k < La) {
            int64_t xv = x[k], yv = y[k];
            x[k] = divmod_p(A * xv + B * yv + c[0], R, c[0]);
            y[k] = divmod_p(C * xv + D * yv + c[1], R, c[1]);
        }
        if (k < Lt) {
            int64_t txv = tx[k], tyv = ty[k];
            tx[k] = divmod_p(aA * txv + aB * tyv + c[2], R, c[2]);
            ty[k] = divmod_p(aC * txv + aD * tyv + c[3], R, c[3]);
        }
    }
    uint32_t *ws[4] = {x, y, tx, ty};
    resolve_p<4>(ws, beg, end, c, S, R);
}

// x <- x - q y p^sh and tx <- tx + q ty p^sh (0 < q < 2^29); L digits.
__device__ void submul2_shift_p(uint32_t *x, const uint32_t *y, int ylen, uint32_t *tx,
                                const uint32_t *ty, int tylen, int La, int Lt, int64_t q,
                                int sh, RRShared &S, const Radix &R) {
    int beg, end;
    chunk_of(max(La, Lt), beg, end);
    int64_t c[2] = {0, 0};
    for (int k = beg; k < end; ++k) {
        const int src = k - sh;
        if (k < La) {
            const int64_t yv = (src >= 0 && src < ylen) ? y[src] : 0;
            x[k] = divmod_p((int64_t)x[k] - q * yv + c[0], R, c[0]);
        }
        if (k < Lt) {
            const int64_t tyv = (src >= 0 && src < tylen) ? ty[src] : 0;
            tx[k] = divmod_p((int64_t)tx[k] + q * tyv + c[1], R, c[1]);
        }
    }
    uint32_t *ws[2] = {x, tx};
    resolve_p<2>(ws, beg, end, c, S, R);
}

// floor(x / y) for x, y < 2^63, y > 0: subtraction for the small quotients
// that dominate Euclid's algorithm, 64-bit division otherwise.
__device__ __forceinline__ uint64_t small_quot(uint64_t x, uint64_t y) {
    if (x < y) return 0;
    uint64_t r = x - y;
    if (r < y) return 1;
    r -= y;
    if (r < y) return 2;
    r -= y;
    if (r < y) return 3;
    return x / y;
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

// zdig: m base-p digits of X (any int64 < 2^59 each; normalised here).
// buf: 4 * cap digits (a, b, ta, tb). On success info[0] = 0,
// info[1] = digits of the denominator, written to den (base p).
__device__ void ratrecon_body(const int64_t *__restrict__ z, int m, uint32_t p, int hN, int hD,
                              uint32_t *__restrict__ base, int cap, uint32_t *__restrict__ den,
                              int den_cap, int32_t *__restrict__ info,
                              const uint32_t *__restrict__ ainit, int alen) {
    __shared__ RRShared S;
    uint32_t *a = base, *b = base + cap, *ta = base + 2 * cap, *tb = base + 3 * cap;
    const int tid = threadIdx.x;
    const Radix R = make_radix(p);
    for (int k = tid; k < cap; k += kRT) {
        a[k] = 0;
        b[k] = 0;
        ta[k] = 0;
        tb[k] = 0;
    }
    __syncthreads();
    if (tid == 0) {
        // b = X mod p^m with digits in [0, p); a = p^m; ta = 0, tb = 1
        int64_t carry = 0;
        for (int i = 0; i < m; ++i) b[i] = divmod_p(z[i] + carry, R, carry);
        if (ainit) {  // first operand given (hN = 0: full extended Euclid)
            for (int i = 0; i < alen; ++i) a[i] = ainit[i];
            S.la = trim(a, alen);
        } else {
            a[m] = 1;
            S.la = m + 1;
        }
        tb[0] = 1;
        S.lb = trim(b, m);
        S.lta = 0;
        S.ltb = 1;
        S.mode = 0;
        // The steps below keep a >= b; a given first operand may be the
        // smaller one: exchange the pair (the coefficients still refer to b
        // as given, so the cofactor found at the zero remainder is the same).
        if (cmp_big(a, S.la, b, S.lb) < 0) {
            const int L = max(S.la, S.lb);
            for (int k = 0; k < L; ++k) {
                const uint32_t t = a[k];
                a[k] = b[k];
                b[k] = t;
            }
            ta[0] = 1;
            tb[0] = 0;
            const int t = S.la;
            S.la = S.lb;
            S.lb = t;
            S.lta = 1;
            S.ltb = 0;
        }
    }
    __syncthreads();
    // Every pass completes at least one Euclid step or one partial quotient
    // subtraction, each removing at least one bit from a or b; the bound
    // below exceeds the total bit length of (a, b) with a wide margin (a has
    // m + 1 digits, or alen when it is given: it can be much longer than b).
    const long max_iter = 4L * 32 * ((ainit && alen > m ? alen : m) + 4) + 1000;
    for (long iter = 0; iter < max_iter; ++iter) {
        if (tid == 0) {
            const int la = S.la, lb = S.lb;
            if (lb <= hN) {
                S.mode = 1;
            } else {
                const int s = la >= 2 ? la - 2 : 0;
                uint64_t ah = top2(a, la, s, p), bh = top2(b, lb, s, p);
                int64_t A = 1, B = 0, C = 0, D = 1;
                int steps = 0;
                while (true) {
                    int64_t d1 = (int64_t)bh + C, d2 = (int64_t)bh + D;
                    if (d1 <= 0 || d2 <= 0) break;
                    if ((int64_t)ah + A < 0 || (int64_t)ah + B < 0) break;
                    const uint64_t n1 = (uint64_t)((int64_t)ah + A), n2 = (uint64_t)((int64_t)ah + B);
                    if (d1 < (1ll << 35) && n1 >= ((uint64_t)d1 << 28)) break;  // quotient >= 2^28
                    const uint64_t q1 = small_quot(n1, (uint64_t)d1);
                    const uint64_t q2 = small_quot(n2, (uint64_t)d2);
                    if (q1 != q2 || q1 >= (1ull << 28)) break;
                    int64_t q = (int64_t)q1;
                    int64_t nC = A - q * C, nD = B - q * D;
                    if (nC >= (1ll << 28) || nC <= -(1ll << 28) || nD >= (1ll << 28) ||
                        nD <= -(1ll << 28))
                        break;
                    uint64_t nbh = ah - (uint64_t)q * bh;
                    // stop short of the bound: the last steps are taken exactly
                    const int est = s + (nbh >= p ? 2 : (nbh ? 1 : 0));
                    if (est <= hN + 2) break;
                    A = C;
                    C = nC;
                    B = D;
                    D = nD;
                    ah = bh;
                    bh = nbh;
                    ++steps;
                }
                S.A = A;
                S.B = B;
                S.C = C;
                S.D = D;
                S.steps = steps;
                if (steps == 0) {
                    if (cmp_big(a, la, b, lb) < 0) {
                        S.sh = -1;  // swap only
                    } else {
                        uint64_t q;
                        int sh;
                        exact_step(a, la, b, lb, p, q, sh);
                        S.q = q;
                        S.sh = sh;
                    }
                }
            }
        }
        __syncthreads();
        if (S.mode != 0) break;
        if (S.steps > 0) {
            const int La = S.la, Lt = max(S.lta, S.ltb) + 2;
            if (Lt > cap) {
                if (tid == 0) S.mode = 2;
                __syncthreads();
                break;
            }
            lincomb4_p(a, b, ta, tb, La, Lt, S.A, S.B, S.C, S.D, S, R);
            if (tid == 0) {
                S.la = trim(a, La);
                S.lb = trim(b, La);
                S.lta = trim(ta, Lt);
                S.ltb = trim(tb, Lt);
            }
            __syncthreads();
        } else {
            if (S.sh >= 0) {
                const int La = S.la, Lt = max(S.lta, S.ltb + S.sh) + 2;
                if (Lt > cap) {
                    if (tid == 0) S.mode = 2;
                    __syncthreads();
                    break;
                }
                submul2_shift_p(a, b, S.lb, ta, tb, S.ltb, La, Lt, (int64_t)S.q, S.sh, S, R);
                if (tid == 0) {
                    S.la = trim(a, La);
                    S.lta = trim(ta, Lt);
                }
                __syncthreads();
            }
            if (tid == 0) S.flag = cmp_big(a, S.la, b, S.lb) < 0;
            __syncthreads();
            if (S.flag) {
                const int L = max(S.la, S.lb), Lt = max(S.lta, S.ltb);
                for (int k = tid; k < max(L, Lt); k += kRT) {
                    if (k < L) {
                        uint32_t t = a[k];
                        a[k] = b[k];
                        b[k] = t;
                    }
                    if (k < Lt) {
                        uint32_t t = ta[k];
                        ta[k] = tb[k];
                        tb[k] = t;
                    }
                }
                __syncthreads();
                if (tid == 0) {
                    int t = S.la;
                    S.la = S.lb;
                    S.lb = t;
                    t = S.lta;
                    S.lta = S.ltb;
                    S.ltb = t;
                }
                __syncthreads();
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        if (S.mode != 1) {
            info[0] = 2;
            return;
        }
        const int ld = S.ltb;
        if (ld == 0 || ld > hD) {
            info[0] = 1;  // no fraction within the bounds
            info[1] = ld;
            return;
        }
        if (ld > den_cap) {
            info[0] = 4;
            info[1] = ld;
            return;
        }
        for (int k = 0; k < ld; ++k) den[k] = tb[k];
        info[0] = 0;
        info[1] = ld;
    }
}

__global__ void __launch_bounds__(kRT)
k_ratrecon(const int64_t *__restrict__ z, int m, uint32_t p, int hN, int hD,
           uint32_t *__restrict__ gbuf, int cap, uint32_t *__restrict__ den, int den_cap,
           int32_t *__restrict__ info, const uint32_t *__restrict__ ainit, int alen) {
    extern __shared__ uint32_t dyn[];
    ratrecon_body(z, m, p, hN, hD, gbuf ? gbuf : dyn, cap, den, den_cap, info, ainit, alen);
}

// One CTA per job of a batch (numbers in shared memory, 4 * cap digits).
__global__ void __launch_bounds__(kRT) k_ratrecon_multi(const RRJob *__restrict__ jobs, int cap) {
    extern __shared__ uint32_t dyn[];
    const RRJob j = jobs[blockIdx.x];
    ratrecon_body(j.z, j.m, j.p, j.hN, j.hD, dyn, cap, j.den, j.den_cap, j.info, nullptr, 0);
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
    const int cap = (m > alen ? m : alen) + 4;
    uint32_t *gbuf = nullptr;
    size_t smem = sizeof(uint32_t) * 4 * (size_t)cap;
    if (smem > 190 * 1024) {
        IDET_TRY(ws.alloc_n(&gbuf, 4 * (size_t)cap));
        smem = 0;
    } else {
        IDET_TRY(allow_max_smem((const void *)k_ratrecon));
    }
    k_ratrecon<<<1, kRT, smem, s>>>(z, m, p, hN, hD, gbuf, cap, den, den_cap, info, ainit, alen);
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
    k_ratrecon_multi<<<count, kRT, smem, s>>>(jobs_dev, cap);
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
