// LU factorisation over Z/p for a batch of primes, and A^{-1} mod p from it.
//
// Section 2.1 (Alg. 2.1, step "Compute det(A) mod p_i") obtains det(A) mod
// p_i from an LU factorisation modulo p_i. Pivoting rule: the first row at or
// below the diagonal whose entry is nonzero mod p (the paper does not fix
// one; any nonzero pivot gives the same determinant, this one makes the
// factors unique). det(A) mod p = (-1)^{#swaps} prod U_kk.
//
// Layout: W residue matrices, prime-major, R[w][i][j] int32 balanced, ld n.
// Small n: the whole matrix of one prime lives in shared memory (one CTA per
// prime). Larger n: right-looking blocked LU with panel width nb:
//   panel  (one CTA per prime, column by column, full-row swaps),
//   TRSM   U12 = L11^{-1} A12,
//   update A22 <- A22 - L21 U12 mod p (the O(n^3) part), int64 delayed
//          reduction on the CUDA cores: balanced residues of a 21-bit prime
//          have |x| < 2^20, so a K-term dot product stays below K 2^40.
// Lift-class primes (31 bits, |x| < 2^30, products < 2^60) fold the
// accumulator every 4 products.
#include <climits>
#include <cstdio>

#include <cooperative_groups.h>
#include <cuda_pipeline.h>

#include "idet_internal.cuh"

namespace idet {

namespace {

constexpr int kSmallN = 192;  // whole-matrix-in-shared-memory limit
constexpr int kPanelThreads = 1024;
constexpr int kNBMax = 32;
constexpr int kFoldWide = 4;

__device__ __forceinline__ uint32_t det_mul(uint32_t det, int32_t piv, const ModP &M) {
    return red_pos((int64_t)det * (int64_t)piv, M);
}

// ---------------------------------------------------------------------------
// Whole-matrix LU in shared memory.

// Inverse mod p < 2^31 by the extended Euclidean algorithm in 32-bit
// arithmetic (all remainders and cofactors stay below p in magnitude).
__device__ __forceinline__ int32_t inv_bal32(int32_t a, uint32_t p) {
    int32_t r0 = (int32_t)p, r1 = a % (int32_t)p;
    if (r1 < 0) r1 += (int32_t)p;
    int32_t t0 = 0, t1 = 1;
    while (r1 != 0) {
        int32_t q = r0 / r1, t;
        t = r0 - q * r1; r0 = r1; r1 = t;
        t = t0 - q * t1; t0 = t1; t1 = t;
    }
    if (t0 > (int32_t)(p - 1) / 2) t0 -= (int32_t)p;
    if (t0 < -(int32_t)(p - 1) / 2) t0 += (int32_t)p;
    return t0;
}

// Montgomery form with R = 2^32 for the panel: x' = x R mod p (balanced).
// For a product t (|t| < 2^62) and q = t p^{-1} mod 2^32 (as int32), t - q p
// is divisible by 2^32 and (t - q p) / 2^32 = hi(t) - hi(q p) (the low words
// agree) is t R^{-1} mod p, of magnitude below |t| / 2^32 + p / 2: one 32 x 32
// -> 64 product and two 32-bit multiplies per modular product.
struct Mont {
    int32_t p, half;
    uint32_t pinv;  // p^{-1} mod 2^32
    int32_t r1;     // 2^32 mod p, balanced
};

__device__ __forceinline__ Mont make_mont(uint32_t p) {
    Mont m;
    m.p = (int32_t)p;
    m.half = (int32_t)((p - 1) / 2);
    uint32_t x = p;  // p p = 1 mod 8; each step doubles the correct bits
    for (int i = 0; i < 4; ++i) x *= 2u - p * x;
    m.pinv = x;
    int64_t r = (int64_t)((1ull << 32) % p);
    if (r > m.half) r -= p;
    m.r1 = (int32_t)r;
    return m;
}

// d r - a u mod p for the fraction-free panel, with d' = d R and u' = u R
// (balanced, R = 2^32) formed once per pivot: t = d' r - a u' has |t| <= p^2/2
// < 2^61, and v = (t - q p) / 2^32 (q = t p^{-1} mod 2^32) is d r - a u mod p
// with |v| < p^2 / 2^33 + p / 2 < 0.75 p: one step either way balances it.
__device__ __forceinline__ int32_t ff_mont(int32_t dm, int32_t r, int32_t a, int32_t um,
                                           const Mont &m) {
    const int64_t t = (int64_t)dm * r - (int64_t)a * um;
    const int32_t q = (int32_t)((uint32_t)t * m.pinv);
    int32_t v = (int32_t)(t >> 32) - __mulhi(q, m.p);
    if (v > m.half) v -= m.p;
    if (v < -m.half) v += m.p;
    return v;
}

// g: the residues (n x n, ld n), or null with A64: the int64 entries (n x n,
// ld n), reduced here while they are loaded.
__device__ void lu_small_body(int32_t *__restrict__ g, int n, const ModP M,
                              LUState *__restrict__ st_out, int32_t *__restrict__ pm,
                              const int64_t *__restrict__ A64 = nullptr) {
    extern __shared__ int32_t sa[];
    __shared__ int s_piv;
    __shared__ int32_t s_inv;
    const int nn = n * n;
    if (A64)
        for (int e = threadIdx.x; e < nn; e += blockDim.x) sa[e] = red_bal(A64[e], M);
    else
        for (int e = threadIdx.x; e < nn; e += blockDim.x) sa[e] = g[e];
    if (pm)
        for (int i = threadIdx.x; i < n; i += blockDim.x) pm[i] = i;
    uint32_t det = 1u % M.p;
    int neg = 0, dead = 0;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) s_piv = sa[k * n + k] != 0 ? k : INT_MAX;
        __syncthreads();
        if (s_piv == INT_MAX) {
            for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x)
                if (sa[i * n + k] != 0) atomicMin(&s_piv, i);
            __syncthreads();
        }
        const int piv = s_piv;
        if (piv == INT_MAX) {
            dead = 1;
            break;
        }
        if (piv != k) {
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                int32_t t = sa[k * n + j];
                sa[k * n + j] = sa[piv * n + j];
                sa[piv * n + j] = t;
            }
            if (threadIdx.x == 0 && pm) {
                int32_t t = pm[k];
                pm[k] = pm[piv];
                pm[piv] = t;
            }
            neg ^= 1;
            __syncthreads();
        }
        const int32_t pv = sa[k * n + k];
        if (threadIdx.x == 0) s_inv = inv_bal32(pv, M.p);
        det = det_mul(det, pv, M);
        __syncthreads();
        const int32_t inv = s_inv;
        // a warp per row below the pivot: lane 0 forms the multiplier, the
        // lanes update the row's columns
        const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int i = k + 1 + (threadIdx.x >> 5); i < n; i += nw) {
            int32_t l = 0;
            if (lane == 0) {
                l = mul_bal(sa[i * n + k], inv, M);
                sa[i * n + k] = l;
            }
            l = __shfl_sync(0xffffffffu, l, 0);
            if (l)
                for (int j = k + 1 + lane; j < n; j += 32)
                    sa[i * n + j] = red_bal((int64_t)sa[i * n + j] - (int64_t)l * sa[k * n + j], M);
        }
        __syncthreads();
    }
    if (g)
        for (int e = threadIdx.x; e < nn; e += blockDim.x) g[e] = sa[e];
    if (threadIdx.x == 0) {
        LUState s;
        s.dead = dead;
        s.neg = neg;
        s.det = dead ? 0u : det;
        s.pad = 0;
        *st_out = s;
    }
}

__global__ void k_lu_small(int32_t *__restrict__ R, int n, const ModP *__restrict__ mods,
                           LUState *__restrict__ st, int32_t *__restrict__ perm) {
    const int w = blockIdx.x;
    lu_small_body(R + (int64_t)w * n * n, n, mods[w], st + w, perm ? perm + (int64_t)w * n : nullptr);
}

// One CTA per (matrix, prime) job of a batch.
__global__ void k_lu_small_multi(const LUSmallJob *__restrict__ jobs) {
    const LUSmallJob j = jobs[blockIdx.x];
    lu_small_body(j.R, j.n, j.mod, j.st, nullptr, j.A64);
    __syncthreads();
    if (threadIdx.x == 0) {
        const LUState t = *j.st;
        uint32_t d = t.dead ? 0u : t.det;
        if (t.neg && d) d = j.mod.p - d;
        *j.det = d;
    }
}

// ---------------------------------------------------------------------------
// Blocked LU pieces.

__global__ void k_state_init(LUState *st, const ModP *mods, int W, int32_t *perm, int64_t n) {
    int w = blockIdx.x;
    if (threadIdx.x == 0) {
        LUState s;
        s.det = 1u % mods[w].p;
        s.neg = 0;
        s.dead = 0;
        s.pad = 0;
        st[w] = s;
    }
    if (perm)
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) perm[(int64_t)w * n + i] = (int32_t)i;
}

// Factor the panel of columns [j0, j0 + jb) on rows [j0, n); rows are swapped
// across all n columns.
__global__ void __launch_bounds__(kPanelThreads)
k_panel(int32_t *__restrict__ R, int64_t n, int64_t j0, int jb,
        const ModP *__restrict__ mods, LUState *__restrict__ st,
        int32_t *__restrict__ perm) {
    __shared__ int32_t s_u[kNBMax];
    __shared__ int s_piv;
    __shared__ int32_t s_inv;
    const int w = blockIdx.x;
    if (st[w].dead) return;
    const ModP M = mods[w];
    int32_t *a = R + (int64_t)w * n * n;
    uint32_t det = st[w].det;
    int neg = st[w].neg;
    for (int c = 0; c < jb; ++c) {
        const int64_t col = j0 + c;
        if (threadIdx.x == 0) s_piv = a[col * n + col] != 0 ? (int)col : INT_MAX;
        __syncthreads();
        if (s_piv == INT_MAX) {
            for (int64_t i = col + 1 + threadIdx.x; i < n; i += blockDim.x)
                if (a[i * n + col] != 0) atomicMin(&s_piv, (int)i);
            __syncthreads();
        }
        const int piv = s_piv;
        if (piv == INT_MAX) {
            if (threadIdx.x == 0) {
                LUState s = st[w];
                s.dead = 1;
                s.det = 0;
                st[w] = s;
            }
            return;
        }
        if (piv != col) {
            for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
                int32_t t = a[col * n + j];
                a[col * n + j] = a[(int64_t)piv * n + j];
                a[(int64_t)piv * n + j] = t;
            }
            if (threadIdx.x == 0 && perm) {
                int32_t *pm = perm + (int64_t)w * n;
                int32_t t = pm[col];
                pm[col] = pm[piv];
                pm[piv] = t;
            }
            neg ^= 1;
            __syncthreads();
        }
        const int32_t pv = a[col * n + col];
        det = det_mul(det, pv, M);
        if (threadIdx.x == 0) s_inv = inv_bal(pv, M.p);
        if (threadIdx.x > c && threadIdx.x < jb) s_u[threadIdx.x] = a[col * n + j0 + threadIdx.x];
        __syncthreads();
        const int32_t inv = s_inv;
        for (int64_t i = col + 1 + threadIdx.x; i < n; i += blockDim.x) {
            int32_t *row = a + i * n + j0;
            int32_t l = mul_bal(row[c], inv, M);
            row[c] = l;
            if (l)
                for (int j = c + 1; j < jb; ++j)
                    row[j] = red_bal((int64_t)row[j] - (int64_t)l * s_u[j], M);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        LUState s = st[w];
        s.det = det;
        s.neg = neg;
        st[w] = s;
    }
}


// Panel factorisation by a cluster of CL CTAs (one cluster per prime).
// The panel (rows [j0, n), columns [j0, j0 + jb)) is split into CL
// contiguous row blocks held in the CTAs' shared memory for the whole
// panel. Every CTA also keeps a replica of the panel's top jb rows -- the
// rows that become the pivot rows -- and applies the same eliminations to
// it, so that each CTA knows every pivot row and pivot without
// communication: a column costs one CTA barrier.
//
// The elimination inside the panel is fraction-free: column c updates each
// row below its pivot d_c by r <- d_c r - a u (a the row's entry in column
// c, u the pivot row), so no modular inverse lies on the chain from one
// column to the next. Every row below pivot c then carries the same factor
// S_c = d_0 ... d_(c-1) (S_0 = 1): the true pivot is d_c / S_c, the true
// multiplier of a row is its stored entry a / d_c (the factors cancel), and
// the true pivot row is the stored one over S_c. At the end of the panel the
// inverses of d_c and S_c come from one modular inverse (Montgomery's batch
// trick) and every row is normalised to the ordinary L and U. Warp 0
// eliminates the next pivot row of the replica first and forms its
// Montgomery form while the other warps update their rows. Only a zero pivot
// (first-nonzero rule; S_c != 0, so the stored and true pivots vanish
// together) needs the cluster: the first nonzero row below it is found across
// the CTAs and the two rows are exchanged in the owners' blocks (through
// distributed shared memory), in every replica, and outside the panel in
// global memory.
//
// That column loop runs only when the replica's block has a zero pivot. In
// the common case one warp factors the block alone first; with all its
// pivots nonzero the rule pivots on the panel's top rows in order, and each
// thread then solves its rows against U11 with no barrier at all.
constexpr int kCl = 8;  // portable cluster size; 16 (opt-in) when few primes leave SMs idle
constexpr int kClThreads = 512;
constexpr int kSP = kNBMax + 1;  // row stride of a CTA's panel block in shared memory

// t R^{-1} mod p for |t| < 2^62 (R = 2^32): (t - q p) / 2^32 with
// q = t p^{-1} mod 2^32, of magnitude below |t| / 2^32 + p / 2.
__device__ __forceinline__ int32_t redc64(int64_t t, const Mont &m) {
    const int32_t q = (int32_t)((uint32_t)t * m.pinv);
    return (int32_t)(t >> 32) - __mulhi(q, m.p);
}

// a b R^{-1} mod p, balanced, for |a b| < p 2^32.
__device__ __forceinline__ int32_t mont_mul(int32_t a, int32_t b, const Mont &m) {
    int32_t v = redc64((int64_t)a * b, m);
    if (v > m.half) v -= m.p;
    if (v < -m.half) v += m.p;
    return v;
}

// 1 / x = x^(p-2) mod p (Fermat) for x != 0, argument and result in
// Montgomery form: square and multiply over the bits of p - 2.
__device__ __forceinline__ int32_t mont_inv(int32_t xm, const Mont &m) {
    const uint32_t e = (uint32_t)m.p - 2;
    int32_t r = m.r1;  // 1 in Montgomery form
    for (int b = 31 - __clz(e); b >= 0; --b) {
        r = mont_mul(r, r, m);
        if ((e >> b) & 1) r = mont_mul(r, xm, m);
    }
    return r;
}

// The panel's common case: when every pivot of the replica's jb x jb block
// is nonzero, the first-nonzero rule takes the panel's top rows in order,
// U11 is the block's U, and every row below solves x U11 = a for its L part
// on its own, with no barrier per column.
//
// replica_lu_cta (all threads): fraction-free LU of the block in Montgomery
// form (d' r' - a' u' reduced once is (d r - a u)'), thread (i, g) updating
// columns g and g + 16 of row i, one CTA barrier per column. False
// (CTA-uniform) at the first zero pivot, with dg untouched. Otherwise lane c
// of a warp inverts d_c (Fermat), the prefix products S_c of the pivots and
// their inverses come from two product scans across the warp, and dg is
// overwritten with the
// block's normalised factors (L_ic = s_ic / d_c below the diagonal, U_ic =
// s_ic / S_i on and above it). -U_kc for k < c < jb (zero elsewhere) goes to
// ut[c][k] for 21-bit primes (narrow), else split at bit 16 into its low
// (ut) and high (ut2) parts; w[c] = 1 / U_cc = S_c / d_c times R^2 (narrow)
// or R^3, for the solves' Montgomery steps; *detf = prod U_cc.
struct ReplicaScratch {
    int32_t fa[kNBMax * kSP];  // the block in Montgomery form
    int32_t invd[kNBMax], invS[kNBMax];
};

__device__ bool replica_lu_cta(int32_t *dg, int jb, const ModP &M, const Mont &mt,
                               ReplicaScratch &rs, int32_t *ut, int32_t *ut2, int32_t *w,
                               bool narrow, int32_t *detf) {
    const int tid = threadIdx.x, lane = tid & 31, g = tid >> 5;
    const int32_t r2 = mul_bal(mt.r1, mt.r1, M);  // R^2 mod p
    for (int e = tid; e < jb * jb; e += blockDim.x) {
        const int i = e / jb, j = e % jb;
        rs.fa[i * kSP + j] = mont_mul(dg[i * kSP + j], r2, mt);
    }
    __syncthreads();
    static_assert(kClThreads == 16 * 32, "thread (i, g) covers columns g and g + 16");
    for (int c = 0; c < jb; ++c) {
        const int32_t dm = rs.fa[c * kSP + c];
        if (dm == 0) return false;  // every thread reads the same pivot
        if (lane > c && lane < jb) {
            int32_t *row = rs.fa + lane * kSP;
            const int32_t *piv = rs.fa + c * kSP;
            const int32_t am = row[c];
            const int32_t x0 = row[g], u0 = piv[g], x1 = row[g + 16], u1 = piv[g + 16];
            if (g > c && g < jb) row[g] = ff_mont(dm, x0, am, u0, mt);
            if (g + 16 > c && g + 16 < jb) row[g + 16] = ff_mont(dm, x1, am, u1, mt);
        }
        __syncthreads();
    }
    if (tid < 32) {
        // all in Montgomery form; lanes past jb carry 1
        const unsigned full = 0xffffffffu;
        const int32_t dm = lane < jb ? rs.fa[lane * kSP + lane] : mt.r1;  // d_c
        const int32_t idm = mont_inv(dm, mt);                               // 1 / d_c
        int32_t S = dm, iS = idm;  // inclusive prefix products, then shifted
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t t = __shfl_up_sync(full, S, o), ti = __shfl_up_sync(full, iS, o);
            if (lane >= o) {
                S = mont_mul(S, t, mt);
                iS = mont_mul(iS, ti, mt);
            }
        }
        S = __shfl_up_sync(full, S, 1);  // S_c = d_0 ... d_(c-1)
        iS = __shfl_up_sync(full, iS, 1);
        if (lane == 0) S = iS = mt.r1;
        int32_t uf = lane < jb ? mont_mul(dm, iS, mt) : mt.r1;  // U_cc = d_c / S_c
#pragma unroll
        for (int o = 16; o; o >>= 1) uf = mont_mul(uf, __shfl_xor_sync(full, uf, o), mt);
        rs.invd[lane] = mont_mul(idm, 1, mt);
        rs.invS[lane] = mont_mul(iS, 1, mt);
        const int32_t ium = mont_mul(S, idm, mt);  // 1 / U_cc = S_c / d_c
        // R^2 / U_cc (21-bit) or R^3 / U_cc for the solves' Montgomery steps
        const int32_t wm = narrow ? r2 : mont_mul(r2, r2, mt);
        w[lane] = lane < jb ? mont_mul(ium, wm, mt) : 0;
        if (lane == 0) *detf = mont_mul(uf, 1, mt);
    }
    __syncthreads();
    for (int e = tid; e < kNBMax * kNBMax; e += blockDim.x) {
        const int i = e & 31, j = e >> 5;  // row i, column j
        int32_t v = 0;
        if (i < jb && j < jb) {
            v = mont_mul(rs.fa[i * kSP + j], j < i ? rs.invd[j] : rs.invS[i], mt);
            dg[i * kSP + j] = v;
        }
        const int32_t nu = (i < j && j < jb) ? -v : 0;  // -U_ij at [j][i]
        ut[j * kNBMax + i] = narrow ? nu : (nu & 0xffff);
        if (!narrow) ut2[j * kNBMax + i] = nu >> 16;
    }
    __syncthreads();
    return true;
}

// x U11 = a for one row below the replica (a: the row's jb panel entries,
// overwritten in place by x, its L part, column by column):
// x_c = (a_c - sum_{k<c} x_k U_kc) / U_cc with ut and w from replica_lu_cta
// (ut[c][k] = 0 for k >= c: the sum runs over all 32 columns, the entries
// past c, solved or not, meeting zeros).
// per = 2: two threads share the row (lanes 2m and 2m + 1, mask their pair),
// each summing every other group of four, the halves exchanged by a shuffle;
// both then hold x_c and store the same value.
// 21-bit primes: at most 31 products below 2^40, exact in int64, reduced
// once by two Montgomery steps (w_c = R^2 / U_cc).
template <int per>
__device__ __forceinline__ void solve_row_narrow(int32_t *row, int jb, const int32_t *ut,
                                                 const int32_t *w, const Mont &mt, int h,
                                                 unsigned mask) {
    for (int c = 0; c < jb; ++c) {
        const int32_t *u = ut + c * kNBMax;
        const int32_t ac = row[c];
        int64_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;  // four chains
        // every group of four (no loop branch; the terms past c are zero)
#pragma unroll
        for (int i = 0; i < 8 / per; ++i) {
            const int k = 4 * (per * i + h);
            const int4 q = *reinterpret_cast<const int4 *>(u + k);
            a0 += (int64_t)row[k] * q.x;
            a1 += (int64_t)row[k + 1] * q.y;
            a2 += (int64_t)row[k + 2] * q.z;
            a3 += (int64_t)row[k + 3] * q.w;
        }
        int64_t sum = (a0 + a1) + (a2 + a3);
        if (per == 2) sum += __shfl_xor_sync(mask, sum, 1);
        row[c] = mont_mul(redc64(sum + ac, mt), w[c], mt);
    }
}

// The same for primes up to 2^31: -U_kc split at bit 16 (ut: its low 16
// bits, ut2: the rest), two int64 sums of terms below 2^46 and 2^44, reduced
// by three Montgomery steps and a Montgomery product with w_c = R^3 / U_cc.
template <int per>
__device__ __forceinline__ void solve_row_wide(int32_t *row, int jb, const int32_t *ut,
                                               const int32_t *ut2, const int32_t *w,
                                               const Mont &mt, int hf, unsigned mask) {
    for (int c = 0; c < jb; ++c) {
        const int32_t *u = ut + c * kNBMax, *h = ut2 + c * kNBMax;
        const int32_t ac = row[c];
        int64_t lo = 0, lo2 = 0, hi = 0, hi2 = 0;  // two chains each
#pragma unroll
        for (int i = 0; i < 8 / per; ++i) {
            const int k = 4 * (per * i + hf);
            const int4 q = *reinterpret_cast<const int4 *>(u + k);
            const int4 r = *reinterpret_cast<const int4 *>(h + k);
            const int32_t x0 = row[k], x1 = row[k + 1], x2 = row[k + 2], x3 = row[k + 3];
            lo += (int64_t)x0 * q.x + (int64_t)x2 * q.z;
            lo2 += (int64_t)x1 * q.y + (int64_t)x3 * q.w;
            hi += (int64_t)x0 * r.x + (int64_t)x2 * r.z;
            hi2 += (int64_t)x1 * r.y + (int64_t)x3 * r.w;
        }
        lo += lo2;
        hi += hi2;
        if (per == 2) {
            lo += __shfl_xor_sync(mask, lo, 1);
            hi += __shfl_xor_sync(mask, hi, 1);
        }
        // t = (lo + 2^16 hi) R^{-1} below 2^47, then t R^{-1} below 2^15 + p/2,
        // times w_c = R^3 / U_cc with one more Montgomery step
        const int64_t t = (int64_t)redc64(hi, mt) * 65536 + redc64(lo + ac, mt);
        row[c] = mont_mul(redc64(t, mt), w[c], mt);
    }
}

// L11^{-1} for the panel's triangular solves. X (32 rows of stride kSP)
// holds the unit lower triangular L11 below its diagonal (jb x jb; rows and
// columns past jb are the identity's); block inversion in place: for the
// diagonal blocks of size s = 2h, whose halves are already inverted,
// X21 <- -X22 (T21 X11) with the product T21 X11 formed in Y first. Five
// levels of two small products, all blocks of a level at once, at most 16
// terms per entry (exact in int64 for 21-bit residues, split at bit 16
// otherwise). Written to out[i][j] (32 x 32, zero outside jb x jb). All the
// CTA's threads, or (NAMED) warps 8-15 alone, synchronised by barrier 1.
template <bool NAMED>
__device__ void tri_inv_lower_cta(int32_t *X, int32_t *Y, const int32_t *dg, int jb,
                                  const ModP &M, bool narrow, int32_t *out) {
    const int tid = NAMED ? (int)threadIdx.x - 256 : (int)threadIdx.x;
    const int nt = NAMED ? 256 : (int)blockDim.x;
    auto sync = [] {
        if (NAMED)
            asm volatile("bar.sync 1, 256;" ::: "memory");
        else
            __syncthreads();
    };
    for (int e = tid; e < kNBMax * kNBMax; e += nt) {
        const int i = e >> 5, j = e & 31;
        X[i * kSP + j] = (j < i && i < jb) ? dg[i * kSP + j] : (i == j ? 1 : 0);
    }
    sync();
    auto dot_fin = [&](int64_t lo, int64_t hi) {
        return narrow ? red_bal(lo, M) : red_bal((int64_t)red_bal(hi, M) * 65536 + red_bal(lo, M), M);
    };
    for (int h = 1; h < kNBMax; h <<= 1) {
        const int hh = h * h, nent = (kNBMax / (2 * h)) * hh;
        const bool act = tid < nent;
        const int b = act ? tid / hh : 0, r = act ? (tid % hh) / h : 0, c = act ? tid % h : 0;
        const int o = 2 * h * b;
        const int32_t *xr = X + (o + h + r) * kSP + o;  // row o + h + r from column o
        if (act) {
            // Y = T21 X11: sum over c <= k < h (X11 is lower triangular)
            int64_t lo = 0, hi = 0;
            for (int k = c; k < h; ++k) {
                const int32_t t = xr[k], u = X[(o + k) * kSP + o + c];
                if (narrow) {
                    lo += (int64_t)t * u;
                } else {
                    lo += (int64_t)t * (u & 0xffff);
                    hi += (int64_t)t * (u >> 16);
                }
            }
            Y[tid] = dot_fin(lo, hi);
        }
        sync();
        if (act) {
            // X21 = -X22 Y: sum over 0 <= k <= r (X22 is lower triangular)
            int64_t lo = 0, hi = 0;
            for (int k = 0; k <= r; ++k) {
                const int32_t t = xr[h + k], u = Y[b * hh + k * h + c];
                if (narrow) {
                    lo += (int64_t)t * u;
                } else {
                    lo += (int64_t)t * (u & 0xffff);
                    hi += (int64_t)t * (u >> 16);
                }
            }
            X[(o + h + r) * kSP + o + c] = -dot_fin(lo, hi);
        }
        sync();
    }
    for (int e = tid; e < kNBMax * kNBMax; e += nt) {
        const int i = e >> 5, j = e & 31;
        out[e] = (i < jb && j < jb) ? X[i * kSP + j] : 0;
    }
}

template <int CL>
__global__ void __launch_bounds__(kClThreads, 2)
k_panel_cluster(int32_t *__restrict__ R, int64_t n, int64_t j0, int jb, int chunk,
                const ModP *__restrict__ mods, LUState *__restrict__ st,
                int32_t *__restrict__ perm, int32_t *__restrict__ tri) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ int32_t sp[];         // chunk x kSP: this CTA's rows
    __shared__ int32_t dg[kNBMax * kSP];    // replica of rows [j0, j0 + jb)
    __shared__ int32_t s_dm[2];             // pivot of column c in Montgomery form, slot c & 1
    __shared__ int s_cand;                  // first nonzero row below a zero pivot
    __shared__ int32_t s_tmp[2][kNBMax];    // the two rows of an exchange
    __shared__ int32_t s_um[2][kNBMax];     // pivot row of column c in Montgomery form, slot c & 1
    __shared__ int32_t s_invd[kNBMax], s_invS[kNBMax];  // 1 / d_c and 1 / S_c
    __shared__ __align__(16) int32_t s_ut[kNBMax * kNBMax];  // -U_kc at [c][k], k < c
    __shared__ __align__(16) int32_t s_ut2[kNBMax * kNBMax]; // its high part (31-bit p)
    __shared__ int32_t s_w[kNBMax];                         // 1 / U_cc (times R^2: 21-bit p)
    __shared__ int32_t s_detf;                              // prod U_cc
    __shared__ ReplicaScratch s_rs;
    __shared__ int32_t s_y[kNBMax * kNBMax / 4];  // block inversion scratch
    const int rank = (int)cluster.block_rank();
    const int w = blockIdx.x / CL;
    const ModP M = mods[w];
    int32_t *a = R + (int64_t)w * n * n;
    const bool dead0 = st[w].dead != 0;  // uniform over the cluster
    if (dead0) return;
    const int64_t rbeg = j0 + (int64_t)rank * chunk;
    const int64_t rend = min(n, rbeg + chunk);
    const int nloc = rend > rbeg ? (int)(rend - rbeg) : 0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // a warp per row: asynchronous copies, all in flight at once
    if (lane < jb) {
        for (int r = warp; r < nloc; r += kClThreads / 32)
            __pipeline_memcpy_async(&sp[r * kSP + lane], &a[(rbeg + r) * n + j0 + lane], 4);
        for (int r = warp; r < jb; r += kClThreads / 32)
            __pipeline_memcpy_async(&dg[r * kSP + lane], &a[(j0 + r) * n + j0 + lane], 4);
    }
    __pipeline_commit();
    __pipeline_wait_prior(0);
    uint32_t det = st[w].det;
    int neg = st[w].neg;
    bool dead = false;
    const Mont mt = make_mont(M.p);
    __syncthreads();
    // the common case first (every replica pivot nonzero): the CTA factors
    // the replica, then each thread solves its rows below it
    const bool narrow = M.p < (1u << 21);
    // (the replicas agree: uniform over the cluster)
    const bool fast = replica_lu_cta(dg, jb, M, mt, s_rs, s_ut, s_ut2, s_w, narrow, &s_detf);
    // L11^{-1} for the triangular solves comes from the last CTA, which has
    // the fewest rows (its replica scratch is free once the factors are out):
    // on warps 8-15 beside the rows when warps 0-7 can take them all
    const bool tri_here = tri && rank == CL - 1;
    int32_t *tri_w = tri ? tri + (int64_t)w * kNBMax * kNBMax : nullptr;
    if (fast) {
        const bool split = tri_here && nloc <= kClThreads / 2;
        if (tri_here && !split) tri_inv_lower_cta<false>(s_rs.fa, s_y, dg, jb, M, narrow, tri_w);
        if (split && warp >= 8) {
            tri_inv_lower_cta<true>(s_rs.fa, s_y, dg, jb, M, narrow, tri_w);
        } else {
            const int nt = split ? kClThreads / 2 : kClThreads;  // threads on rows
            const int per = 2 * nloc <= nt ? 2 : 1;              // threads per row
            const int h = tid % per;
            const unsigned mask = per == 2 ? 3u << (lane & 30) : 0xffffffffu;
            for (int r = tid / per; r < nloc; r += nt / per) {
                const int64_t gr = rbeg + r - j0;  // row within the panel
                int32_t *row = sp + r * kSP;
                if (gr < jb) {
                    for (int j = 0; j < jb; ++j) row[j] = dg[gr * kSP + j];
                } else if (per == 2) {
                    if (narrow)
                        solve_row_narrow<2>(row, jb, s_ut, s_w, mt, h, mask);
                    else
                        solve_row_wide<2>(row, jb, s_ut, s_ut2, s_w, mt, h, mask);
                } else {
                    if (narrow)
                        solve_row_narrow<1>(row, jb, s_ut, s_w, mt, 0, mask);
                    else
                        solve_row_wide<1>(row, jb, s_ut, s_ut2, s_w, mt, 0, mask);
                }
            }
        }
        if (tid == 0) det = det_mul(det, s_detf, M);
    } else {
        if (tid == 0) s_dm[0] = mul_bal(dg[0], mt.r1, M);
        if (tid < jb) s_um[0][tid] = mul_bal(dg[tid], mt.r1, M);
        __syncthreads();
        for (int c = 0; c < jb; ++c) {
            const int64_t col = j0 + c;
            if (dg[c * kSP + c] == 0) {
                // (the replicas are identical: every CTA of the cluster is here)
                if (tid == 0) s_cand = INT_MAX;
                cluster.sync();
                for (int r = tid; r < nloc; r += kClThreads) {
                    const int64_t gi = rbeg + r;
                    if (gi > col && sp[r * kSP + c] != 0) atomicMin(&s_cand, (int)gi);
                }
                cluster.sync();
                int best = INT_MAX;
                for (int k = 0; k < CL; ++k)
                    best = min(best, *cluster.map_shared_rank(&s_cand, k));
                if (best == INT_MAX) {
                    dead = true;
                    break;
                }
                const int64_t piv = best;
                const int po = (int)((piv - j0) / chunk), co = (int)((col - j0) / chunk);
                int32_t *prow = cluster.map_shared_rank(sp, po) +
                                (int)(piv - (j0 + (int64_t)po * chunk)) * kSP;
                int32_t *crow = cluster.map_shared_rank(sp, co) +
                                (int)(col - (j0 + (int64_t)co * chunk)) * kSP;
                if (tid < jb) {
                    s_tmp[0][tid] = crow[tid];
                    s_tmp[1][tid] = prow[tid];
                }
                cluster.sync();  // both rows read everywhere before they change
                if (rank == 0 && tid < jb) {
                    crow[tid] = s_tmp[1][tid];
                    prow[tid] = s_tmp[0][tid];
                }
                if (tid < jb) {
                    dg[c * kSP + tid] = s_tmp[1][tid];
                    if (piv < j0 + jb) dg[(int)(piv - j0) * kSP + tid] = s_tmp[0][tid];
                }
                // parts outside the panel, in global memory (rank 0)
                if (rank == 0) {
                    for (int64_t j = tid; j < n; j += kClThreads) {
                        if (j >= j0 && j < j0 + jb) continue;
                        int32_t t = a[col * n + j];
                        a[col * n + j] = a[piv * n + j];
                        a[piv * n + j] = t;
                    }
                    if (tid == 0 && perm) {
                        int32_t *pm = perm + (int64_t)w * n;
                        int32_t t = pm[col];
                        pm[col] = pm[piv];
                        pm[piv] = t;
                    }
                }
                neg ^= 1;
                cluster.sync();
                if (tid == 0) s_dm[c & 1] = mul_bal(dg[c * kSP + c], mt.r1, M);
                if (tid < jb) s_um[c & 1][tid] = mul_bal(dg[c * kSP + tid], mt.r1, M);
                __syncthreads();
            }
            const int32_t dm = s_dm[c & 1];
            const int32_t *um = s_um[c & 1];
            if (warp == 0) {
                // the next pivot row of the replica, then its Montgomery form
                if (c + 1 < jb) {
                    int32_t *row = dg + (c + 1) * kSP;
                    const int32_t av = row[c];
                    if (lane > c && lane < jb) row[lane] = ff_mont(dm, row[lane], av, um[lane], mt);
                    __syncwarp();
                    if (lane < jb) s_um[(c + 1) & 1][lane] = mul_bal(row[lane], mt.r1, M);
                    if (lane == 0) s_dm[(c + 1) & 1] = mul_bal(row[c + 1], mt.r1, M);
                }
            } else {
                // a thread per row: this CTA's rows below the pivot, then the
                // replica's rows c + 2 .. jb - 1 (the row stride kSP = 33 words
                // keeps the lanes of a warp on distinct banks); the entry in
                // column c stays as the row's (unnormalised) multiplier
                const int items = nloc + max(0, jb - c - 2);
                for (int it = tid - 32; it < items; it += kClThreads - 32) {
                    int32_t *row;
                    if (it < nloc) {
                        if (rbeg + it <= col) continue;
                        row = sp + it * kSP;
                    } else {
                        row = dg + (c + 2 + (it - nloc)) * kSP;
                    }
                    // (a zero entry still scales the row by d_c: every row below
                    // the pivot must carry the same factor S_(c+1))
                    const int32_t av = row[c];
                    for (int j = c + 1; j < jb; ++j) row[j] = ff_mont(dm, row[j], av, um[j], mt);
                }
            }
            __syncthreads();
        }
        if (!dead) {
            // 1 / d_c and 1 / S_c (S_c = d_0 ... d_(c-1)) from one inverse:
            // prefix products P_c = d_0 ... d_c, then 1 / P_(jb-1) unwound
            if (tid == 0) {
                int32_t pre[kNBMax];
                int32_t pr = 1;
                for (int c = 0; c < jb; ++c) {
                    pr = mul_bal(pr, dg[c * kSP + c], M);
                    pre[c] = pr;
                }
                int32_t ip = inv_bal32(pr, M.p);  // 1 / P_(jb-1)
                for (int c = jb - 1; c >= 0; --c) {
                    // 1 / d_c = P_(c-1) / P_c; 1 / P_(c-1) = d_c / P_c
                    s_invd[c] = c > 0 ? mul_bal(ip, pre[c - 1], M) : ip;
                    ip = mul_bal(ip, dg[c * kSP + c], M);
                }
                int32_t is = 1;  // 1 / S_c = 1 / P_(c-1)
                for (int c = 0; c < jb; ++c) {
                    s_invS[c] = is;
                    is = mul_bal(is, s_invd[c], M);
                }
                // det *= prod_c d_c / S_c
                for (int c = 0; c < jb; ++c)
                    det = det_mul(det, mul_bal(dg[c * kSP + c], s_invS[c], M), M);
            }
            __syncthreads();
            // normalise this CTA's rows: multipliers (columns below the row's
            // diagonal) times 1 / d_c; a pivot row's U part times 1 / S_r
            for (int e = tid; e < nloc * jb; e += kClThreads) {
                const int r = e / jb, j = e % jb;
                const int64_t gr = rbeg + r - j0;  // row within the panel
                int32_t &v = sp[r * kSP + j];
                if (j < gr)
                    v = mul_bal(v, s_invd[j], M);
                else
                    v = mul_bal(v, s_invS[gr], M);
            }
            if (tri_here) {
                // the replica's L part likewise, for L11^{-1} below
                for (int e = tid; e < jb * jb; e += kClThreads) {
                    const int r = e / jb, j = e % jb;
                    if (j < r) dg[r * kSP + j] = mul_bal(dg[r * kSP + j], s_invd[j], M);
                }
            }
        }
    }
    cluster.sync();  // no CTA leaves while others may still read its block
    if (dead) {
        if (rank == 0 && tid == 0) {
            LUState s = st[w];
            s.dead = 1;
            s.det = 0;
            st[w] = s;
        }
        return;
    }
    if (lane < jb)
        for (int r = warp; r < nloc; r += kClThreads / 32)
            a[(rbeg + r) * n + j0 + lane] = sp[r * kSP + lane];
    if (rank == 0 && tid == 0) {
        LUState s = st[w];
        s.det = det;
        s.neg = neg;
        st[w] = s;
    }
    if (!fast && tri_here) tri_inv_lower_cta<false>(s_rs.fa, s_y, dg, jb, M, narrow, tri_w);
}

// X[r0 .. r0+jb)[cols] <- L^{-1} X, L unit lower triangular (jb x jb) at
// (lr0, lr0) of matrix Lm (ld n). One thread per column.
template <bool WIDE>
__global__ void k_trsm_lower(const int32_t *__restrict__ Lm, int64_t strideL,
                             int32_t *__restrict__ X, int64_t strideX, int64_t n,
                             int64_t lr0, int64_t xr0, int jb, int64_t c0,
                             int64_t ncols, const ModP *__restrict__ mods,
                             const LUState *__restrict__ st) {
    __shared__ int32_t sL[kNBMax][kNBMax + 1];
    const int w = blockIdx.y;
    if (st && st[w].dead) return;
    const ModP M = mods[w];
    const int32_t *L = Lm + (int64_t)w * strideL;
    int32_t *x = X + (int64_t)w * strideX;
    for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
        int r = e / jb, k = e % jb;
        sL[r][k] = L[(lr0 + r) * n + lr0 + k];
    }
    __syncthreads();
    const int64_t j = c0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= c0 + ncols) return;
    int32_t u[kNBMax];
#pragma unroll
    for (int r = 0; r < kNBMax; ++r) {
        if (r < jb) {
            int64_t acc = x[(xr0 + r) * n + j];
#pragma unroll
            for (int k = 0; k < kNBMax; ++k) {
                if (k < r) {
                    acc -= (int64_t)sL[r][k] * u[k];
                    if (WIDE && (k % kFoldWide) == kFoldWide - 1) acc = red_bal(acc, M);
                }
            }
            u[r] = red_bal(acc, M);
            x[(xr0 + r) * n + j] = u[r];
        }
    }
}

// Triangular solves by explicit inverses of the nb x nb diagonal blocks:
// k_tri_inv forms T^{-1} once per prime (one thread per column of the
// inverse: forward substitution on e_c for a unit lower T, backward with the
// diagonal inverses for an upper T), k_tri_apply then computes
// X_block <- T^{-1} X_block for all columns as independent 32-term dot
// products (all reads of a column before the block barrier, all writes
// after it, so the update in place is safe). The nb-step dependency chain is
// paid once per block instead of once per column.
// sum_k t_k u_k mod p for balanced residues: one exact int64 sum for 21-bit
// primes, two (u split at bit 16) for 31-bit primes; |sum| < 2^53 for 32
// terms either way.
template <bool WIDE>
struct DotAcc {
    int64_t lo = 0, hi = 0;
    __device__ __forceinline__ void add(int32_t t, int32_t u) {
        if (WIDE) {
            lo += (int64_t)t * (u & 0xffff);
            hi += (int64_t)t * (u >> 16);
        } else {
            lo += (int64_t)t * u;
        }
    }
    __device__ __forceinline__ int32_t get(const ModP &M) const {
        return WIDE ? red_bal((int64_t)red_bal(hi, M) * 65536 + red_bal(lo, M), M)
                    : red_bal(lo, M);
    }
};

// Inverse of a triangular kNBMax x kNBMax block by products only: a unit
// lower T = I + N has N nilpotent (N^32 = 0), so
//   T^{-1} = (I - N)(I + N^2)(I + N^4)(I + N^8)(I + N^16);
// an upper T = D (I + N') with N' = D^{-1} (T - D) strictly upper gives
// T^{-1} = (I + N')^{-1} D^{-1}. Eight 32 x 32 products, one output entry
// per thread (1024 threads); rows and columns beyond jb are the identity.
template <bool WIDE, bool UPPER>
__global__ void __launch_bounds__(kNBMax * kNBMax)
k_tri_inv(const int32_t *__restrict__ Tm, int64_t strideT, int64_t n, int64_t r0, int jb,
          const ModP *__restrict__ mods, const LUState *__restrict__ st, int32_t *__restrict__ Inv) {
    __shared__ int32_t sP[kNBMax][kNBMax + 1], sS[kNBMax][kNBMax + 1], sQ[kNBMax][kNBMax + 1];
    __shared__ int32_t sD[kNBMax];
    const int w = blockIdx.x;
    if (st && st[w].dead) return;
    const ModP M = mods[w];
    const int32_t *T = Tm + (int64_t)w * strideT;
    const int i = threadIdx.x / kNBMax, j = threadIdx.x % kNBMax;
    const int32_t t = (i < jb && j < jb) ? T[(r0 + i) * n + r0 + j] : 0;
    if (UPPER && i == j) sD[i] = i < jb ? inv_bal32(t, M.p) : 1;
    __syncthreads();
    // N: strictly lower (unit lower T) or D^{-1} times the strictly upper part
    int32_t nij = 0;
    if (!UPPER && i > j) nij = t;
    if (UPPER && j > i) nij = mul_bal(t, sD[i], M);
    sP[i][j] = nij;
    sS[i][j] = (i == j ? 1 : 0) - nij;  // I - N, entries within the balanced range
    __syncthreads();
    auto prod = [&](int32_t (*A)[kNBMax + 1], int32_t (*B)[kNBMax + 1]) {
        DotAcc<WIDE> acc;
#pragma unroll
        for (int k = 0; k < kNBMax; ++k) acc.add(A[i][k], B[k][j]);
        return acc.get(M);
    };
    for (int lev = 1; lev < 5; ++lev) {
        const int32_t p2 = prod(sP, sP);  // N^(2^lev)
        __syncthreads();
        sP[i][j] = p2;
        __syncthreads();
        const int32_t q = prod(sS, sP);   // S N^(2^lev)
        __syncthreads();
        sS[i][j] = red_bal((int64_t)sS[i][j] + q, M);
        __syncthreads();
    }
    int32_t v = sS[i][j];
    if (UPPER) v = mul_bal(v, sD[j], M);
    Inv[(int64_t)w * kNBMax * kNBMax + i * kNBMax + j] = (i < jb && j < jb) ? v : 0;
    (void)sQ;
}

// X[xr0 .. xr0+jb)[c0 .. c0+ncols) <- Inv X, per prime (blockIdx.y): one
// 32 x 32 tile of X per CTA (kTaThreads = 256). Lane r of every warp keeps
// row r of Inv in registers (split at bit 16 for 31-bit primes); the tile
// sits in shared memory (rows of 36 words: 16-byte aligned, a warp's row
// access spanning all banks) and is read as broadcasts, four columns per
// access. Warp q forms the tile's columns 4q .. 4q + 3 for all rows and
// writes them back over its own columns; the tile then goes out row by row.
constexpr int kTaThreads = 256;

template <bool WIDE>
__global__ void __launch_bounds__(kTaThreads)
k_tri_apply(const int32_t *__restrict__ Inv, int32_t *__restrict__ X, int64_t strideX, int64_t n,
            int64_t xr0, int jb, int64_t c0, int64_t ncols, const ModP *__restrict__ mods,
            const LUState *__restrict__ st) {
    constexpr int kTS = 36, kWarps = kTaThreads / 32;
    __shared__ __align__(16) int32_t sY[kNBMax * kTS];
    __shared__ int32_t sI[kNBMax * (kNBMax + 1)];
    const int w = blockIdx.y;
    if (st && st[w].dead) return;
    const ModP M = mods[w];
    const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
    const int64_t cb0 = c0 + (int64_t)blockIdx.x * 32;
    const int nc = (int)min((int64_t)32, c0 + ncols - cb0);  // columns in this tile
    int32_t *x = X + (int64_t)w * strideX;
    const int32_t *I = Inv + (int64_t)w * kNBMax * kNBMax;
    for (int r = q; r < kNBMax; r += kWarps) {
        sY[r * kTS + lane] = (r < jb && lane < nc) ? x[(xr0 + r) * n + cb0 + lane] : 0;
        sI[r * (kNBMax + 1) + lane] = I[r * kNBMax + lane];  // zero past jb
    }
    __syncthreads();
    // row `lane` of Inv
    int32_t t[kNBMax], th[WIDE ? kNBMax : 1];
#pragma unroll
    for (int k = 0; k < kNBMax; ++k) t[k] = sI[lane * (kNBMax + 1) + k];
    if (WIDE) {
#pragma unroll
        for (int k = 0; k < kNBMax; ++k) {
            th[k] = t[k] >> 16;
            t[k] &= 0xffff;
        }
    }
    static_assert(kWarps * 4 == kNBMax, "one group of four columns per warp");
    {
        const int cb = 4 * q;
        int64_t lo[4] = {0, 0, 0, 0}, hi[4] = {0, 0, 0, 0};
#pragma unroll
        for (int k = 0; k < kNBMax; ++k) {
            const int4 y = *reinterpret_cast<const int4 *>(sY + k * kTS + cb);
            lo[0] += (int64_t)t[k] * y.x;
            lo[1] += (int64_t)t[k] * y.y;
            lo[2] += (int64_t)t[k] * y.z;
            lo[3] += (int64_t)t[k] * y.w;
            if (WIDE) {
                hi[0] += (int64_t)th[WIDE ? k : 0] * y.x;
                hi[1] += (int64_t)th[WIDE ? k : 0] * y.y;
                hi[2] += (int64_t)th[WIDE ? k : 0] * y.z;
                hi[3] += (int64_t)th[WIDE ? k : 0] * y.w;
            }
        }
        int32_t v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
            v[i] = WIDE ? red_bal((int64_t)red_bal(hi[i], M) * 65536 + red_bal(lo[i], M), M)
                        : red_bal(lo[i], M);
        __syncwarp();  // every lane has read these columns
#pragma unroll
        for (int i = 0; i < 4; ++i) sY[lane * kTS + cb + i] = v[i];
    }
    __syncthreads();
    for (int r = q; r < jb; r += kWarps)
        if (lane < nc) x[(xr0 + r) * n + cb0 + lane] = sY[r * kTS + lane];
}

// One block row of 4 x 32 rows (rows J0 .. J0 + JB) of Y <- T^{-1} Y for
// the columns [c0, c0 + ncols), one tile of 32 columns per CTA and one
// prime per blockIdx.y, in one launch: the block's rows of the tile stay in
// shared memory while, for each 32-row sub-block s in solve order (lower T:
// top down; upper T: bottom up), X_s <- T_ss^{-1} X_s (the inverse of
// sub-block s of prime w at Inv + s inv_sub + w inv_prime, 32 x 32 as
// k_tri_inv and the panel write them) and then X_d <- X_d - T_ds X_s for the
// sub-blocks d still to come (T_ds read from the factor, ld n). All ten
// 32 x 32 factor blocks are copied in at once (dynamic shared memory, slot
// d(d+1)/2 + s of the lower triangle, s(s+1)/2 + d of the upper); every
// step keeps row r of its block in lane r's registers (split at bit 16 for
// 31-bit primes) and has warp q form the tile's columns 4q .. 4q + 3 with
// two accumulator chains per column.
constexpr int kTbSlot = kNBMax * (kNBMax + 1);  // words per factor block
constexpr size_t kTbSmem = sizeof(int32_t) * 10 * kTbSlot;

template <bool WIDE, bool UPPER>
__global__ void __launch_bounds__(kTaThreads)
k_trsm_block(const int32_t *__restrict__ T0, int64_t strideT, const int32_t *__restrict__ Inv,
             int64_t inv_sub, int64_t inv_prime, int32_t *__restrict__ Y0, int64_t strideY,
             int64_t n, int64_t J0, int JB, int64_t c0, int64_t ncols,
             const ModP *__restrict__ mods, const LUState *__restrict__ st) {
    constexpr int kTS = 36, kWarps = kTaThreads / 32, kRows = 4 * kNBMax;
    static_assert(kWarps * 4 == kNBMax, "one group of four columns per warp");
    __shared__ __align__(16) int32_t sY[kRows * kTS];
    extern __shared__ int32_t sF[];  // 10 slots of kTbSlot words
    const int w = blockIdx.y;
    if (st && st[w].dead) return;
    const ModP M = mods[w];
    const int32_t *T = T0 + (int64_t)w * strideT;
    int32_t *Y = Y0 + (int64_t)w * strideY;
    const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
    const int64_t cb0 = c0 + (int64_t)blockIdx.x * 32;
    const int nc = (int)min((int64_t)32, c0 + ncols - cb0);  // columns in this tile
    const int nsub = (JB + kNBMax - 1) / kNBMax;
    auto slot = [](int d, int s_) { return UPPER ? s_ * (s_ + 1) / 2 + d : d * (d + 1) / 2 + s_; };
    // the tile and the factor blocks, all copies in flight at once
    for (int r = q; r < kRows; r += kWarps) {
        if (r < JB && lane < nc)
            __pipeline_memcpy_async(&sY[r * kTS + lane], &Y[(J0 + r) * n + cb0 + lane], 4);
        else
            sY[r * kTS + lane] = 0;
    }
    for (int s_ = 0; s_ < nsub; ++s_) {
        const int rs = min(kNBMax, JB - kNBMax * s_);
        for (int d = UPPER ? 0 : s_; d <= (UPPER ? s_ : nsub - 1); ++d) {
            int32_t *dst = sF + slot(d, s_) * kTbSlot;
            const int32_t *src = d == s_ ? Inv + inv_sub * s_ + inv_prime * w
                                         : T + (J0 + kNBMax * d) * n + J0 + kNBMax * s_;
            const int64_t ld = d == s_ ? kNBMax : n;
            const int fr = d == s_ ? kNBMax : min(kNBMax, JB - kNBMax * d);
            const int fc = d == s_ ? kNBMax : rs;
            for (int r = q; r < kNBMax; r += kWarps) {
                if (r < fr && lane < fc)
                    __pipeline_memcpy_async(&dst[r * (kNBMax + 1) + lane], &src[r * ld + lane], 4);
                else
                    dst[r * (kNBMax + 1) + lane] = 0;
            }
        }
    }
    __pipeline_commit();
    __pipeline_wait_prior(0);
    __syncthreads();
    // rows of sub-block d <- F X_s (d == s) or X_d - F X_s, F in slot (d, s)
    auto step = [&](int s_, int d) {
        const int32_t *F = sF + slot(d, s_) * kTbSlot + lane * (kNBMax + 1);
        int32_t t[kNBMax], th[WIDE ? kNBMax : 1];
#pragma unroll
        for (int k = 0; k < kNBMax; ++k) t[k] = F[k];
        if (WIDE) {
#pragma unroll
            for (int k = 0; k < kNBMax; ++k) {
                th[k] = t[k] >> 16;
                t[k] &= 0xffff;
            }
        }
        const int cb = 4 * q;
        int64_t lo[2][4] = {}, hi[2][4] = {};
#pragma unroll
        for (int k = 0; k < kNBMax; ++k) {
            const int4 y = *reinterpret_cast<const int4 *>(sY + (kNBMax * s_ + k) * kTS + cb);
            const int h = k & 1;
            lo[h][0] += (int64_t)t[k] * y.x;
            lo[h][1] += (int64_t)t[k] * y.y;
            lo[h][2] += (int64_t)t[k] * y.z;
            lo[h][3] += (int64_t)t[k] * y.w;
            if (WIDE) {
                hi[h][0] += (int64_t)th[WIDE ? k : 0] * y.x;
                hi[h][1] += (int64_t)th[WIDE ? k : 0] * y.y;
                hi[h][2] += (int64_t)th[WIDE ? k : 0] * y.z;
                hi[h][3] += (int64_t)th[WIDE ? k : 0] * y.w;
            }
        }
        int32_t v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t l = lo[0][i] + lo[1][i];
            v[i] = WIDE ? red_bal((int64_t)red_bal(hi[0][i] + hi[1][i], M) * 65536 + red_bal(l, M), M)
                        : red_bal(l, M);
        }
        __syncwarp();  // (d == s) every lane has read these columns of the rows
        int32_t *o = sY + (kNBMax * d + lane) * kTS + cb;
#pragma unroll
        for (int i = 0; i < 4; ++i) o[i] = d == s_ ? v[i] : red_bal((int64_t)o[i] - v[i], M);
    };
    for (int i = 0; i < nsub; ++i) {
        const int s_ = UPPER ? nsub - 1 - i : i;
        step(s_, s_);
        __syncthreads();  // X_s is final
        for (int d = UPPER ? 0 : s_ + 1; d < (UPPER ? s_ : nsub); ++d) step(s_, d);
        __syncthreads();
    }
    for (int r = q; r < JB; r += kWarps)
        if (lane < nc) Y[(J0 + r) * n + cb0 + lane] = sY[r * kTS + lane];
}

// C <- C - A B mod p (batched over primes by blockIdx.z). A: M x K (lda),
// B: K x N (ldb), C: M x N (ldc). 64 x 64 tile, 256 threads, 4 x 4 outputs
// per thread, int64 accumulators.
constexpr int BM = 64, BN = 64, BK = 32;

template <bool WIDE>
__global__ void __launch_bounds__(256)
k_gemm_sub(const int32_t *__restrict__ A, int64_t lda, int64_t strideA,
           const int32_t *__restrict__ B, int64_t ldb, int64_t strideB,
           int32_t *__restrict__ C, int64_t ldc, int64_t strideC, int M, int N,
           int K, const ModP *__restrict__ mods, const LUState *__restrict__ st) {
    __shared__ int32_t As[BK][BM + 1];
    __shared__ int32_t Bs[BK][BN];
    const int w = blockIdx.z;
    if (st && st[w].dead) return;
    const ModP Mo = mods[w];
    const int32_t *a = A + (int64_t)w * strideA;
    const int32_t *b = B + (int64_t)w * strideB;
    int32_t *c = C + (int64_t)w * strideC;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    // 21-bit primes: one exact int64 sum per output (|products| < 2^40).
    // 31-bit primes: A split as a = 2^16 a_hi + a_lo (a_lo in [0, 2^16),
    // |a_hi| < 2^14), two exact sums, |a_hi b| < 2^44 and a_lo b < 2^46,
    // so K <= 128 terms stay below 2^53; reduced once at the end.
    int64_t acc[4][4], acch[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = acch[i][j] = 0;
    for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            int r = tid / 32 + 8 * t, cc = tid % 32;
            int gm = m0 + r, gk = k0 + cc;
            As[cc][r] = (gm < M && gk < K) ? a[(int64_t)gm * lda + gk] : 0;
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            int r = tid / 64 + 4 * t, cc = tid % 64;
            int gk = k0 + r, gn = n0 + cc;
            Bs[r][cc] = (gk < K && gn < N) ? b[(int64_t)gk * ldb + gn] : 0;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < BK; ++k) {
            int32_t av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[k][tx + 16 * j];
            if (WIDE) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int32_t lo = av[i] & 0xffff, hi = av[i] >> 16;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        acc[i][j] += (int64_t)lo * bv[j];
                        acch[i][j] += (int64_t)hi * bv[j];
                    }
                }
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] += (int64_t)av[i] * bv[j];
            }
        }
        __syncthreads();
    }
    if (WIDE) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                acc[i][j] = (int64_t)red_bal(acch[i][j], Mo) * 65536 + red_bal(acc[i][j], Mo);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int gn = n0 + tx + 16 * j;
            if (gn >= N) continue;
            int32_t *p = c + (int64_t)gm * ldc + gn;
            *p = red_bal((int64_t)*p - red_bal(acc[i][j], Mo), Mo);
        }
    }
}

__global__ void k_finalize_det(const LUState *st, const ModP *mods, int W, uint32_t *det_out) {
    int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    LUState s = st[w];
    uint32_t p = mods[w].p;
    uint32_t d = s.dead ? 0u : s.det;
    if (s.neg && d) d = p - d;
    det_out[w] = d;
}

// Y = P (row i has its 1 in column perm[i]), or the identity when perm is null.
__global__ void k_perm_identity(int32_t *Y, const int32_t *perm, int64_t n) {
    const int64_t total = n * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e / n, j = e - i * n;
        Y[e] = ((perm ? perm[i] : i) == j) ? 1 : 0;
    }
}

// out = W P for the permutation of the LU (P has its 1 of row k in column
// perm[k]): column k of W goes to column perm[k]; columns n .. ld - 1 of out
// are zero.
__global__ void k_cols_by_perm(const int32_t *__restrict__ W, const int32_t *__restrict__ perm,
                               int64_t n, int32_t *__restrict__ out, int64_t ld) {
    const int64_t total = n * ld;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / ld, k = e - i * ld;
        if (k < n)
            out[i * ld + perm[k]] = W[i * n + k];
        else
            out[e] = 0;
    }
}

template <bool WIDE>
int gemm_sub(const int32_t *A, int64_t lda, int64_t sA, const int32_t *B, int64_t ldb,
             int64_t sB, int32_t *C, int64_t ldc, int64_t sC, int M, int N, int K,
             const ModP *mods, const LUState *st, int W, cudaStream_t s) {
    if (M <= 0 || N <= 0 || K <= 0) return IDET_OK;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, W);
    k_gemm_sub<WIDE><<<grid, 256, 0, s>>>(A, lda, sA, B, ldb, sB, C, ldc, sC, M, N,
                                           K, mods, st);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

template <bool WIDE>
int trsm_lower(const int32_t *Lm, int64_t sL, int32_t *X, int64_t sX, int64_t n,
               int64_t lr0, int64_t xr0, int jb, int64_t c0, int64_t ncols,
               const ModP *mods, const LUState *st, int W, cudaStream_t s,
               int32_t *tri = nullptr, bool have_inv = false) {
    if (ncols <= 0) return IDET_OK;
    if (tri) {
        // explicit inverse of the diagonal block (unless tri holds it from
        // an earlier solve with the same block), then a dense apply
        if (!have_inv) {
            k_tri_inv<WIDE, false><<<W, kNBMax * kNBMax, 0, s>>>(Lm, sL, n, lr0, jb, mods, st, tri);
            count_launch();
        }
        k_tri_apply<WIDE><<<dim3((unsigned)((ncols + 31) / 32), W), kTaThreads, 0, s>>>(
            tri, X, sX, n, xr0, jb, c0, ncols, mods, st);
        count_launch();
        IDET_CUDA_TRY(cudaGetLastError());
        return IDET_OK;
    }
    // narrow blocks: a TRSM row block has few columns per prime
    dim3 grid((unsigned)((ncols + 31) / 32), W);
    k_trsm_lower<WIDE><<<grid, 32, 0, s>>>(Lm, sL, X, sX, n, lr0, xr0, jb, c0, ncols,
                                             mods, st);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

// Cluster size of the panel: 16 CTAs per prime (the non-portable size)
// when the primes' clusters still fit on the SMs and the device schedules
// them, else 8. With few primes (the lifting prime's LU is one) most SMs
// would otherwise idle through the panels, and a column's work per CTA halves.
static int panel_cluster_size(int W) {
    static int ok16 = -1;  // 16-CTA clusters of this kernel can be scheduled
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return kCl;
    if (W * 16 > sms - t_reserve_sms) return kCl;
    if (ok16 < 0) {
        ok16 = 0;
        if (allow_max_smem((const void *)k_panel_cluster<16>) == IDET_OK &&
            cudaFuncSetAttribute((const void *)k_panel_cluster<16>,
                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at;
            at.id = cudaLaunchAttributeClusterDimension;
            at.val.clusterDim.x = 16;
            at.val.clusterDim.y = 1;
            at.val.clusterDim.z = 1;
            cfg.gridDim = dim3(16);
            cfg.blockDim = dim3(kClThreads);
            cfg.dynamicSmemBytes = 64 * 1024;
            cfg.attrs = &at;
            cfg.numAttrs = 1;
            int nc = 0;
            if (cudaOccupancyMaxActiveClusters(&nc, (const void *)k_panel_cluster<16>, &cfg) ==
                    cudaSuccess &&
                nc >= 1)
                ok16 = 1;
        }
        cudaGetLastError();
    }
    return ok16 ? 16 : kCl;
}

static int launch_panel_cluster(int CL, int W, size_t psmem, cudaStream_t s, int32_t *R, int64_t n,
                                int64_t j0, int jb, int chunk, const ModP *mods, LUState *st,
                                int32_t *perm, int32_t *tri) {
    const void *kern =
        CL == 16 ? (const void *)k_panel_cluster<16> : (const void *)k_panel_cluster<kCl>;
    IDET_TRY(allow_max_smem(kern));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = CL;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(W * CL));
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = psmem;
    cfg.stream = s;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    if (CL == 16)
        IDET_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_panel_cluster<16>, R, n, j0, jb, chunk, mods, st,
                                         perm, tri));
    else
        IDET_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_panel_cluster<kCl>, R, n, j0, jb, chunk, mods, st,
                                         perm, tri));
    return IDET_OK;
}

// Two-level right-looking LU: block columns of NB = 128 (the trailing
// update's K, so that the Schur complement is read and written once per 128
// columns), each factored by 32-wide cluster panels with updates confined to
// the block column; then U12 = L11^{-1} A12 by 32-row blocks and the rank-128
// update A22 <- A22 - L21 U12.
template <bool WIDE>
int lu_blocked(int32_t *R, int64_t n, const ModP *mods, int W, int nb, int32_t *perm,
               LUState *st, cudaStream_t s, int path, void *scratch = nullptr,
               int32_t *tri = nullptr) {
    k_state_init<<<W, 256, 0, s>>>(st, mods, W, perm, n);
    count_launch();
    const int64_t nn = n * n;
    const int NB = 4 * nb;
    auto upd = [&](int64_t r, int64_t c, int64_t kr, int M, int N, int K) -> int {
        // C = R[r.., c..] -= R[r.., kr..kr+K) * R[kr..kr+K, c..]
        if (M <= 0 || N <= 0 || K <= 0) return IDET_OK;
        const int32_t *Ap = R + r * n + kr;
        const int32_t *Bp = R + kr * n + c;
        int32_t *Cp = R + r * n + c;
        if (path == IDET_PATH_TC05)
            return gemm_sub_tc05(Ap, n, nn, Bp, n, nn, Cp, n, nn, M, N, K, mods, st, W, scratch, s,
                                 WIDE ? 5 : 3);
        if (!WIDE && path != IDET_PATH_INT64)
            return gemm_sub_tc(path, Ap, n, nn, Bp, n, nn, Cp, n, nn, M, N, K, mods, st, W,
                               scratch, s);
        return gemm_sub<WIDE>(Ap, n, nn, Bp, n, nn, Cp, n, nn, M, N, K, mods, st, W, s);
    };
    for (int64_t J0 = 0; J0 < n; J0 += NB) {
        const int JB = (int)((n - J0) < NB ? (n - J0) : NB);
        for (int64_t j0 = J0; j0 < J0 + JB; j0 += nb) {
            const int jb = (int)((J0 + JB - j0) < nb ? (J0 + JB - j0) : nb);
            // the inverse of this panel's L11 goes to slot (j0 - J0) / nb of
            // tri, for the solve inside the block column and again for the
            // block row below; the cluster panel forms it from its replica
            int32_t *tri_p = tri ? tri + (size_t)((j0 - J0) / nb) * W * kNBMax * kNBMax : nullptr;
            const int CL = panel_cluster_size(W);
            // rows per CTA: the last CTA, which also forms L11^{-1}, takes at
            // most 128 (its rows then fit on half its warps, two threads a
            // row) when the others stay within 256 (two threads a row too)
            const int64_t rows = n - j0;
            int chunk = (int)((rows + CL - 1) / CL);
            if (rows > 128) {
                const int chunk_t = (int)((rows - 128 + CL - 2) / (CL - 1));
                if (chunk_t <= kClThreads / 2 && chunk_t >= chunk) chunk = chunk_t;
            }
            const size_t psmem = sizeof(int32_t) * (size_t)chunk * kSP;
            // The cluster panel also forms L11^{-1} from its replica (in its
            // last CTA, beside the other CTAs' rows); k_panel leaves it to a
            // separate launch.
            const bool cluster_panel = psmem <= 200 * 1024;
            if (psmem <= 200 * 1024) {
                IDET_TRY(launch_panel_cluster(CL, W, psmem, s, R, n, j0, jb, chunk, mods, st,
                                              perm, cluster_panel ? tri_p : nullptr));
            } else {
                k_panel<<<W, kPanelThreads, 0, s>>>(R, n, j0, jb, mods, st, perm);
            }
            count_launch();
            IDET_CUDA_TRY(cudaGetLastError());
            const int64_t inner = J0 + JB - (j0 + jb);  // columns left in the block column
            if (inner > 0) {
                IDET_TRY(trsm_lower<WIDE>(R, nn, R, nn, n, j0, j0, jb, j0 + jb, inner, mods, st,
                                          W, s, tri_p, tri_p && cluster_panel));
                IDET_TRY(upd(j0 + jb, j0 + jb, j0, (int)(n - j0 - jb), (int)inner, jb));
            } else if (tri_p && !cluster_panel && n - J0 - JB > 0) {
                k_tri_inv<WIDE, false><<<W, kNBMax * kNBMax, 0, s>>>(R, nn, n, j0, jb, mods, st,
                                                                      tri_p);
                count_launch();
                IDET_CUDA_TRY(cudaGetLastError());
            }
        }
        const int64_t rest = n - J0 - JB;
        if (rest <= 0) break;
        if (tri && nb == kNBMax) {
            // U12 = L11^{-1} A12 for the block row: the four sub-block solves
            // and the updates among them in one launch
            const int64_t tw = (int64_t)kNBMax * kNBMax;
            IDET_TRY(allow_max_smem((const void *)k_trsm_block<WIDE, false>));
            k_trsm_block<WIDE, false><<<dim3((unsigned)((rest + 31) / 32), W), kTaThreads, kTbSmem, s>>>(
                R, nn, tri, tw * W, tw, R, nn, n, J0, JB, J0 + JB, rest, mods, st);
            count_launch();
            IDET_CUDA_TRY(cudaGetLastError());
        } else {
            for (int64_t i0 = J0; i0 < J0 + JB; i0 += nb) {
                const int ib = (int)((J0 + JB - i0) < nb ? (J0 + JB - i0) : nb);
                int32_t *tri_p =
                    tri ? tri + (size_t)((i0 - J0) / nb) * W * kNBMax * kNBMax : nullptr;
                IDET_TRY(trsm_lower<WIDE>(R, nn, R, nn, n, i0, i0, ib, J0 + JB, rest, mods, st,
                                          W, s, tri_p, tri_p != nullptr));
                const int64_t below = J0 + JB - (i0 + ib);
                if (below > 0) IDET_TRY(upd(i0 + ib, J0 + JB, i0, (int)below, (int)rest, ib));
            }
        }
        IDET_TRY(upd(J0 + JB, J0 + JB, J0, (int)rest, (int)rest, JB));
    }
    return IDET_OK;
}

}  // namespace

int lu_factor_batched(int32_t *R, int64_t n, const ModP *mods_dev,
                      const ModP *mods_host, int W, bool wide, int nb,
                      int32_t *perm, uint32_t *det_out, int update_path,
                      Workspace &ws) {
    (void)mods_host;
    cudaStream_t s = ws.stream();
    if (W <= 0) return IDET_OK;
    LUState *st = nullptr;
    IDET_TRY(ws.alloc_n(&st, W));
    idet_tuned tuned{};
    const bool have_tuned = tuned_lookup(n, wide ? 31 : 21, &tuned);
    if (nb <= 0 && have_tuned) nb = tuned.nb;
    if (nb <= 0 || nb > kNBMax) nb = kNBMax;
    if (n <= kSmallN) {
        size_t smem = sizeof(int32_t) * n * n;
        IDET_TRY(allow_max_smem((const void *)k_lu_small));
        k_lu_small<<<W, 512, smem, s>>>(R, (int)n, mods_dev, st, perm);
        count_launch();
        IDET_CUDA_TRY(cudaGetLastError());
    } else if (wide) {
        // 31-bit primes: the tcgen05 update with five limbs, or int64
        const int path = update_path == IDET_PATH_INT64 ||
                                 (update_path == IDET_PATH_AUTO && have_tuned &&
                                  tuned.update_path == IDET_PATH_INT64)
                             ? IDET_PATH_INT64
                             : IDET_PATH_TC05;
        int32_t *tri = nullptr;
        void *scratch = nullptr;
        IDET_TRY(ws.alloc_n(&tri, (size_t)4 * W * kNBMax * kNBMax));  // 4 panels per block column
        if (path == IDET_PATH_TC05) IDET_TRY(ws.alloc(&scratch, tc05_scratch_bytes(n, W, 5)));
        IDET_TRY(lu_blocked<true>(R, n, mods_dev, W, nb, perm, st, s, path, scratch, tri));
        if (path == IDET_PATH_TC05) IDET_TRY(tc05_check_error(s));
    } else {
        // default trailing-update arithmetic for 21-bit primes: the tcgen05
        // bf16-limb path (measured fastest at n = 1000 and 4000)
        const int path = update_path != IDET_PATH_AUTO
                             ? update_path
                             : (have_tuned && tuned.update_path != IDET_PATH_AUTO ? tuned.update_path
                                                                                  : IDET_PATH_TC05);
        void *scratch = nullptr;
        if (path == IDET_PATH_TC05) IDET_TRY(ws.alloc(&scratch, tc05_scratch_bytes(n, W, 3)));
        const bool legacy_tc =
            path == IDET_PATH_I8 || path == IDET_PATH_BF16 || path == IDET_PATH_F64;
        if (legacy_tc) IDET_TRY(ws.alloc(&scratch, tc_scratch_bytes(n, W, path)));
        int32_t *tri = nullptr;
        IDET_TRY(ws.alloc_n(&tri, (size_t)4 * W * kNBMax * kNBMax));  // 4 panels per block column
        IDET_TRY(lu_blocked<false>(R, n, mods_dev, W, nb, perm, st, s, path, scratch, tri));
        if (path == IDET_PATH_TC05) IDET_TRY(tc05_check_error(s));
        if (legacy_tc) IDET_TRY(tc_check_error(s));
    }
    k_finalize_det<<<(W + 127) / 128, 128, 0, s>>>(st, mods_dev, W, det_out);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

// A^{-1} = U^{-1} L^{-1} P: Y <- P, Y <- L^{-1} Y (blocked forward
// substitution), Y <- U^{-1} Y (blocked back substitution).
int lu_inverse(const int32_t *R, const int32_t *perm, int64_t n, const ModP &mod_host,
               const ModP *mod_dev, bool wide, int nb, int32_t *Y, int32_t *out, int64_t ld_out,
               Workspace &ws) {
    cudaStream_t s = ws.stream();
    idet_tuned tuned{};
    const bool have_tuned = tuned_lookup(n, wide ? 31 : 21, &tuned);
    if (nb <= 0 && have_tuned) nb = tuned.nb;
    if (nb <= 0 || nb > kNBMax) nb = kNBMax;
    // A^{-1} = U^{-1} L^{-1} P: Y <- I, Y <- L^{-1} Y (lower triangular: a
    // block row of it has no nonzero right of its diagonal block, so every
    // solve and update of the forward pass stops at that column), Y <- U^{-1} Y
    // (full), then out = Y P.
    k_perm_identity<<<148 * 4, 256, 0, s>>>(Y, nullptr, n);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    // Y <- L^{-1} Y and Y <- U^{-1} Y, two-level: blocks of NB = 4 nb rows;
    // inside a block, nb-row triangular solves with rank-nb updates of the
    // block's remaining rows; then one rank-NB update of all rows outside it
    const int NB = 4 * nb;
    // The diagonal nb x nb blocks of L and U do not change during the
    // solves: invert all of them up front, the full blocks in one launch per
    // factor (block b of the factor is batch entry b, stride nb (n + 1)),
    // a ragged last block in one more.
    const int64_t nbk = (n + nb - 1) / nb, nfull = n / nb;
    const size_t tsz = (size_t)kNBMax * kNBMax;
    int32_t *triL = nullptr, *triU = nullptr;
    ModP *mrep = nullptr;
    IDET_TRY(ws.alloc_n(&triL, tsz * nbk));
    IDET_TRY(ws.alloc_n(&triU, tsz * nbk));
    IDET_TRY(ws.alloc_n(&mrep, nbk));
    {
        std::vector<ModP> mh((size_t)nbk, mod_host);
        IDET_CUDA_TRY(cudaMemcpyAsync(mrep, mh.data(), sizeof(ModP) * nbk, cudaMemcpyHostToDevice, s));
        const int64_t strideD = (int64_t)nb * (n + 1);
        const int last = (int)(n - nfull * nb);
        if (wide) {
            if (nfull) {
                k_tri_inv<true, false><<<(unsigned)nfull, kNBMax * kNBMax, 0, s>>>(R, strideD, n, 0, nb, mrep, nullptr, triL);
                k_tri_inv<true, true><<<(unsigned)nfull, kNBMax * kNBMax, 0, s>>>(R, strideD, n, 0, nb, mrep, nullptr, triU);
            }
            if (last) {
                k_tri_inv<true, false><<<1, kNBMax * kNBMax, 0, s>>>(R, 0, n, nfull * nb, last, mrep, nullptr, triL + tsz * nfull);
                k_tri_inv<true, true><<<1, kNBMax * kNBMax, 0, s>>>(R, 0, n, nfull * nb, last, mrep, nullptr, triU + tsz * nfull);
            }
        } else {
            if (nfull) {
                k_tri_inv<false, false><<<(unsigned)nfull, kNBMax * kNBMax, 0, s>>>(R, strideD, n, 0, nb, mrep, nullptr, triL);
                k_tri_inv<false, true><<<(unsigned)nfull, kNBMax * kNBMax, 0, s>>>(R, strideD, n, 0, nb, mrep, nullptr, triU);
            }
            if (last) {
                k_tri_inv<false, false><<<1, kNBMax * kNBMax, 0, s>>>(R, 0, n, nfull * nb, last, mrep, nullptr, triL + tsz * nfull);
                k_tri_inv<false, true><<<1, kNBMax * kNBMax, 0, s>>>(R, 0, n, nfull * nb, last, mrep, nullptr, triU + tsz * nfull);
            }
        }
        count_launch((nfull ? 2 : 0) + (last ? 2 : 0));
        IDET_CUDA_TRY(cudaGetLastError());
    }
    auto apply = [&](const int32_t *tri_blk, int64_t k0, int kb, int64_t ncols) -> int {
        const dim3 grid((unsigned)((ncols + 31) / 32), 1);
        if (wide)
            k_tri_apply<true><<<grid, kTaThreads, 0, s>>>(tri_blk, Y, 0, n, k0, kb, 0, ncols, mod_dev,
                                                   nullptr);
        else
            k_tri_apply<false><<<grid, kTaThreads, 0, s>>>(tri_blk, Y, 0, n, k0, kb, 0, ncols, mod_dev,
                                                    nullptr);
        count_launch();
        IDET_CUDA_TRY(cudaGetLastError());
        return IDET_OK;
    };
    // the updates on tcgen05 unless the table chose int64 for this size
    const bool tc = !(have_tuned && tuned.update_path == IDET_PATH_INT64);
    void *scratch = nullptr;
    if (tc) IDET_TRY(ws.alloc(&scratch, tc05_scratch_bytes(n, 1, wide ? 5 : 3)));
    LUState *st1 = nullptr;
    if (tc) {
        IDET_TRY(ws.alloc_n(&st1, 1));
        IDET_CUDA_TRY(cudaMemsetAsync(st1, 0, sizeof(LUState), s));
    }
    auto gsub = [&](const int32_t *Ap, const int32_t *Bp, int32_t *Cp, int64_t M, int K,
                    int64_t N) -> int {
        if (M <= 0 || K <= 0 || N <= 0) return IDET_OK;
        if (tc)
            return gemm_sub_tc05(Ap, n, 0, Bp, n, 0, Cp, n, 0, (int)M, (int)N, K, mod_dev, st1, 1,
                                 scratch, s, wide ? 5 : 3);
        if (wide)
            return gemm_sub<true>(Ap, n, 0, Bp, n, 0, Cp, n, 0, (int)M, (int)N, K, mod_dev, nullptr,
                                  1, s);
        return gemm_sub<false>(Ap, n, 0, Bp, n, 0, Cp, n, 0, (int)M, (int)N, K, mod_dev, nullptr, 1,
                               s);
    };
    // with nb = 32 a block row's four sub-block solves and the updates among
    // them run in one launch (k_trsm_block)
    const bool fused = nb == kNBMax;
    auto block_solve = [&](bool upper, int64_t J0, int JB, int64_t ncols) -> int {
        const dim3 grid((unsigned)((ncols + 31) / 32));
        IDET_TRY(allow_max_smem(wide ? (upper ? (const void *)k_trsm_block<true, true>
                                              : (const void *)k_trsm_block<true, false>)
                                     : (upper ? (const void *)k_trsm_block<false, true>
                                              : (const void *)k_trsm_block<false, false>)));
        const int32_t *inv = (upper ? triU : triL) + tsz * (J0 / nb);
        const int64_t is = (int64_t)tsz;
        if (wide) {
            if (upper)
                k_trsm_block<true, true><<<grid, kTaThreads, kTbSmem, s>>>(
                    R, 0, inv, is, 0, Y, 0, n, J0, JB, 0, ncols, mod_dev, nullptr);
            else
                k_trsm_block<true, false><<<grid, kTaThreads, kTbSmem, s>>>(
                    R, 0, inv, is, 0, Y, 0, n, J0, JB, 0, ncols, mod_dev, nullptr);
        } else {
            if (upper)
                k_trsm_block<false, true><<<grid, kTaThreads, kTbSmem, s>>>(
                    R, 0, inv, is, 0, Y, 0, n, J0, JB, 0, ncols, mod_dev, nullptr);
            else
                k_trsm_block<false, false><<<grid, kTaThreads, kTbSmem, s>>>(
                    R, 0, inv, is, 0, Y, 0, n, J0, JB, 0, ncols, mod_dev, nullptr);
        }
        count_launch();
        IDET_CUDA_TRY(cudaGetLastError());
        return IDET_OK;
    };
    for (int64_t J0 = 0; J0 < n; J0 += NB) {
        const int JB = (int)((n - J0) < NB ? (n - J0) : NB);
        if (fused) {
            IDET_TRY(block_solve(false, J0, JB, J0 + JB));
        } else {
            for (int64_t k0 = J0; k0 < J0 + JB; k0 += nb) {
                const int kb = (int)((J0 + JB - k0) < nb ? (J0 + JB - k0) : nb);
                IDET_TRY(apply(triL + tsz * (k0 / nb), k0, kb, k0 + kb));
                IDET_TRY(gsub(R + (k0 + kb) * n + k0, Y + k0 * n, Y + (k0 + kb) * n,
                              J0 + JB - (k0 + kb), kb, k0 + kb));
            }
        }
        IDET_TRY(gsub(R + (J0 + JB) * n + J0, Y + J0 * n, Y + (J0 + JB) * n, n - J0 - JB, JB,
                      J0 + JB));
    }
    const int64_t nblk = (n + NB - 1) / NB;
    for (int64_t bj = nblk - 1; bj >= 0; --bj) {
        const int64_t J0 = bj * NB;
        const int JB = (int)((n - J0) < NB ? (n - J0) : NB);
        const int64_t nsub = (JB + nb - 1) / nb;
        if (fused) {
            IDET_TRY(block_solve(true, J0, JB, n));
        } else {
            for (int64_t bi = nsub - 1; bi >= 0; --bi) {
                const int64_t k0 = J0 + bi * nb;
                const int kb = (int)((J0 + JB - k0) < nb ? (J0 + JB - k0) : nb);
                IDET_TRY(apply(triU + tsz * (k0 / nb), k0, kb, n));
                // rows J0 .. k0 of the block: Y_r -= U[r, k0..k0+kb) Y[k0..k0+kb)
                IDET_TRY(gsub(R + J0 * n + k0, Y + k0 * n, Y + J0 * n, k0 - J0, kb, n));
            }
        }
        // rows above the block
        IDET_TRY(gsub(R + J0, Y + J0 * n, Y, J0, JB, n));
    }
    if (tc) IDET_TRY(tc05_check_error(s));
    k_cols_by_perm<<<148 * 4, 256, 0, s>>>(Y, perm, n, out, ld_out);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

}  // namespace idet

namespace idet {

// Whole-matrix LU for n <= 192 into caller-provided buffers (no workspace):
// R holds W residue matrices (n x n), st W states, det_out W residues.
int lu_small_into(int32_t *R, int n, const ModP *mods_dev, int W, LUState *st,
                  uint32_t *det_out, cudaStream_t s) {
    if (n < 1 || n > kSmallN || W < 1) {
        set_last_error("lu_small_into: n must be in [1, %d]", kSmallN);
        return IDET_ERR_ARG;
    }
    const size_t smem = sizeof(int32_t) * (size_t)n * n;
    IDET_TRY(allow_max_smem((const void *)k_lu_small));
    k_lu_small<<<W, 512, smem, s>>>(R, n, mods_dev, st, nullptr);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    k_finalize_det<<<(W + 127) / 128, 128, 0, s>>>(st, mods_dev, W, det_out);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

}  // namespace idet

namespace idet {

int lu_small_multi(const LUSmallJob *jobs_dev, int count, int max_n, cudaStream_t s) {
    if (count <= 0) return IDET_OK;
    if (max_n > kSmallN) {
        set_last_error("lu_small_multi: n must be at most %d", kSmallN);
        return IDET_ERR_ARG;
    }
    IDET_TRY(allow_max_smem((const void *)k_lu_small_multi));
    k_lu_small_multi<<<count, 512, sizeof(int32_t) * (size_t)max_n * max_n, s>>>(jobs_dev);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

}  // namespace idet
