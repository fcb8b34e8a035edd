// Dixon lifting for a batch of independent small systems (Section 2.2), one
// CTA per system: the two matrix-vector products of each lifting step are
// separated by CTA barriers only, so many systems advance at once without a
// grid-wide barrier (the single-system kernel in k_lift.cu spends most of
// its time in grid barriers when n is small).
//
//   r_0 = b;  x_i = C (r_i mod p) mod p (balanced);  r_{i+1} = (r_i - A x_i)/p
//
// C = A^{-1} mod p and A are int32 rows of ld entries (ld a multiple of 4,
// zero padded), read from global memory (L2-resident for the batch sizes
// this serves); r mod p, x and r live in shared memory. Exactness as in
// k_lift.cu: x uses the 16-bit split of r mod p with int64 partial sums,
// r_{i+1} is formed modulo 2^64 and multiplied by p^{-1} mod 2^64.
#include <climits>

#include <cooperative_groups.h>

#include "idet_internal.cuh"

namespace idet {

namespace {

constexpr int kBT = 512;
constexpr int kBW = kBT / 32;
constexpr int kRows = 4;  // rows per warp in flight

__device__ __forceinline__ int64_t wsum(int64_t v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kBT) k_lift_multi(const LiftJob *__restrict__ jobs) {
    extern __shared__ __align__(16) unsigned char smb[];
    __shared__ int64_t s_z[kBW];
    const LiftJob J = jobs[blockIdx.x];
    const int n = J.n, ld = J.ld, nq = ld / 4;
    const ModP M = J.mod;
    int32_t *rm = (int32_t *)smb;            // ld
    int32_t *xs = rm + ld;                   // ld
    int64_t *rs = (int64_t *)(xs + ld);      // n (ld is a multiple of 4: 16-byte aligned)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < ld; i += kBT) {
        if (i < n) {
            const int64_t bi = J.b[i];
            rs[i] = bi;
            rm[i] = red_bal(bi, M);
        } else {
            rm[i] = 0;
        }
        xs[i] = 0;
    }
    __syncthreads();
    const int4 *rm4 = (const int4 *)rm, *x4 = (const int4 *)xs;
    for (int it = 0; it < J.m; ++it) {
        // x = C (r mod p) mod p
        int64_t zp = 0;
        for (int r0 = warp * kRows; r0 < n; r0 += kBW * kRows) {
            int64_t lo[kRows], hi[kRows];
#pragma unroll
            for (int k = 0; k < kRows; ++k) lo[k] = hi[k] = 0;
#pragma unroll 2
            for (int q = lane; q < nq; q += 32) {
                const int4 v = rm4[q];
                const int4 vl = make_int4(v.x & 0xffff, v.y & 0xffff, v.z & 0xffff, v.w & 0xffff);
                const int4 vh = make_int4(v.x >> 16, v.y >> 16, v.z >> 16, v.w >> 16);
#pragma unroll
                for (int k = 0; k < kRows; ++k) {
                    if (r0 + k < n) {
                        const int4 c = __ldg((const int4 *)(J.C + (int64_t)(r0 + k) * ld) + q);
                        lo[k] += (int64_t)c.x * vl.x + (int64_t)c.y * vl.y + (int64_t)c.z * vl.z +
                                 (int64_t)c.w * vl.w;
                        hi[k] += (int64_t)c.x * vh.x + (int64_t)c.y * vh.y + (int64_t)c.z * vh.z +
                                 (int64_t)c.w * vh.w;
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < kRows; ++k) {
                const int64_t l = wsum(lo[k]), h = wsum(hi[k]);
                if (lane == 0 && r0 + k < n) {
                    const int32_t x = red_bal((int64_t)red_bal(h, M) * 65536 + red_bal(l, M), M);
                    xs[r0 + k] = x;
                    if (J.digits) J.digits[(int64_t)it * n + r0 + k] = x;
                    if (J.u) zp += (int64_t)J.u[r0 + k] * x;
                }
            }
        }
        if (lane == 0) s_z[warp] = zp;
        __syncthreads();
        if (tid == 0 && J.z) {
            int64_t t = 0;
            for (int k = 0; k < kBW; ++k) t += s_z[k];
            J.z[it] = t;
        }
        // r <- (r - A x) / p
        for (int r0 = warp * kRows; r0 < n; r0 += kBW * kRows) {
            uint64_t acc[kRows];
#pragma unroll
            for (int k = 0; k < kRows; ++k) acc[k] = 0;
#pragma unroll 2
            for (int q = lane; q < nq; q += 32) {
                const int4 x = x4[q];
#pragma unroll
                for (int k = 0; k < kRows; ++k) {
                    if (r0 + k < n) {
                        const int4 a = __ldg((const int4 *)(J.A + (int64_t)(r0 + k) * ld) + q);
                        acc[k] += (uint64_t)((int64_t)a.x * x.x) + (uint64_t)((int64_t)a.y * x.y) +
                                  (uint64_t)((int64_t)a.z * x.z) + (uint64_t)((int64_t)a.w * x.w);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < kRows; ++k) {
                const uint64_t t = (uint64_t)wsum((int64_t)acc[k]);
                if (lane == 0 && r0 + k < n) {
                    const int row = r0 + k;
                    const int64_t rn = (int64_t)(((uint64_t)rs[row] - t) * J.pinv);
                    rs[row] = rn;
                    rm[row] = red_bal(rn, M);
                }
            }
        }
        __syncthreads();
    }
    for (int i = tid; i < n; i += kBT) J.r[i] = rs[i];
}

}  // namespace

int launch_lift_multi(const LiftJob *jobs_dev, int count, int max_ld, cudaStream_t s) {
    if (count <= 0) return IDET_OK;
    const size_t smem = (size_t)max_ld * (4 + 4 + 8) + 64;
    if (smem > 200 * 1024) {
        set_last_error("batched lift: n too large");
        return IDET_ERR_ARG;
    }
    IDET_TRY(allow_max_smem((const void *)k_lift_multi));
    k_lift_multi<<<count, kBT, smem, s>>>(jobs_dev);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

}  // namespace idet

// ---------------------------------------------------------------------------
// Whole-matrix elimination over Z/p by a cluster of kEC CTAs, one cluster per
// job of a batch (n up to ~640: the matrix lives in the cluster's
// distributed shared memory, kEC contiguous row blocks).
//   mode 0 (LU): det A mod p with the first-nonzero pivot rule (Section 2.1);
//   mode 1 (Gauss-Jordan, in place): A^{-1} mod p, balanced, written to the
//            job's Cinv (ld entries per row, zero padded); row exchanges are
//            logged and undone as column exchanges at the end.
// Per column: the pivot row is found (the owner tests the diagonal, otherwise
// every block reports its first nonzero row and all take the minimum), rows
// are exchanged through DSMEM if needed, every block copies the pivot row and
// updates its own rows.

namespace idet {

namespace {

constexpr int kEC = 8;
constexpr int kECT = 512;

__device__ __forceinline__ int32_t inv32(int32_t a, uint32_t p) {
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

__global__ void __cluster_dims__(kEC, 1, 1) __launch_bounds__(kECT)
k_elim_cluster(const ElimJob *__restrict__ jobs, int mode) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) int32_t es[];
    __shared__ int s_cand[2];
    __shared__ int32_t s_inv;
    const ElimJob J = jobs[blockIdx.x / kEC];
    const int rank = (int)cl.block_rank();
    const int n = J.n, chunk = (n + kEC - 1) / kEC;
    const ModP M = J.mod;
    const int rbeg = rank * chunk, rend = min(n, rbeg + chunk);
    const int nloc = rend > rbeg ? rend - rbeg : 0;
    int32_t *rows = es;                      // chunk x n
    int32_t *prow = es + (size_t)chunk * n;  // n: pivot row copy
    int32_t *swp = prow + n;                 // n: row exchanged with row k (GJ)
    const int tid = threadIdx.x;
    for (int e = tid; e < nloc * n; e += kECT) {
        const int r = e / n, c = e % n;
        const int64_t a = J.A[(int64_t)(rbeg + r) * J.lda + c];
        rows[e] = red_bal(a, M);
        if (J.A32) J.A32[(int64_t)(rbeg + r) * J.ld + c] = (int32_t)a;
    }
    if (J.A32 && J.ld > n)
        for (int e = tid; e < nloc * (J.ld - n); e += kECT) {
            const int r = e / (J.ld - n), c = n + e % (J.ld - n);
            J.A32[(int64_t)(rbeg + r) * J.ld + c] = 0;
        }
    for (int k = tid; k < n; k += kECT) swp[k] = k;
    int32_t *fcol = swp + n;                 // chunk: column k of this block's rows
    uint32_t det = 1u % M.p;
    int neg = 0, dead = 0;
    __syncthreads();
    cl.sync();
    for (int k = 0; k < n; ++k) {
        const int owner = k / chunk;
        // the owner of row k-1 writes it now: every block finished reading it
        if (k > 0 && rank == (k - 1) / chunk) {
            int32_t *row = rows + (size_t)(k - 1 - rbeg) * n;
            for (int c = tid; c < n; c += kECT) row[c] = prow[c];
        }
        int32_t *kr = cl.map_shared_rank(rows, owner) + (size_t)(k - owner * chunk) * n;
        if (tid == 0) s_inv = kr[k];
        __syncthreads();
        if (s_inv == 0) {
            const int par = k & 1;
            if (tid == 0) s_cand[par] = INT_MAX;
            __syncthreads();
            for (int r = tid; r < nloc; r += kECT)
                if (rbeg + r > k && rows[r * n + k] != 0) atomicMin(&s_cand[par], rbeg + r);
            cl.sync();
            int best = INT_MAX;
            for (int q = 0; q < kEC; ++q) best = min(best, *cl.map_shared_rank(&s_cand[par], q));
            if (best == INT_MAX) {
                dead = 1;
                break;
            }
            const int po = best / chunk;
            int32_t *pr = cl.map_shared_rank(rows, po) + (size_t)(best - po * chunk) * n;
            if (rank == 0)
                for (int c = tid; c < n; c += kECT) {
                    const int32_t t = kr[c];
                    kr[c] = pr[c];
                    pr[c] = t;
                }
            if (tid == 0) swp[k] = best;
            neg ^= 1;
            cl.sync();
        }
        for (int c = tid; c < n; c += kECT) prow[c] = kr[c];
        for (int r = tid; r < nloc; r += kECT) fcol[r] = rows[r * n + k];
        __syncthreads();
        const int32_t pv = prow[k];
        if (tid == 0) s_inv = inv32(pv, M.p);
        det = red_pos((int64_t)det * pv, M);
        __syncthreads();
        const int32_t inv = s_inv;
        // pivot row scaled by 1/a_kk, with 1/a_kk in column k (the owner
        // writes it into row k at the start of the next column)
        for (int c = tid; c < n; c += kECT) prow[c] = (c == k) ? inv : mul_bal(prow[c], inv, M);
        __syncthreads();
        // other rows: a_ij -= a_ik prow_j (j != k), a_ik = -a_ik / a_kk
        const int rg = tid >> 7, ct = tid & 127;
        for (int r = rg; r < nloc; r += 4) {
            if (rbeg + r == k) continue;
            const int32_t f = fcol[r];
            int32_t *row = rows + (size_t)r * n;
            if (f)
                for (int c = ct; c < n; c += 128)
                    if (c != k) row[c] = red_bal((int64_t)row[c] - (int64_t)f * prow[c], M);
            if (ct == 0) row[k] = mul_bal(-f, inv, M);
        }
        __syncthreads();
        cl.sync();
    }
    if (!dead && rank == (n - 1) / chunk) {
        int32_t *row = rows + (size_t)(n - 1 - rbeg) * n;
        for (int c = tid; c < n; c += kECT) row[c] = prow[c];
    }
    __syncthreads();
    cl.sync();
    if (mode == 0) {
        if (rank == 0 && tid == 0) {
            uint32_t d = dead ? 0u : det;
            if (!dead && neg && d) d = M.p - d;
            *J.det = d;
        }
        return;
    }
    if (rank == 0 && tid == 0) *J.det = dead ? 0u : 1u;
    if (dead) return;
    // undo the row exchanges as column exchanges, last first
    for (int k = n - 1; k >= 0; --k) {
        const int q = swp[k];
        if (q == k) continue;
        for (int r = tid; r < nloc; r += kECT) {
            const int32_t t = rows[r * n + k];
            rows[r * n + k] = rows[r * n + q];
            rows[r * n + q] = t;
        }
        __syncthreads();
    }
    for (int e = tid; e < nloc * J.ld; e += kECT) {
        const int r = e / J.ld, c = e % J.ld;
        J.Cinv[(int64_t)(rbeg + r) * J.ld + c] = c < n ? rows[r * n + c] : 0;
    }
}

// det A mod p by division-free elimination on an 8-CTA cluster (the
// matrix in distributed shared memory as for k_elim_cluster): at step k,
// with pivot d_k = a_kk (first nonzero at or below the diagonal, Section
// 2.1's rule), every row i > k becomes d_k a_i - a_ik a_k, which multiplies
// the trailing determinant by d_k^(n-k-1). Hence
//   det A = (-1)^swaps Q_n / prod_{j=1}^{n-1} Q_j,  Q_j = d_0 ... d_{j-1},
// with one inverse at the end instead of one per column. Every block reads
// the next pivot row straight from its owner after the column's cluster
// barrier; only a zero pivot takes the search (uniform over the cluster).
__global__ void __cluster_dims__(kEC, 1, 1) __launch_bounds__(kECT)
k_det_cluster(const ElimJob *__restrict__ jobs) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) int32_t es[];
    __shared__ int s_cand[2];
    __shared__ int32_t s_pv;
    const ElimJob J = jobs[blockIdx.x / kEC];
    const int rank = (int)cl.block_rank();
    const int n = J.n, chunk = (n + kEC - 1) / kEC;
    const ModP M = J.mod;
    const int rbeg = rank * chunk, rend = min(n, rbeg + chunk);
    const int nloc = rend > rbeg ? rend - rbeg : 0;
    int32_t *rows = es;                      // chunk x n
    int32_t *prow = es + (size_t)chunk * n;  // n: pivot row copy
    const int tid = threadIdx.x;
    for (int e = tid; e < nloc * n; e += kECT) {
        const int r = e / n, c = e % n;
        rows[e] = red_bal(J.A[(int64_t)(rbeg + r) * J.lda + c], M);
    }
    int32_t Q = 1, den = 1;
    int neg = 0, dead = 0;
    __syncthreads();
    cl.sync();
    for (int k = 0; k < n; ++k) {
        const int owner = k / chunk;
        int32_t *kr = cl.map_shared_rank(rows, owner) + (size_t)(k - owner * chunk) * n;
        if (tid == 0) s_pv = kr[k];
        __syncthreads();
        int32_t pv = s_pv;
        if (pv == 0) {
            const int par = k & 1;
            if (tid == 0) s_cand[par] = INT_MAX;
            __syncthreads();
            for (int r = tid; r < nloc; r += kECT)
                if (rbeg + r > k && rows[r * n + k] != 0) atomicMin(&s_cand[par], rbeg + r);
            cl.sync();
            int best = INT_MAX;
            for (int q = 0; q < kEC; ++q) best = min(best, *cl.map_shared_rank(&s_cand[par], q));
            if (best == INT_MAX) {
                dead = 1;
                break;
            }
            const int po = best / chunk;
            int32_t *pr = cl.map_shared_rank(rows, po) + (size_t)(best - po * chunk) * n;
            if (rank == 0)
                for (int c = k + tid; c < n; c += kECT) {
                    const int32_t t = kr[c];
                    kr[c] = pr[c];
                    pr[c] = t;
                }
            neg ^= 1;
            cl.sync();
            if (tid == 0) s_pv = kr[k];
            __syncthreads();
            pv = s_pv;
        }
        for (int c = k + 1 + tid; c < n; c += kECT) prow[c] = kr[c];
        if (tid == 0) {
            Q = mul_bal(Q, pv, M);
            if (k < n - 1) den = mul_bal(den, Q, M);
        }
        __syncthreads();
        // rows by 4 groups, columns by 128 threads
        const int rg = tid >> 7, ct = tid & 127;
        for (int r = max(0, k + 1 - rbeg) + rg; r < nloc; r += 4) {
            int32_t *row = rows + (size_t)r * n;
            const int32_t l = row[k];
            for (int c = k + 1 + ct; c < n; c += 128)
                row[c] = red_bal((int64_t)pv * row[c] - (int64_t)l * prow[c], M);
        }
        __syncthreads();
        cl.sync();
    }
    cl.sync();  // no CTA leaves while others may still read its rows
    if (rank == 0 && tid == 0) {
        uint32_t d = 0;
        if (!dead) {
            int32_t v = mul_bal(Q, inv32(den, M.p), M);
            if (neg) v = -v;
            d = v < 0 ? (uint32_t)(v + (int32_t)M.p) : (uint32_t)v;
        }
        *J.det = d;
    }
}

}  // namespace

static size_t elim_smem(int n) {
    const int chunk = (n + kEC - 1) / kEC;
    return sizeof(int32_t) * ((size_t)chunk * n + 2 * (size_t)n + chunk) + 64;
}

bool elim_cluster_fits(int n) { return n >= 1 && elim_smem(n) <= 200 * 1024; }

int launch_elim_cluster(const ElimJob *jobs_dev, int count, int max_n, int mode, cudaStream_t s) {
    if (count <= 0) return IDET_OK;
    const size_t smem = elim_smem(max_n);
    if (!elim_cluster_fits(max_n)) {
        set_last_error("cluster elimination: n = %d too large", max_n);
        return IDET_ERR_ARG;
    }
    IDET_TRY(allow_max_smem((const void *)k_elim_cluster));
    if (mode == 0) {
        IDET_TRY(allow_max_smem((const void *)k_det_cluster));
        k_det_cluster<<<count * kEC, kECT, smem, s>>>(jobs_dev);
    } else {
        k_elim_cluster<<<count * kEC, kECT, smem, s>>>(jobs_dev, mode);
    }
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    return IDET_OK;
}

}  // namespace idet
