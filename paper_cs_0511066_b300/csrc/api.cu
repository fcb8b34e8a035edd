// C ABI of libidet and the host-side control of Alg. 4.1 (i_max = 1).
//
// The host code here only sequences kernels and takes the paper's control
// decisions (which primes, when to stop, how many lifting steps); every
// arithmetic step on A, its residues, the lifting state and the multi-word
// results runs in the kernels of k_*.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <set>
#include <string>
#include <functional>
#include <thread>
#include <unordered_set>
#include <vector>

#include "idet_internal.cuh"

namespace idet {

// ---------------------------------------------------------------------------
// Errors, allocator, launch counter

static thread_local char g_err[1024] = "no error";
std::atomic<unsigned long long> g_launches{0};
thread_local bool t_native_alloc = false;
thread_local int t_reserve_sms = 0;

void set_last_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int allow_max_smem(const void *kernel) {
    // the attribute belongs to the current device: remember (device, kernel)
    static std::mutex mu;
    static std::set<std::pair<int, const void *>> done;
    int dev = 0, optin = 0;
    IDET_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (done.count({dev, kernel})) return IDET_OK;
    cudaFuncAttributes fa;
    IDET_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    IDET_CUDA_TRY(cudaFuncGetAttributes(&fa, kernel));
    IDET_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       optin - (int)fa.sharedSizeBytes));
    done.insert({dev, kernel});
    return IDET_OK;
}

static idet_alloc_fn g_alloc = nullptr;
static idet_free_fn g_free = nullptr;
static void *g_actx = nullptr;

Workspace::Workspace(cudaStream_t s) : stream_(s), native_(t_native_alloc || !g_alloc) {}

Workspace::~Workspace() {
    for (size_t i = ptrs_.size(); i-- > 0;) {
        if (!native_)
            g_free(ptrs_[i], (void *)stream_, g_actx);
        else
            cudaFreeAsync(ptrs_[i], stream_);
    }
}

int Workspace::raw_alloc(void **ptr, size_t bytes) {
    void *p = nullptr;
    if (!native_) {
        p = g_alloc(bytes, (void *)stream_, g_actx);
    } else if (cudaMallocAsync(&p, bytes, stream_) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (!p) {
        set_last_error("workspace: could not allocate %zu bytes of device memory", bytes);
        return IDET_ERR_NOMEM;
    }
    ptrs_.push_back(p);
    *ptr = p;
    return IDET_OK;
}

int Workspace::alloc(void **ptr, size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    if (bytes >= kDirect) return raw_alloc(ptr, bytes);
    if (bytes > chunk_left_) {
        void *c = nullptr;
        IDET_TRY(raw_alloc(&c, kChunk));
        chunk_ = (char *)c;
        chunk_left_ = kChunk;
    }
    *ptr = chunk_;
    chunk_ += bytes;
    chunk_left_ -= bytes;
    return IDET_OK;
}

// ---------------------------------------------------------------------------
// Primes and random numbers (parameter choice; Alg. 2.1 draws its primes at random)

static const uint32_t kLo21 = 1u << 20, kHi21 = 1u << 21;

static const std::vector<uint32_t> &pool21() {
    static std::vector<uint32_t> pool;
    static std::once_flag once;
    std::call_once(once, [] {
        std::vector<uint8_t> comp(kHi21, 0);
        for (uint32_t i = 2; (uint64_t)i * i < kHi21; ++i)
            if (!comp[i])
                for (uint32_t j = i * i; j < kHi21; j += i) comp[j] = 1;
        for (uint32_t v = kLo21 + 1; v < kHi21; ++v)
            if (!comp[v]) pool.push_back(v);
    });
    return pool;
}

struct SplitMix {
    uint64_t s;
    explicit SplitMix(uint64_t seed) : s(seed) {}
    uint64_t next() {
        uint64_t z = (s += 0x9e3779b97f4a7c15ull);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        return z ^ (z >> 31);
    }
    uint64_t below(uint64_t n) { return next() % n; }
};

static uint64_t powmod64(uint64_t a, uint64_t e, uint64_t m) {
    unsigned __int128 r = 1, b = a % m;
    while (e) {
        if (e & 1) r = r * b % m;
        b = b * b % m;
        e >>= 1;
    }
    return (uint64_t)r;
}

// Deterministic Miller-Rabin for 32-bit integers (bases 2, 7, 61).
static bool is_prime32(uint32_t n) {
    if (n < 2) return false;
    for (uint32_t q : {2u, 3u, 5u, 7u, 11u, 13u, 61u})
        if (n % q == 0) return n == q;
    uint32_t d = n - 1;
    int s = 0;
    while (!(d & 1)) {
        d >>= 1;
        ++s;
    }
    for (uint32_t a : {2u, 7u, 61u}) {
        uint64_t x = powmod64(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool ok = false;
        for (int r = 1; r < s; ++r) {
            x = (unsigned __int128)x * x % n;
            if (x == n - 1) {
                ok = true;
                break;
            }
        }
        if (!ok) return false;
    }
    return true;
}

static uint32_t random_prime31(SplitMix &g) {
    while (true) {
        uint32_t c = (uint32_t)((1u << 30) + (g.next() % (1u << 30))) | 1u;
        if (c < (1u << 31) && is_prime32(c)) return c;
    }
}

// Random primes sampled without replacement (Alg. 2.1) from one of two
// pools: the 73,586 primes in (2^20, 2^21) (l = 2^20), or the 50,697,537
// primes in (2^30, 2^31) (l = 2^30), drawn by rejection sampling.
struct PrimeDraw {
    int bits;
    std::vector<uint32_t> order;
    size_t next = 0;
    SplitMix g;
    std::unordered_set<uint32_t> seen;
    explicit PrimeDraw(uint64_t seed, int b = 21) : bits(b), g(seed ^ 0x5eed5eedull) {
        if (bits != 31) {
            order = pool21();
            for (size_t i = order.size() - 1; i > 0; --i) std::swap(order[i], order[g.below(i + 1)]);
        }
    }
    bool take(uint32_t &p) {
        if (bits == 31) {
            if (seen.size() >= (1u << 24)) return false;
            do {
                p = random_prime31(g);
            } while (!seen.insert(p).second);
            return true;
        }
        if (next >= order.size()) return false;
        p = order[next++];
        return true;
    }
    double pool() const { return bits == 31 ? 50697537.0 : (double)pool21().size(); }
    double log2l() const { return bits == 31 ? 30.0 : 20.0; }
};

static uint64_t inv_mod_2_64(uint64_t p) {
    uint64_t x = p;  // p * p = 1 mod 8
    for (int i = 0; i < 6; ++i) x *= 2 - p * x;
    return x;
}

// ---------------------------------------------------------------------------
// Early-termination control of Alg. 2.1 (Lemma 2.1(iii), (iv)).

static double log2_sum(double a, double b) {  // log2(2^a + 2^b)
    double hi = std::max(a, b), lo = std::min(a, b);
    if (lo == -INFINITY) return hi;
    return hi + std::log2(1.0 + std::exp2(lo - hi));
}

// Lemma 2.1(iv): k >= ceil(log(1/eps) / (log P' - log(log_l H))), with
// P' = |P| - ceil(log_l H). Returns 0 when the pool is too small for it.
static int k_default(double eps_log2, double pool, double log2H, double log2l) {
    double lH = log2H / log2l;
    if (lH <= 0) return 1;
    double Pp = pool - std::ceil(lH);
    if (Pp <= lH) return 0;
    return std::max(1, (int)std::ceil(-eps_log2 / (std::log2(Pp) - std::log2(lH))));
}

// A stop at the bound (prod p >= 2H, Lemma 2.1(i)) is taken kCertBits bits
// past it and then checked: the reconstructed r must satisfy |r| <= H, as
// det does. A wrong modular determinant (a fault) makes every later mixed-
// radix digit uniformly random, so |r| > H then, except with probability
// about 2^-kCertBits; the stop is reported as inconsistent (why = 3).
constexpr double kCertBits = 40.0;

struct CraScan {
    // Alg. 2.1 over digits[0..count): returns the index t of the prime at
    // which the loop stops (-1 if it does not) and why (1 ET, 2 bound, 3 bound
    // reached but the residues contradict |det| <= H).
    static int scan(const std::vector<int32_t> &dig, const std::vector<uint32_t> &pr,
                    double log2H, double eps_log2, double log2l, double pool, bool certify,
                    int *why) {
        double log2M = 0;
        std::vector<double> lM(dig.size());
        int k = 0, top = -1;
        for (size_t t = 0; t < dig.size(); ++t) {
            log2M += std::log2((double)pr[t]);
            lM[t] = log2M;
            if (t > 0 && dig[t] == 0)
                ++k;
            else
                k = 0;
            if (dig[t] != 0) top = (int)t;
            // the sum of t + 1 rounded logarithms is below the true log2 M
            // by less than 1e-12 (t + 1); the check below needs a lower bound
            if (log2M - 1e-12 * (double)(t + 1) >= 1.0 + log2H + kCertBits) {
                // |r| >= (|v_top| - 1/2) prod_{j<top} p_j with balanced digits
                double lo = -INFINITY;
                if (top == 0)
                    lo = std::log2(std::fabs((double)dig[0]));
                else if (top > 0)
                    lo = lM[top - 1] + std::log2(std::fabs((double)dig[top]) - 0.5);
                *why = lo > log2H + 1e-9 ? 3 : 2;
                return (int)t;
            }
            if (certify || k == 0) continue;
            // |r| < (|v_top| + 1) prod_{j<top} p_j
            double lr = -INFINITY;
            if (top >= 0)
                lr = (top > 0 ? lM[top - 1] : 0.0) + std::log2(std::fabs((double)dig[top]) + 1.0);
            double num = log2_sum(log2H, lr);
            double Rp = std::ceil((num - lM[t - k]) / log2l - 1e-12);
            if (Rp < 0) Rp = 0;
            double ratio = 1.0;
            double i_used = (double)(t + 1);
            for (int j = 0; j < k; ++j) {
                double nn = std::max(0.0, Rp - j);
                double dd = pool - i_used + k - 1 - j;
                if (dd <= 0) {
                    ratio = INFINITY;
                    break;
                }
                ratio *= nn / dd;
            }
            if (ratio < std::exp2(eps_log2)) {
                *why = 1;
                return (int)t;
            }
        }
        *why = 0;
        return -1;
    }
};

static int inconsistent_residues() {
    set_last_error("Chinese remaindering: past the bound 2H the reconstruction exceeds H, so a "
                   "modular determinant is wrong");
    return IDET_ERR_INTERNAL;
}

// ---------------------------------------------------------------------------
// Helpers

struct DevMatrix {
    const int64_t *A = nullptr;  // n x n, ld n (device)
    int64_t n = 0;
};

static int stage_matrix(const int64_t *A, int64_t n, int64_t lda, int on_device, Workspace &ws,
                        DevMatrix &out) {
    out.n = n;
    if (on_device && lda == n) {  // compact on the device already: used in place
        out.A = A;
        return IDET_OK;
    }
    int64_t *d = nullptr;
    IDET_TRY(ws.alloc_n(&d, (size_t)n * n));
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    IDET_CUDA_TRY(cudaMemcpy2DAsync(d, sizeof(int64_t) * n, A, sizeof(int64_t) * lda,
                                    sizeof(int64_t) * n, n, kind, ws.stream()));
    out.A = d;
    return IDET_OK;
}

static int write_int(idet_int *out, int sign, const uint32_t *limbs_host, uint32_t nl) {
    if (!out) return IDET_ERR_ARG;
    if (nl > out->cap || (nl > 0 && !out->limbs)) {
        out->nlimbs = nl;
        set_last_error("output integer needs %u limbs, capacity is %u", nl, out->cap);
        return IDET_ERR_BUFFER;
    }
    out->sign = nl ? sign : 0;
    out->nlimbs = nl;
    if (nl) memcpy(out->limbs, limbs_host, sizeof(uint32_t) * nl);
    return IDET_OK;
}

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t s;
    explicit Timer(cudaStream_t st) : s(st) {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, s);
    }
    double stop() {
        cudaEventRecord(b, s);
        return elapsed();
    }
    // end mark on the stream now; elapsed() waits for it later
    void mark() { cudaEventRecord(b, s); }
    double elapsed() {
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        return ms;
    }
    ~Timer() {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
};

// result = K * sum_{i<c} dig_i prod_{j<i} prs_j (K given as device limbs, or
// null for K = 1), written to out.
static int assemble_int(Workspace &ws, const std::vector<uint32_t> &prs,
                        const std::vector<int32_t> &dig, int c, const uint32_t *Kdev, int Klen,
                        idet_int *out) {
        cudaStream_t s = ws.stream();
        double bits = 64;
        for (int i = 0; i < c; ++i) bits += std::log2((double)prs[i]);
        const int cap = (int)(bits / 32) + Klen + 4;
        uint32_t *dp = nullptr, *buf = nullptr;
        int32_t *dg = nullptr, *info = nullptr;
        IDET_TRY(ws.alloc_n(&dp, c + 1));
        IDET_TRY(ws.alloc_n(&dg, c + 1));
        IDET_TRY(ws.alloc_n(&buf, 2 * (size_t)cap));
        IDET_TRY(ws.alloc_n(&info, 4));
        uint32_t one = 1;
        uint32_t *Kd = (uint32_t *)Kdev;
        if (!Kd) {
            IDET_TRY(ws.alloc_n(&Kd, 1));
            IDET_CUDA_TRY(cudaMemcpyAsync(Kd, &one, 4, cudaMemcpyHostToDevice, s));
            Klen = 1;
        }
        IDET_CUDA_TRY(cudaMemcpyAsync(dp, prs.data(), 4 * c, cudaMemcpyHostToDevice, s));
        IDET_CUDA_TRY(cudaMemcpyAsync(dg, dig.data(), 4 * c, cudaMemcpyHostToDevice, s));
        IDET_TRY(launch_mixed_to_int(dp, dg, c, Kd, Klen, buf, cap, info, s));
        int32_t hinfo[3];
        IDET_CUDA_TRY(cudaMemcpyAsync(hinfo, info, 12, cudaMemcpyDeviceToHost, s));
        IDET_CUDA_TRY(cudaStreamSynchronize(s));
        if (hinfo[2]) {
            set_last_error("reconstruction buffer too small");
            return IDET_ERR_INTERNAL;
        }
        std::vector<uint32_t> host(hinfo[1] > 0 ? hinfo[1] : 1);
        if (hinfo[1] > 0)
            IDET_CUDA_TRY(cudaMemcpyAsync(host.data(), buf, 4 * (size_t)hinfo[1],
                                          cudaMemcpyDeviceToHost, s));
        IDET_CUDA_TRY(cudaStreamSynchronize(s));
        return write_int(out, hinfo[0], host.data(), (uint32_t)hinfo[1]);
    }

// Per-call state of the determinant computation.
struct DetJob {
    DevMatrix M;
    Workspace &ws;
    cudaStream_t s;
    idet_opts o;
    int nb;
    // matrix statistics
    double log2H = 0;
    std::vector<double> rowsq;
    uint64_t amax = 0;
    std::vector<double> colsq;
    void *Anar = nullptr;  // A as int8/int16/int32, rows padded to ldl
    int abytes = 4;
    int64_t ldl = 0;
    // CRA state
    PrimeDraw draw;
    std::vector<uint32_t> primes;   // factored primes
    std::vector<uint32_t> dets;     // det(A) mod primes
    idet_stats st{};

    // A^{-1} mod a lifting prime formed ahead of the solve (on a second
    // stream while the first CRA wave is factored), or null
    int32_t *pre_Cinv = nullptr;
    uint32_t pre_p = 0;

    // work run by the host while the reconstruction kernel is on the device
    // (the first CRA wave, on a stream of its own), and its status
    std::function<int()> during_rr;
    int during_rr_rc = IDET_OK;
    bool during_rr_ran = false;

    // LU factors kept from a wave of 31-bit CRA primes (primes[lu_first ..
    // lu_first + lu_count)): residues and permutations, prime-major
    int32_t *lu_R = nullptr, *lu_perm = nullptr;
    int lu_first = 0, lu_count = 0;

    // multi-word entries (idet_int_det_mp): sign x L base-2^32 limbs
    const uint32_t *mag = nullptr;
    const int8_t *sgn = nullptr;
    int L = 0;

    DetJob(const DevMatrix &m, Workspace &w, const idet_opts &opts, int prime_bits = 21)
        : M(m), ws(w), s(w.stream()), o(opts), draw(opts.seed, prime_bits) {
        nb = o.nb > 0 ? o.nb : 32;
    }

    // A mod p for W primes into R (W x n x n balanced int32)
    int reduce(const ModP *md, int W, int32_t *R) {
        if (mag) return launch_reduce_mp(mag, sgn, M.n, L, md, W, R, s);
        return launch_reduce(M.A, M.n, M.n, md, W, R, s);
    }

    int stats() {
        const int64_t n = M.n;
        double *d_rowsq = nullptr;
        unsigned long long *d_amax = nullptr;
        IDET_TRY(ws.alloc_n(&d_rowsq, n));
        IDET_TRY(ws.alloc_n(&d_amax, 1));
        IDET_TRY(launch_row_stats(M.A, n, n, d_rowsq, d_amax, s));
        rowsq.resize(n);
        IDET_CUDA_TRY(cudaMemcpyAsync(rowsq.data(), d_rowsq, sizeof(double) * n,
                                      cudaMemcpyDeviceToHost, s));
        IDET_CUDA_TRY(cudaMemcpyAsync(&amax, d_amax, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
        double *d_colsq = nullptr;
        IDET_TRY(ws.alloc_n(&d_colsq, n));
        IDET_TRY(launch_col_stats(M.A, n, n, d_colsq, s));
        colsq.resize(n);
        IDET_CUDA_TRY(cudaMemcpyAsync(colsq.data(), d_colsq, sizeof(double) * n,
                                      cudaMemcpyDeviceToHost, s));
        IDET_CUDA_TRY(cudaStreamSynchronize(s));
        unsigned long long am = 0;
        if (!entry_range(amax, &am)) {
            set_last_error("entries must lie in [-2^31, 2^31 - 1]");
            return IDET_ERR_ARG;
        }
        amax = am;
        // Hadamard: |det A| <= prod of the row norms and <= prod of the
        // column norms (Lemma 2.1 uses H = (sqrt(n) ||A||)^n, which bounds
        // both); the smaller one is used.
        double hr = 0, hc = 0;
        for (double v : rowsq) hr += v > 0 ? 0.5 * std::log2(v) : -INFINITY;
        for (double v : colsq) hc += v > 0 ? 0.5 * std::log2(v) : -INFINITY;
        // margin for the rounding of the logarithms and their sum (upper
        // bound kept)
        log2H = std::min(hr, hc);
        if (log2H > -INFINITY) log2H = log2H * (1 + 1e-12) + 1e-6 * (double)n;
        st.log2_H = log2H;
        return IDET_OK;
    }

    // det(A) mod p for W more primes (appended to primes/dets).
    int factor_wave(int W) {
        const int64_t n = M.n;
        std::vector<uint32_t> pw;
        for (int i = 0; i < W; ++i) {
            uint32_t p;
            if (!draw.take(p)) break;
            pw.push_back(p);
        }
        W = (int)pw.size();
        if (W == 0) {
            set_last_error("prime pool exhausted");
            return IDET_ERR_INTERNAL;
        }
        std::vector<ModP> mh(W);
        for (int i = 0; i < W; ++i) mh[i] = make_mod(pw[i]);
        ModP *md = nullptr;
        int32_t *R = nullptr, *perm = nullptr;
        uint32_t *dd = nullptr;
        // primes of the lifting class (31 bits): the factors of the first
        // wave are kept, so that the lift can take one of these primes and
        // its LU instead of factoring a prime of its own
        const bool keep = draw.bits == 31 && !lu_R && !mag;
        IDET_TRY(ws.alloc_n(&md, W));
        IDET_TRY(ws.alloc_n(&R, (size_t)W * n * n));
        IDET_TRY(ws.alloc_n(&dd, W));
        if (keep) IDET_TRY(ws.alloc_n(&perm, (size_t)W * n));
        IDET_CUDA_TRY(cudaMemcpyAsync(md, mh.data(), sizeof(ModP) * W, cudaMemcpyHostToDevice, s));
        Timer t(s);
        IDET_TRY(reduce(md, W, R));
        IDET_TRY(lu_factor_batched(R, n, md, mh.data(), W, draw.bits == 31, o.nb, perm, dd,
                                   o.update_path, ws));
        if (keep) {
            lu_R = R;
            lu_perm = perm;
            lu_first = (int)primes.size();
            lu_count = W;
        }
        std::vector<uint32_t> res(W);
        IDET_CUDA_TRY(cudaMemcpyAsync(res.data(), dd, sizeof(uint32_t) * W,
                                      cudaMemcpyDeviceToHost, s));
        st.ms_lu += t.stop();
        for (int i = 0; i < W; ++i) {
            // failure-detection hook: a wrong modular determinant, made on
            // the host, for the prime with 1-based index o.inject_fault
            if (o.inject_fault > 0 && (int)primes.size() + 1 == o.inject_fault)
                res[i] = (res[i] + 1) % pw[i];
            primes.push_back(pw[i]);
            dets.push_back(res[i]);
        }
        st.primes_used += W;
        st.lu_macs += (2.0 / 3.0) * (double)n * n * n * W;
        return IDET_OK;
    }

    // Garner digits of the residues res (mod prs) on the device.
    int cra_digits(const std::vector<uint32_t> &prs, const std::vector<uint32_t> &res,
                   std::vector<int32_t> &dig) {
        const int c = (int)prs.size();
        dig.assign(c, 0);
        if (c == 0) return IDET_OK;
        uint32_t *dp = nullptr, *dr = nullptr;
        int32_t *dg = nullptr;
        IDET_TRY(ws.alloc_n(&dp, c));
        IDET_TRY(ws.alloc_n(&dr, c));
        IDET_TRY(ws.alloc_n(&dg, c));
        IDET_CUDA_TRY(cudaMemcpyAsync(dp, prs.data(), 4 * c, cudaMemcpyHostToDevice, s));
        IDET_CUDA_TRY(cudaMemcpyAsync(dr, res.data(), 4 * c, cudaMemcpyHostToDevice, s));
        IDET_TRY(launch_cra_append(dp, dr, dg, 0, c, nullptr, s));
        IDET_CUDA_TRY(cudaMemcpyAsync(dig.data(), dg, 4 * c, cudaMemcpyDeviceToHost, s));
        IDET_CUDA_TRY(cudaStreamSynchronize(s));
        return IDET_OK;
    }

    // result = K * sum_{i<c} dig_i prod_{j<i} prs_j, K given as device limbs.
    int assemble(const std::vector<uint32_t> &prs, const std::vector<int32_t> &dig, int c,
                 const uint32_t *Kdev, int Klen, idet_int *out) {
        return assemble_int(ws, prs, dig, c, Kdev, Klen, out);
    }
};

// LU + inverse mod a 31-bit prime; returns IDET_ERR_SINGULAR if A is
// singular mod p. Cinv: n rows of ld4 entries (zero padded columns).
static int inverse_mod_prime(const DevMatrix &M, uint32_t p, int nb, Workspace &ws, int32_t *Cinv,
                             int64_t ld4) {
    cudaStream_t s = ws.stream();
    const int64_t n = M.n;
    ModP mh = make_mod(p);
    ModP *md = nullptr;
    int32_t *R = nullptr, *perm = nullptr, *Y = nullptr;
    uint32_t *dd = nullptr;
    IDET_TRY(ws.alloc_n(&md, 1));
    IDET_TRY(ws.alloc_n(&R, (size_t)n * n));
    IDET_TRY(ws.alloc_n(&perm, n));
    IDET_TRY(ws.alloc_n(&dd, 1));
    IDET_CUDA_TRY(cudaMemcpyAsync(md, &mh, sizeof(ModP), cudaMemcpyHostToDevice, s));
    IDET_TRY(launch_reduce(M.A, n, n, md, 1, R, s));
    IDET_TRY(lu_factor_batched(R, n, md, &mh, 1, true, nb, perm, dd, IDET_PATH_AUTO, ws));
    uint32_t det = 0;
    IDET_CUDA_TRY(cudaMemcpyAsync(&det, dd, 4, cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaStreamSynchronize(s));
    if (det == 0) return IDET_ERR_SINGULAR;
    IDET_TRY(ws.alloc_n(&Y, (size_t)n * n));
    IDET_TRY(lu_inverse(R, perm, n, mh, md, true, nb, Y, Cinv, ld4, ws));
    return IDET_OK;
}

// The lifting prime and C = A^{-1} mod p: a CRA prime of the lifting class
// whose LU the first wave kept (det A != 0 mod p), else random 31-bit primes
// (up to 6, a prime dividing det A is skipped) with an LU of their own.
static int lift_prime_inverse(DetJob &J, int32_t *Cinv, int64_t ld4, uint32_t *p_out) {
    Workspace &ws = J.ws;
    cudaStream_t s = J.s;
    const int64_t n = J.M.n;
    for (int w = 0; w < J.lu_count && J.lu_R; ++w) {
        const int k = J.lu_first + w;
        if (J.dets[k] == 0) continue;
        const uint32_t p = J.primes[k];
        const ModP mh = make_mod(p);
        ModP *md = nullptr;
        IDET_TRY(ws.alloc_n(&md, 1));
        IDET_CUDA_TRY(cudaMemcpyAsync(md, &mh, sizeof(ModP), cudaMemcpyHostToDevice, s));
        const int32_t *R = J.lu_R + (size_t)w * n * n;
        const int32_t *perm = J.lu_perm + (size_t)w * n;
        int32_t *Y = nullptr;
        IDET_TRY(ws.alloc_n(&Y, (size_t)n * n));
        IDET_TRY(lu_inverse(R, perm, n, mh, md, true, J.nb, Y, Cinv, ld4, ws));
        J.st.inverse_macs += (2.0 / 3.0) * (double)n * n * n;
        *p_out = p;
        return IDET_OK;
    }
    SplitMix g(J.o.seed ^ 0x11f7ull);
    int rc = IDET_ERR_SINGULAR;
    uint32_t p = 0;
    for (int tries = 0; tries < 6 && rc == IDET_ERR_SINGULAR; ++tries) {
        p = random_prime31(g);
        rc = inverse_mod_prime(J.M, p, J.nb, ws, Cinv, ld4);
    }
    if (rc == IDET_OK) J.st.inverse_macs += (4.0 / 3.0) * (double)n * n * n;
    *p_out = p;
    return rc;
}

// A in the narrowest of int8/int16/int32 holding max |a_ij| = amax, rows
// padded with zeros to ldl = n rounded up to a multiple of 16.
static int make_Anar(const DevMatrix &M, uint64_t amax, Workspace &ws, void **out, int *abytes,
                     int64_t *ldl) {
    const int64_t n = M.n;
    *ldl = (n + 15) / 16 * 16;
    *abytes = amax <= 127 ? 1 : (amax <= 32767 ? 2 : 4);
    void *a = nullptr;
    IDET_TRY(ws.alloc(&a, (size_t)n * *ldl * *abytes + 64));
    IDET_TRY(launch_narrow(M.A, n, n, a, *ldl, *abytes, ws.stream()));
    *out = a;
    return IDET_OK;
}

// Section 2.2: one Dixon solve with right-hand side b, then the denominator
// of the projection u . x by rational reconstruction. Kdig receives the
// base-p digits of the denominator (host), Kp the lift prime.
struct LiftResult {
    uint32_t p = 0;
    int m = 0;
    bool has_den = false;
    uint32_t *Kbin = nullptr;  // the denominator in 32-bit limbs (device)
    int Klen = 0;
    double log2K = 0;
    int timed_out = 0;
};

static int den_to_binary(Workspace &ws, const std::vector<uint32_t> &den, uint32_t p,
                         uint32_t **Kbin, int *Klen, double *log2K);

static int solve_and_denominator(DetJob &J, const int64_t *b_dev, const std::vector<int64_t> &b_host,
                                 const int32_t *u_dev, double log2u1, LiftResult &out) {
    const int64_t n = J.M.n;
    Workspace &ws = J.ws;
    cudaStream_t s = J.s;
    if (!J.Anar) IDET_TRY(make_Anar(J.M, J.amax, ws, &J.Anar, &J.abytes, &J.ldl));
    int32_t *Cinv = J.pre_Cinv;
    uint32_t p = J.pre_p;
    if (!Cinv) {
        IDET_TRY(ws.alloc_n(&Cinv, (size_t)n * J.ldl));
        Timer tinv(s);
        const int rc = lift_prime_inverse(J, Cinv, J.ldl, &p);
        J.st.ms_inverse += tinv.stop();
        if (rc != IDET_OK) return rc;
    }
    // Bounds (Cramer): x_j = N_j / det A. The denominator of u.x divides
    // det A, |det A| <= H; the numerator of u.x is at most
    // ||u||_1 max_j |N_j| with |N_j| = |det A_j(b)| <= ||b||_2 prod_{k != j}
    // ||col_k||_2 (Hadamard on the columns of A with column j replaced by b).
    double log2D = J.log2H, log2N = log2u1, bb = 1.0, lc = 0, lcmin = INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        double bi = (double)b_host[i];
        bb += bi * bi;
        double c = 0.5 * std::log2(std::max(J.colsq[i], 1.0));
        lc += c;
        lcmin = std::min(lcmin, c);
    }
    log2N += 0.5 * std::log2(bb * (1 + 1e-12)) + lc - lcmin;
    const double lp = std::log2((double)p);
    const int hN = (int)std::ceil((log2N + 1) / lp);
    const int hD = (int)std::ceil((log2D + 1) / lp);
    const int m = hN + hD + 2;
    LiftArgs a{};
    a.Cinv = Cinv;
    a.b = b_dev;
    a.u = u_dev;
    a.n = n;
    a.m = m;
    a.mod = make_mod(p);
    a.pinv = inv_mod_2_64(p);
    int64_t *z = nullptr, *r = nullptr;
    IDET_TRY(ws.alloc_n(&z, m));
    IDET_TRY(ws.alloc_n(&r, n));
    a.zproj = z;
    a.r = r;
    a.digits = nullptr;
    a.amax = J.amax;
    float kms = 0;
    LiftInfo li{};
    IDET_TRY(launch_lift(a, J.Anar, J.abytes, J.ldl, ws, &out.timed_out, &kms, &li));
    J.st.ms_lift_kernel += li.ms_steps;
    J.st.ms_lift_setup += li.ms_setup;
    J.st.lift_bytes += li.bytes;
    J.st.lift_path = li.path;
    uint32_t *den = nullptr;
    int32_t *info = nullptr;
    const int den_cap = hD + 4;
    IDET_TRY(ws.alloc_n(&den, den_cap));
    IDET_TRY(ws.alloc_n(&info, 4));
    Timer trr(s);
    // the denominator straight in binary where the numbers fit in shared
    // memory, else in base p and converted
    const bool bin = ratrecon_bin_fits(m, hN, hD);
    if (bin)
        IDET_TRY(launch_ratrecon_bin(z, m, p, hN, hD, den, den_cap, info, ws));
    else
        IDET_TRY(launch_ratrecon(z, m, p, hN, hD, den, den_cap, info, ws));
    trr.mark();  // the reconstruction kernel's end, on its stream
    if (J.during_rr) {
        // the reconstruction holds one SM: the other SMs take the hook's work
        auto hook = std::move(J.during_rr);
        J.during_rr = nullptr;
        J.during_rr_rc = hook();
        J.during_rr_ran = true;
    }
    int32_t hinfo[4] = {0, 0, 0, 0};
    IDET_CUDA_TRY(cudaMemcpyAsync(hinfo, info, 16, cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaStreamSynchronize(s));
    J.st.ms_rr += trr.elapsed();
    if (hinfo[0] != 0) {
        set_last_error("rational reconstruction failed (code %d)", hinfo[0]);
        return IDET_ERR_INTERNAL;
    }
    if (bin) {
        out.Kbin = den;
        out.Klen = hinfo[1];
        out.log2K = std::log2((double)(uint32_t)hinfo[3]) + std::max(0, hinfo[2] - 31);
    } else {
        Timer tb(s);
        std::vector<uint32_t> dd(hinfo[1]);
        IDET_CUDA_TRY(cudaMemcpyAsync(dd.data(), den, 4 * (size_t)hinfo[1],
                                      cudaMemcpyDeviceToHost, s));
        IDET_CUDA_TRY(cudaStreamSynchronize(s));
        IDET_TRY(den_to_binary(ws, dd, p, &out.Kbin, &out.Klen, &out.log2K));
        J.st.ms_rr += tb.stop();
    }
    out.has_den = true;
    out.p = p;
    out.m = m;
    return IDET_OK;
}

static double rhs_range_log2(int64_t n, double log2H) {
    // Alg. 4.1: S = 13 E(#factors)^3 ceil(log H)^4, E(#factors) =
    // ceil(sqrt(2 log2 n)) + 3 (Section 4.1), clamped to 2^62.
    double e = std::ceil(std::sqrt(2.0 * std::log2((double)std::max<int64_t>(n, 2)))) + 3;
    double lh = std::ceil(std::max(log2H, 1.0));
    double l2 = std::log2(13.0) + 3 * std::log2(e) + 4 * std::log2(lh);
    return std::min(l2, 62.0);
}

// Primes per wave after the first (the first wave has the k0 primes of
// Lemma 2.1(iv)): the caller's, else the autotuner's, else max(8, k0).
static int default_wave(const idet_opts &o, int64_t n, int prime_bits, int k0) {
    if (o.wave > 0) return o.wave;
    idet_tuned t{};
    if (tuned_lookup(n, prime_bits, &t) && t.wave > 0) return std::max(t.wave, 1);
    return std::max(8, k0);
}

// Alg. 2.1 on det(A) for the first primes (Alg. 4.1 lines 1-4), or all the
// way in CRA-only / certified mode. *done when det has been written.
static int det_first(DetJob &J, int k0, int wave, bool cra_only, idet_int *det, bool *done) {
    const idet_opts &o = J.o;
    std::vector<int32_t> dig;
    int why = 0;
    *done = false;
    IDET_TRY(J.factor_wave(cra_only ? wave : std::max(k0, 1)));
    while (true) {
        Timer t(J.s);
        IDET_TRY(J.cra_digits(J.primes, J.dets, dig));
        J.st.ms_cra += t.stop();
        const int stop = CraScan::scan(dig, J.primes, J.log2H, o.log2_epsilon, J.draw.log2l(),
                                       J.draw.pool(), o.certify != 0, &why);
        if (stop >= 0) {
            J.st.et_stop = why;
            J.st.primes_in_cra = stop + 1;
            if (why == 3) return inconsistent_residues();
            Timer t2(J.s);
            const int rc = J.assemble(J.primes, dig, stop + 1, nullptr, 0, det);
            J.st.ms_cra += t2.stop();
            *done = true;
            return rc;
        }
        if (!cra_only) return IDET_OK;
        IDET_TRY(J.factor_wave(wave));
    }
}

// K from its base-p digits: base-2^32 limbs on the device, and log2 K.
static int den_to_binary(Workspace &ws, const std::vector<uint32_t> &den, uint32_t p,
                         uint32_t **Kbin, int *Klen, double *log2K) {
    cudaStream_t s = ws.stream();
    const int kd = (int)den.size();
    const int cap = kd + 2;
    uint32_t *dd = nullptr;
    int32_t *dl = nullptr;
    IDET_TRY(ws.alloc_n(&dd, kd));
    IDET_TRY(ws.alloc_n(Kbin, cap));
    IDET_TRY(ws.alloc_n(&dl, 1));
    IDET_CUDA_TRY(cudaMemcpyAsync(dd, den.data(), 4 * (size_t)kd, cudaMemcpyHostToDevice, s));
    IDET_TRY(launch_radix_to_binary(dd, kd, p, *Kbin, cap, dl, s));
    IDET_CUDA_TRY(cudaMemcpyAsync(Klen, dl, 4, cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaStreamSynchronize(s));
    const double top = den[kd - 1] + (kd > 1 ? den[kd - 2] / (double)p : 0.0);
    *log2K = std::log2(top) + (kd - 1) * std::log2((double)p);
    return IDET_OK;
}

// Alg. 2.1 on det(A)/K, using the residues already computed first
// (Section 4: the modular determinants computed so far are reused). Primes
// dividing K are skipped. K = null: det(A) itself. to_bound: no early
// termination, stop once the product of the primes reaches 2H/K.
static int det_over_K(DetJob &J, const uint32_t *Kbin, int Klen, double log2K, int wave,
                      idet_int *det, bool to_bound = false, double budget_ms = -1,
                      bool *done = nullptr) {
    const idet_opts &o = J.o;
    Workspace &ws = J.ws;
    cudaStream_t s = J.s;
    const double log2HK = std::max(0.0, J.log2H - log2K);
    std::vector<int32_t> dig;
    int why = 0;
    if (done) *done = false;
    if (J.primes.empty()) IDET_TRY(J.factor_wave(wave));
    double spent = 0;  // device time of the waves factored here (budgeted resume)
    while (true) {
        std::vector<uint32_t> prs, res;
        Timer t(s);
        if (Kbin) {
            const int c = (int)J.primes.size();
            uint32_t *dp = nullptr, *di = nullptr, *dout = nullptr;
            int32_t *dskip = nullptr;
            IDET_TRY(ws.alloc_n(&dp, c));
            IDET_TRY(ws.alloc_n(&di, c));
            IDET_TRY(ws.alloc_n(&dout, c));
            IDET_TRY(ws.alloc_n(&dskip, c));
            IDET_CUDA_TRY(cudaMemcpyAsync(dp, J.primes.data(), 4 * c, cudaMemcpyHostToDevice, s));
            IDET_CUDA_TRY(cudaMemcpyAsync(di, J.dets.data(), 4 * c, cudaMemcpyHostToDevice, s));
            IDET_TRY(launch_div_by_K(Kbin, Klen, dp, di, dout, dskip, c, s));
            std::vector<uint32_t> hout(c);
            std::vector<int32_t> hskip(c);
            IDET_CUDA_TRY(cudaMemcpyAsync(hout.data(), dout, 4 * c, cudaMemcpyDeviceToHost, s));
            IDET_CUDA_TRY(cudaMemcpyAsync(hskip.data(), dskip, 4 * c, cudaMemcpyDeviceToHost, s));
            IDET_CUDA_TRY(cudaStreamSynchronize(s));
            for (int i = 0; i < c; ++i)
                if (!hskip[i]) {
                    prs.push_back(J.primes[i]);
                    res.push_back(hout[i]);
                }
        } else {
            prs = J.primes;
            res = J.dets;
        }
        IDET_TRY(J.cra_digits(prs, res, dig));
        const int stop = CraScan::scan(dig, prs, Kbin ? log2HK : J.log2H, o.log2_epsilon,
                                       J.draw.log2l(), J.draw.pool(), to_bound, &why);
        J.st.ms_cra += t.stop();
        if (stop >= 0) {
            J.st.et_stop = why;
            J.st.primes_in_cra = stop + 1;
            if (why == 3) return inconsistent_residues();
            Timer t2(s);
            const int rc = J.assemble(prs, dig, stop + 1, Kbin, Klen, det);
            J.st.ms_cra += t2.stop();
            if (done) *done = rc == IDET_OK;
            return rc;
        }
        if (budget_ms >= 0 && spent >= budget_ms) return IDET_OK;  // resumed later
        const double before = J.st.ms_lu;
        IDET_TRY(J.factor_wave(wave));
        spent += J.st.ms_lu - before;
    }
}

// Section 2.2 for multi-word entries, output-sensitive: the lift runs in
// chunks and after each chunk of m digits tries to reconstruct u . x with
// balanced bounds (numerator < p^(m-2-h), denominator D < p^h). A candidate
// D is accepted only when every y_j = D X_j mod p^m is small, |y_j| < p^h,
// and n max|a_ij| p^h + D max|b_i| < p^m / 2: then A y = D b holds over Z
// (A X = b mod p^m, and both sides are below p^m / 2), so x = y / D, every
// D x_j is an integer and D, the denominator of u . x, is the lcm of the
// denominators of x, s~_n. Without acceptance by m_cap digits, no K.
struct MpLift {
    uint32_t p = 0;
    int m = 0;
    std::vector<uint32_t> den;
};

static int mp_lift(DetJob &J, unsigned int abits, MpLift &out) {
    const int64_t n = J.M.n;
    Workspace &ws = J.ws;
    cudaStream_t s = J.s;
    SplitMix g(J.o.seed ^ 0x11f7ull);
    // A^{-1} mod p for a 31-bit p with det A != 0 mod p
    Timer tinv(s);
    int32_t *R = nullptr, *perm = nullptr, *C = nullptr;
    ModP *md = nullptr;
    uint32_t *dd = nullptr;
    IDET_TRY(ws.alloc_n(&R, (size_t)n * n));
    IDET_TRY(ws.alloc_n(&perm, n));
    IDET_TRY(ws.alloc_n(&md, 1));
    IDET_TRY(ws.alloc_n(&dd, 1));
    uint32_t p = 0;
    ModP mh{};
    for (int tries = 0;; ++tries) {
        if (tries == 6) return IDET_ERR_SINGULAR;
        p = random_prime31(g);
        mh = make_mod(p);
        IDET_CUDA_TRY(cudaMemcpyAsync(md, &mh, sizeof(ModP), cudaMemcpyHostToDevice, s));
        IDET_TRY(launch_reduce_mp(J.mag, J.sgn, n, J.L, md, 1, R, s));
        IDET_TRY(lu_factor_batched(R, n, md, &mh, 1, true, J.nb, perm, dd, IDET_PATH_AUTO, ws));
        uint32_t det = 0;
        IDET_CUDA_TRY(cudaMemcpyAsync(&det, dd, 4, cudaMemcpyDeviceToHost, s));
        IDET_CUDA_TRY(cudaStreamSynchronize(s));
        if (det != 0) break;
    }
    int32_t *Ysc = nullptr;
    IDET_TRY(ws.alloc_n(&C, (size_t)n * n));
    IDET_TRY(ws.alloc_n(&Ysc, (size_t)n * n));
    IDET_TRY(lu_inverse(R, perm, n, mh, md, true, J.nb, Ysc, C, n, ws));
    J.st.ms_inverse += tinv.stop();
    J.st.inverse_macs += (4.0 / 3.0) * (double)n * n * n;
    // A as signed base-2^15 digit planes
    const int T = (int)((abits + 1 + 14) / 15) + 1;
    const int64_t ldp = (n + 7) / 8 * 8;
    int16_t *planes = nullptr;
    IDET_TRY(ws.alloc_n(&planes, (size_t)T * n * ldp));
    IDET_TRY(launch_mp_planes(J.mag, J.sgn, n, J.L, T, ldp, planes, s));
    // b (Alg. 4.1 range S) and the projection u
    SplitMix gb(J.o.seed ^ 0xb5ull);
    const double l2S = rhs_range_log2(n, J.log2H);
    const uint64_t S = (uint64_t)std::exp2(std::floor(l2S));
    const double lp = std::log2((double)p);
    const double log2n = std::log2((double)n);
    // |r - A x| < |r| + n 2^abits p / 2 and |r| < n 2^abits + |b|: digits
    // 0..len-2 of 15 bits and a signed top digit below 2^14
    const int lv = (int)std::ceil(log2n) + (int)abits + 34;
    const int len = std::max(6, (lv + 1 - 14 + 14) / 15 + 2);
    std::vector<int32_t> rdh((size_t)n * len), rmh(n), uh(n);
    double u1 = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t b = (int64_t)(gb.below(S)) - (int64_t)(S / 2);
        for (int k = 0; k < len; ++k) {
            const int sh = std::min(15 * k, 63);
            int64_t d = b >> sh;
            rdh[(size_t)i * len + k] = (int32_t)(k < len - 1 ? (d & 0x7fff) : d);
        }
        int64_t bm = b % (int64_t)p;
        if (bm > (int64_t)(p - 1) / 2) bm -= p;
        if (bm < -(int64_t)(p - 1) / 2) bm += p;
        rmh[i] = (int32_t)bm;
    }
    for (int64_t i = 0; i < n; ++i) {
        uh[i] = (int32_t)(gb.next() & 0xffff);
        u1 += uh[i];
    }
    const double log2b = std::log2((double)S);
    const int gu = (int)std::ceil(std::log2(u1 + 1) / lp);
    int32_t *rd = nullptr, *rm = nullptr, *ud = nullptr, *x = nullptr, *info = nullptr;
    IDET_TRY(ws.alloc_n(&rd, (size_t)n * len));
    IDET_TRY(ws.alloc_n(&rm, n));
    IDET_TRY(ws.alloc_n(&ud, n));
    IDET_TRY(ws.alloc_n(&x, n));
    IDET_TRY(ws.alloc_n(&info, 4));
    IDET_CUDA_TRY(cudaMemcpyAsync(rd, rdh.data(), 4 * rdh.size(), cudaMemcpyHostToDevice, s));
    IDET_CUDA_TRY(cudaMemcpyAsync(rm, rmh.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, s));
    IDET_CUDA_TRY(cudaMemcpyAsync(ud, uh.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, s));
    IDET_CUDA_TRY(cudaMemsetAsync(info, 0, 16, s));
    // the static length (Hadamard bounds) caps the lift
    double lc = 0, lcmin = INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        lc += J.colsq[i];
        lcmin = std::min(lcmin, J.colsq[i]);
    }
    const double log2N = std::log2(u1 + 1) + log2b + 0.5 * log2n + lc - lcmin;
    const int64_t m_static = (int64_t)std::ceil((log2N + 1) / lp) +
                             (int64_t)std::ceil((J.log2H + 1) / lp) + 2;
    const int m_cap = (int)std::min<int64_t>(m_static, 1 << 14);
    int mcap = 64;
    int32_t *digits = nullptr;
    int64_t *z = nullptr;
    IDET_TRY(ws.alloc_n(&digits, (size_t)mcap * n));
    IDET_TRY(ws.alloc_n(&z, mcap));
    IDET_CUDA_TRY(cudaMemsetAsync(z, 0, 8 * (size_t)mcap, s));
    MpLiftArgs a{};
    a.C = C;
    a.ldc = n;
    a.n = n;
    a.planes = planes;
    a.T = T;
    a.ldp = ldp;
    a.u = ud;
    a.x = x;
    a.rm = rm;
    a.rd = rd;
    a.len = len;
    a.info = info;
    a.mod = mh;
    a.pinv15 = (uint32_t)(inv_mod_2_64(p) & 0x7fff);
    uint32_t *den = nullptr;
    int32_t *rinfo = nullptr, *flags = nullptr;
    IDET_TRY(ws.alloc_n(&rinfo, 4));
    IDET_TRY(ws.alloc_n(&flags, n));
    std::vector<int32_t> hflags(n);
    int it = 0, next_check = 16;
    bool ok = false;
    double kms = 0;
    while (!ok && it < m_cap) {
        const int target = std::min(next_check, m_cap);
        if (target > mcap) {
            int ncap = mcap;
            while (ncap < target) ncap *= 2;
            int32_t *nd = nullptr;
            int64_t *nz = nullptr;
            IDET_TRY(ws.alloc_n(&nd, (size_t)ncap * n));
            IDET_TRY(ws.alloc_n(&nz, ncap));
            IDET_CUDA_TRY(cudaMemcpyAsync(nd, digits, 4 * (size_t)it * n, cudaMemcpyDeviceToDevice, s));
            IDET_CUDA_TRY(cudaMemsetAsync(nz, 0, 8 * (size_t)ncap, s));
            IDET_CUDA_TRY(cudaMemcpyAsync(nz, z, 8 * (size_t)it, cudaMemcpyDeviceToDevice, s));
            digits = nd;
            z = nz;
            mcap = ncap;
        }
        a.digits = digits;
        a.z = z;
        Timer tk(s);
        for (; it < target; ++it) IDET_TRY(launch_mp_step(a, it, s));
        kms += tk.stop();
        next_check = it + std::max(8, it / 4);
        // checkpoint: balanced bounds
        const int h = (it - 2 - gu) / 2;
        if (h < 1) continue;
        const bool cert = log2n + abits + h * lp + 2 < it * lp - 1 && h * lp + log2b + 2 < it * lp - 1;
        if (!cert) continue;
        const int hN = it - 2 - h, den_cap = h + 2;
        IDET_TRY(ws.alloc_n(&den, den_cap));
        Timer trr(s);
        IDET_TRY(launch_ratrecon(z, it, p, hN, h, den, den_cap, rinfo, ws));
        int32_t hi[2] = {0, 0};
        IDET_CUDA_TRY(cudaMemcpyAsync(hi, rinfo, 8, cudaMemcpyDeviceToHost, s));
        IDET_CUDA_TRY(cudaStreamSynchronize(s));
        if (hi[0] != 0) {
            J.st.ms_rr += trr.stop();
            continue;
        }
        IDET_TRY(launch_lif_check(digits, n, it, den, hi[1], p, h, flags, s));
        IDET_CUDA_TRY(cudaMemcpyAsync(hflags.data(), flags, 4 * (size_t)n, cudaMemcpyDeviceToHost, s));
        IDET_CUDA_TRY(cudaStreamSynchronize(s));
        J.st.ms_rr += trr.stop();
        bool all = true;
        for (int64_t j = 0; j < n && all; ++j) all = hflags[j] == 0;
        if (!all) continue;
        out.den.resize(hi[1]);
        IDET_CUDA_TRY(cudaMemcpyAsync(out.den.data(), den, 4 * (size_t)hi[1], cudaMemcpyDeviceToHost, s));
        IDET_CUDA_TRY(cudaStreamSynchronize(s));
        // s~_n divides det A and p does not: a denominator divisible by p is
        // not the reduced one
        ok = out.den[0] != 0;
    }
    int32_t hinfo = 0;
    IDET_CUDA_TRY(cudaMemcpyAsync(&hinfo, info, 4, cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaStreamSynchronize(s));
    if (hinfo != 0) {
        set_last_error("multi-word lift: residual out of range");
        return IDET_ERR_INTERNAL;
    }
    J.st.ms_lift_kernel += kms;
    J.st.lift_bytes += (double)it * ((double)T * 2.0 + 4.0) * (double)n * (double)n;
    out.p = p;
    out.m = it;
    if (!ok) out.den.clear();
    return IDET_OK;
}

}  // namespace idet

using namespace idet;

// ---------------------------------------------------------------------------
// C ABI

extern "C" {

void idet_default_opts(idet_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->log2_epsilon = -64.0;
    o->seed = 0x1de7u;
    o->certify = 0;
    o->update_path = IDET_PATH_AUTO;
    o->nb = 0;
    o->wave = 0;
    o->lif = 1;
}

const char *idet_last_error(void) { return g_err; }

void idet_set_allocator(idet_alloc_fn a, idet_free_fn f, void *ctx) {
    g_alloc = a;
    g_free = f;
    g_actx = ctx;
}

uint64_t idet_launch_count(void) { return g_launches; }

int idet_det_mod_primes(const int64_t *A, int64_t n, int64_t lda, int32_t on_device,
                        const uint32_t *primes, int32_t nprimes, const idet_opts *opts,
                        void *stream, uint32_t *det_mod) {
    if (n < 0 || n > IDET_MAX_ORDER || lda < n || (n > 0 && !A) || nprimes < 0 ||
        (nprimes > 0 && (!primes || !det_mod))) {
        set_last_error("invalid argument");
        return IDET_ERR_ARG;
    }
    if (nprimes == 0) return IDET_OK;
    bool wide = primes[0] > (1u << 30);
    for (int i = 0; i < nprimes; ++i) {
        uint32_t p = primes[i];
        bool w = p > (1u << 30);
        bool ok = w ? (p < (1u << 31) && is_prime32(p)) : (p > kLo21 && p < kHi21 && is_prime32(p));
        if (!ok || w != wide) {
            set_last_error("primes must be odd primes of one class: (2^20, 2^21) or (2^30, 2^31)");
            return IDET_ERR_ARG;
        }
    }
    if (n == 0) {
        for (int i = 0; i < nprimes; ++i) det_mod[i] = 1;
        return IDET_OK;
    }
    idet_opts o;
    idet_default_opts(&o);
    if (opts) o = *opts;
    cudaStream_t s = (cudaStream_t)stream;
    Workspace ws(s);
    DevMatrix M;
    IDET_TRY(stage_matrix(A, n, lda, on_device, ws, M));
    double *rowsq = nullptr;
    unsigned long long *amax = nullptr, hmax = 0;
    IDET_TRY(ws.alloc_n(&rowsq, n));
    IDET_TRY(ws.alloc_n(&amax, 1));
    IDET_TRY(launch_row_stats(M.A, n, n, rowsq, amax, s));
    IDET_CUDA_TRY(cudaMemcpyAsync(&hmax, amax, 8, cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaStreamSynchronize(s));
    if (!entry_range(hmax, &hmax)) {
        set_last_error("entries must lie in [-2^31, 2^31 - 1]");
        return IDET_ERR_ARG;
    }
    const int W = nprimes;
    std::vector<ModP> mh(W);
    for (int i = 0; i < W; ++i) mh[i] = make_mod(primes[i]);
    ModP *md = nullptr;
    int32_t *R = nullptr;
    uint32_t *dd = nullptr;
    IDET_TRY(ws.alloc_n(&md, W));
    IDET_TRY(ws.alloc_n(&R, (size_t)W * n * n));
    IDET_TRY(ws.alloc_n(&dd, W));
    IDET_CUDA_TRY(cudaMemcpyAsync(md, mh.data(), sizeof(ModP) * W, cudaMemcpyHostToDevice, s));
    IDET_TRY(launch_reduce(M.A, n, n, md, W, R, s));
    IDET_TRY(lu_factor_batched(R, n, md, mh.data(), W, wide, o.nb, nullptr, dd, o.update_path, ws));
    IDET_CUDA_TRY(cudaMemcpyAsync(det_mod, dd, 4 * (size_t)W, cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaStreamSynchronize(s));
    return IDET_OK;
}

int idet_lu_mod_prime(const int64_t *A, int64_t n, int64_t lda, int32_t on_device, uint32_t p,
                      const idet_opts *opts, void *stream, uint32_t *lu, int32_t *perm) {
    if (n <= 0 || n > IDET_MAX_ORDER || lda < n || !A || !lu || !perm) {
        set_last_error("invalid argument");
        return IDET_ERR_ARG;
    }
    bool wide = p > (1u << 30);
    if (!(wide ? (p < (1u << 31) && is_prime32(p)) : (p > kLo21 && p < kHi21 && is_prime32(p)))) {
        set_last_error("p must be a prime in (2^20, 2^21) or (2^30, 2^31)");
        return IDET_ERR_ARG;
    }
    idet_opts o;
    idet_default_opts(&o);
    if (opts) o = *opts;
    cudaStream_t s = (cudaStream_t)stream;
    Workspace ws(s);
    DevMatrix M;
    IDET_TRY(stage_matrix(A, n, lda, on_device, ws, M));
    ModP mh = make_mod(p);
    ModP *md = nullptr;
    int32_t *R = nullptr, *pm = nullptr;
    uint32_t *dd = nullptr;
    IDET_TRY(ws.alloc_n(&md, 1));
    IDET_TRY(ws.alloc_n(&R, (size_t)n * n));
    IDET_TRY(ws.alloc_n(&pm, n));
    IDET_TRY(ws.alloc_n(&dd, 1));
    IDET_CUDA_TRY(cudaMemcpyAsync(md, &mh, sizeof(ModP), cudaMemcpyHostToDevice, s));
    IDET_TRY(launch_reduce(M.A, n, n, md, 1, R, s));
    IDET_TRY(lu_factor_batched(R, n, md, &mh, 1, wide, o.nb, pm, dd, o.update_path, ws));
    std::vector<int32_t> h((size_t)n * n);
    uint32_t det = 0;
    IDET_CUDA_TRY(cudaMemcpyAsync(h.data(), R, 4 * h.size(), cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaMemcpyAsync(perm, pm, 4 * (size_t)n, cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaMemcpyAsync(&det, dd, 4, cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaStreamSynchronize(s));
    for (size_t i = 0; i < h.size(); ++i) lu[i] = h[i] < 0 ? (uint32_t)(h[i] + (int64_t)p) : (uint32_t)h[i];
    return det == 0 ? IDET_ERR_SINGULAR : IDET_OK;
}

// The Dixon iteration for nrhs (1 or 2) right-hand sides B[k] (rows of B)
// in one lift: digits [k][i][j], residuals [k][j] (host arrays).
static int dixon_common(const int64_t *A, int64_t n, int64_t lda, const int64_t *B, int nrhs,
                        uint32_t p, int32_t m, int32_t on_device, void *stream, int32_t *digits,
                        int64_t *residual, idet_stats *stats) {
    if (n <= 0 || n > IDET_MAX_ORDER || lda < n || !A || !B || m < 0 || (m > 0 && !digits) ||
        !residual || (nrhs != 1 && nrhs != 2) ||
        !(p > (1u << 30) && p < (1u << 31) && is_prime32(p))) {
        set_last_error("invalid argument");
        return IDET_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    Workspace ws(s);
    DevMatrix M;
    IDET_TRY(stage_matrix(A, n, lda, on_device, ws, M));
    int64_t *bd = nullptr;
    IDET_TRY(ws.alloc_n(&bd, (size_t)nrhs * n));
    IDET_CUDA_TRY(cudaMemcpyAsync(bd, B, 8 * (size_t)nrhs * n,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    std::vector<int64_t> bh((size_t)nrhs * n);
    IDET_CUDA_TRY(cudaMemcpyAsync(bh.data(), bd, 8 * bh.size(), cudaMemcpyDeviceToHost, s));
    int32_t *Cinv = nullptr, *dig = nullptr;
    int64_t ldl = 0, *r = nullptr;
    double *rowsq = nullptr;
    unsigned long long *d_amax = nullptr, hmax = 0;
    IDET_TRY(ws.alloc_n(&rowsq, n));
    IDET_TRY(ws.alloc_n(&d_amax, 1));
    IDET_TRY(launch_row_stats(M.A, n, n, rowsq, d_amax, s));
    IDET_CUDA_TRY(cudaMemcpyAsync(&hmax, d_amax, 8, cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaStreamSynchronize(s));
    if (!entry_range(hmax, &hmax)) {
        set_last_error("entries must lie in [-2^31, 2^31 - 1]");
        return IDET_ERR_ARG;
    }
    for (int64_t v : bh)
        if (v >= (1ll << 62) || v <= -(1ll << 62)) {
            set_last_error("right-hand side entries must satisfy |b_i| < 2^62");
            return IDET_ERR_ARG;
        }
    void *Anar = nullptr;
    int abytes = 4;
    IDET_TRY(make_Anar(M, hmax, ws, &Anar, &abytes, &ldl));
    IDET_TRY(ws.alloc_n(&Cinv, (size_t)n * ldl));
    IDET_TRY(inverse_mod_prime(M, p, 32, ws, Cinv, ldl));
    IDET_TRY(ws.alloc_n(&r, (size_t)nrhs * n));
    IDET_TRY(ws.alloc_n(&dig, (size_t)nrhs * m * n + 1));
    LiftArgs a{};
    a.Cinv = Cinv;
    a.b = bd;
    a.n = n;
    a.m = m;
    a.mod = make_mod(p);
    a.pinv = inv_mod_2_64(p);
    a.digits = dig;
    a.r = r;
    a.amax = hmax;
    a.nrhs = nrhs;
    if (nrhs == 2) {
        a.b2 = bd + n;
        a.digits2 = dig + (size_t)m * n;
        a.r2 = r + n;
    }
    int to = 0;
    float ms = 0;
    LiftInfo li{};
    IDET_TRY(launch_lift(a, Anar, abytes, ldl, ws, &to, &ms, &li));
    if (m > 0)
        IDET_CUDA_TRY(cudaMemcpyAsync(digits, dig, 4 * (size_t)nrhs * m * n,
                                      cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaMemcpyAsync(residual, r, 8 * (size_t)nrhs * n, cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaStreamSynchronize(s));
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->lift_iters = m;
        stats->lift_path = li.path;
        stats->ms_lift_kernel = li.ms_steps;
        stats->ms_lift_setup = li.ms_setup;
        stats->lift_bytes = li.bytes;
        stats->lift_timed_out = to;
    }
    return IDET_OK;
}

int idet_dixon_digits(const int64_t *A, int64_t n, int64_t lda, const int64_t *b, uint32_t p,
                      int32_t m, int32_t on_device, void *stream, int32_t *digits,
                      int64_t *residual) {
    return dixon_common(A, n, lda, b, 1, p, m, on_device, stream, digits, residual, nullptr);
}

int idet_dixon_digits_block(const int64_t *A, int64_t n, int64_t lda, const int64_t *B,
                            int32_t nrhs, uint32_t p, int32_t m, int32_t on_device, void *stream,
                            int32_t *digits, int64_t *residual, idet_stats *stats) {
    return dixon_common(A, n, lda, B, nrhs, p, m, on_device, stream, digits, residual, stats);
}

int idet_crt_symmetric(const uint32_t *residues, const uint32_t *primes, int32_t count,
                       void *stream, idet_int *r, int32_t *trailing) {
    if (count < 0 || (count > 0 && (!residues || !primes)) || !r) {
        set_last_error("invalid argument");
        return IDET_ERR_ARG;
    }
    for (int i = 0; i < count; ++i)
        if (!(primes[i] > 2 && primes[i] < (1u << 31) && is_prime32(primes[i]))) {
            set_last_error("primes must be odd primes below 2^31");
            return IDET_ERR_ARG;
        }
    {
        // Garner's method needs pairwise coprime moduli: a repeated prime
        // has no inverse modulo the product of the others
        std::vector<uint32_t> srt(primes, primes + count);
        std::sort(srt.begin(), srt.end());
        if (std::adjacent_find(srt.begin(), srt.end()) != srt.end()) {
            set_last_error("primes must be pairwise distinct");
            return IDET_ERR_ARG;
        }
    }
    if (count == 0) {
        if (trailing) *trailing = 0;
        return write_int(r, 0, nullptr, 0);
    }
    cudaStream_t s = (cudaStream_t)stream;
    Workspace ws(s);
    idet_opts o;
    idet_default_opts(&o);
    DevMatrix M;
    DetJob J(M, ws, o);
    std::vector<uint32_t> prs(primes, primes + count), res(residues, residues + count);
    for (int i = 0; i < count; ++i) res[i] %= prs[i];
    std::vector<int32_t> dig;
    IDET_TRY(J.cra_digits(prs, res, dig));
    if (trailing) {
        int k = 0;
        for (int t = count - 1; t > 0 && dig[t] == 0; --t) ++k;
        *trailing = k;
    }
    return J.assemble(prs, dig, count, nullptr, 0, r);
}

int idet_cra_early_termination(const uint32_t *residues, const uint32_t *primes, int32_t count,
                               double log2_H, double log2_epsilon, double log2_l,
                               double pool_size, int32_t certify, void *stream, idet_int *r,
                               int32_t *stop_index, int32_t *reason) {
    if (count < 0 || (count > 0 && (!residues || !primes)) || !r || !stop_index || !reason ||
        !(log2_l > 0) || !(pool_size >= 1) || std::isnan(log2_H) || !(log2_epsilon < 0)) {
        set_last_error("invalid argument");
        return IDET_ERR_ARG;
    }
    for (int i = 0; i < count; ++i)
        if (!(primes[i] > 2 && primes[i] < (1u << 31) && is_prime32(primes[i]))) {
            set_last_error("primes must be odd primes below 2^31");
            return IDET_ERR_ARG;
        }
    {
        std::vector<uint32_t> srt(primes, primes + count);
        std::sort(srt.begin(), srt.end());
        if (std::adjacent_find(srt.begin(), srt.end()) != srt.end()) {
            set_last_error("primes must be pairwise distinct");
            return IDET_ERR_ARG;
        }
    }
    *stop_index = -1;
    *reason = 0;
    if (count == 0) return write_int(r, 0, nullptr, 0);
    cudaStream_t s = (cudaStream_t)stream;
    Workspace ws(s);
    idet_opts o;
    idet_default_opts(&o);
    DevMatrix M;
    DetJob J(M, ws, o);
    std::vector<uint32_t> prs(primes, primes + count), res(residues, residues + count);
    for (int i = 0; i < count; ++i) res[i] %= prs[i];
    std::vector<int32_t> dig;
    IDET_TRY(J.cra_digits(prs, res, dig));
    int why = 0;
    const int stop = CraScan::scan(dig, prs, log2_H, log2_epsilon, log2_l, pool_size,
                                   certify != 0, &why);
    *stop_index = stop;
    *reason = why;
    return J.assemble(prs, dig, stop >= 0 ? stop + 1 : count, nullptr, 0, r);
}

static int lif_common(DetJob &J, const int64_t *b_dev, const std::vector<int64_t> &bh,
                      LiftResult &lr);
static int introspective2(DetJob &J, int wave, idet_int *det);

int idet_int_det(const int64_t *A, int64_t n, int64_t lda, int32_t on_device,
                 const idet_opts *opts, void *stream, idet_int *det, idet_stats *stats) {
    if (n < 0 || n > IDET_MAX_ORDER || lda < n || (n > 0 && !A) || !det) {
        set_last_error("invalid argument");
        return IDET_ERR_ARG;
    }
    const unsigned long long launches0 = g_launches;
    if (n == 0) {
        uint32_t one = 1;
        return write_int(det, 1, &one, 1);
    }
    idet_opts o;
    idet_default_opts(&o);
    if (opts) o = *opts;
    cudaStream_t s = (cudaStream_t)stream;
    Workspace ws(s);
    Timer total(s);
    DevMatrix M;
    IDET_TRY(stage_matrix(A, n, lda, on_device, ws, M));
    if (o.prime_bits != 0 && o.prime_bits != 21 && o.prime_bits != 31) {
        set_last_error("prime_bits must be 0, 21 or 31");
        return IDET_ERR_ARG;
    }
    DetJob J(M, ws, o, o.prime_bits == 31 ? 31 : 21);
    IDET_TRY(J.stats());
    auto finish = [&](int rc) {
        J.st.ms_total = total.stop();
        J.st.launches = g_launches - launches0;
        if (stats) *stats = J.st;
        return rc;
    };
    if (J.log2H == -INFINITY || J.amax == 0) {  // a zero row: det = 0
        J.st.et_stop = 2;
        return finish(write_int(det, 0, nullptr, 0));
    }
    const bool certify = o.certify != 0;
    const int k0 = k_default(o.log2_epsilon, J.draw.pool(), J.log2H, J.draw.log2l());
    const int wave = default_wave(o, n, J.draw.bits, k0);

    // Alg. 2.1 on det(A): the first k0 primes (Alg. 4.1 lines 1-4), or all
    // the way in CRA-only / certified mode. lif = 2 (solve first, the order
    // of Abbott, Bronstein and Mulders that Fig. 2 compares against) skips
    // it and reconstructs det(A)/K to the bound 2H/K after the solve.
    const bool solve_first = o.lif == 2 && !certify;
    // Section 4 lets the modular LUs run behind the solves, and the random
    // systems be solved together or one after another: the LU and inverse mod
    // the lifting prime do not depend on the CRA, so they run on a second
    // stream, from a second host thread, while the first CRA wave is factored
    // (its workspace from the stream-ordered pool, as the serving workers').
    std::thread inv_thread;
    int inv_rc = IDET_OK;
    std::string inv_err;
    float inv_ms = 0;
    int32_t *inv_C = nullptr;
    uint32_t inv_p = 0;
    // From n = 500 on (21-bit CRA primes, one solve) the order is
    // speculative instead: the inverse mod the lifting prime and the lift
    // run first, and the first CRA wave is factored on a second stream while
    // the rational reconstruction -- one CTA, about a fifth of the solve at
    // n = 4000 -- runs beside it (Section 4 lets the LUs run behind the
    // solves). The wave's early-termination verdict still decides
    // first: if it stops, its determinant is returned and K is not used. A
    // lifting prime that divides det(A) (probably det(A) = 0) falls back to
    // the wave-first order below.
    bool spec = o.lif == 1 && !certify && o.i_max < 2 && J.draw.bits != 31 && n >= 500 &&
                !getenv("IDET_ET_FIRST");
    if (spec) {
        IDET_TRY(make_Anar(J.M, J.amax, ws, &J.Anar, &J.abytes, &J.ldl));
        int32_t *Cinv = nullptr;
        IDET_TRY(ws.alloc_n(&Cinv, (size_t)n * J.ldl));
        SplitMix g(J.o.seed ^ 0x11f7ull);
        const uint32_t p = random_prime31(g);
        Timer tinv(s);
        const int rc = inverse_mod_prime(J.M, p, J.nb, ws, Cinv, J.ldl);
        J.st.ms_inverse += tinv.stop();
        if (rc == IDET_OK) {
            J.pre_Cinv = Cinv;
            J.pre_p = p;
            J.st.inverse_macs += (4.0 / 3.0) * (double)n * n * n;
        } else if (rc == IDET_ERR_SINGULAR) {
            spec = false;
        } else {
            return finish(rc);
        }
    }
    // Otherwise, from n = 1500 on, the LU and inverse mod the lifting prime
    // run on a second stream beside the first wave.
    const bool overlap = !spec && o.lif == 1 && !certify && o.i_max < 2 && J.draw.bits != 31 &&
                         n >= 1500 && !getenv("IDET_SERIAL_INVERSE");
    if (overlap && !solve_first) {
        IDET_TRY(make_Anar(J.M, J.amax, ws, &J.Anar, &J.abytes, &J.ldl));
        IDET_TRY(ws.alloc_n(&inv_C, (size_t)n * J.ldl));
        IDET_CUDA_TRY(cudaStreamSynchronize(s));  // A staged, Anar formed
        int dev = 0;
        IDET_CUDA_TRY(cudaGetDevice(&dev));
        inv_thread = std::thread([&J, &inv_rc, &inv_err, &inv_ms, &inv_p, inv_C, dev] {
            t_native_alloc = true;
            if (cudaSetDevice(dev) != cudaSuccess) {
                inv_rc = IDET_ERR_CUDA;
                inv_err = "lift inverse: cudaSetDevice failed";
                return;
            }
            cudaStream_t s2 = nullptr;
            if (cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking) != cudaSuccess) {
                inv_rc = IDET_ERR_CUDA;
                inv_err = "lift inverse: cudaStreamCreate failed";
                return;
            }
            {
                Workspace ws2(s2);
                Timer t(s2);
                SplitMix g(J.o.seed ^ 0x11f7ull);
                int rc = IDET_ERR_SINGULAR;
                for (int tries = 0; tries < 6 && rc == IDET_ERR_SINGULAR; ++tries) {
                    inv_p = random_prime31(g);
                    rc = inverse_mod_prime(J.M, inv_p, J.nb, ws2, inv_C, J.ldl);
                }
                inv_ms = (float)t.stop();
                inv_rc = rc;
                if (rc != IDET_OK) inv_err = idet_last_error();
                cudaStreamSynchronize(s2);
            }
            cudaStreamSynchronize(s2);
            cudaStreamDestroy(s2);
        });
    }
    auto join_inverse = [&]() -> int {
        if (!inv_thread.joinable()) return IDET_OK;
        inv_thread.join();
        J.st.ms_inverse += inv_ms;
        if (inv_rc == IDET_OK) {
            J.pre_Cinv = inv_C;
            J.pre_p = inv_p;
            J.st.inverse_macs += (4.0 / 3.0) * (double)n * n * n;
            return IDET_OK;
        }
        if (inv_rc == IDET_ERR_SINGULAR) return IDET_OK;  // the solve reports it again
        set_last_error("%s", inv_err.c_str());
        return inv_rc;
    };
    bool spec_done = false;
    if (spec) {
        J.during_rr = [&]() -> int {
            cudaStream_t s2 = nullptr;
            IDET_CUDA_TRY(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
            int rc;
            const bool native0 = t_native_alloc;
            t_native_alloc = true;  // stream-ordered allocations on s2
            {
                Workspace ws2(s2);
                t_native_alloc = native0;
                DetJob J2(J.M, ws2, J.o, J.draw.bits);
                J2.log2H = J.log2H;
                J2.amax = J.amax;
                J2.rowsq = J.rowsq;
                J2.colsq = J.colsq;
                J2.nb = J.nb;
                J2.st.log2_H = J.st.log2_H;
                t_reserve_sms = 1;
                rc = det_first(J2, k0, wave, false, det, &spec_done);
                t_reserve_sms = 0;
                cudaStreamSynchronize(s2);
                // the wave's residues, and the prime stream, continue in J
                J.primes = J2.primes;
                J.dets = J2.dets;
                J.draw = J2.draw;
                J.st.ms_lu += J2.st.ms_lu;
                J.st.ms_cra += J2.st.ms_cra;
                J.st.primes_used += J2.st.primes_used;
                J.st.lu_macs += J2.st.lu_macs;
                if (spec_done) {
                    J.st.et_stop = J2.st.et_stop;
                    J.st.primes_in_cra = J2.st.primes_in_cra;
                }
            }
            cudaStreamDestroy(s2);
            return rc;
        };
    } else if (!solve_first) {
        bool done = false;
        const int rc0 = det_first(J, k0, wave, certify || !o.lif, det, &done);
        const int rcj = join_inverse();
        if (rc0 != IDET_OK || done) return finish(rc0);
        if (rcj != IDET_OK) return finish(rcj);
    }

    // Alg. 4.1 with i_max = 2: two solves and the extended bonus
    if (o.i_max >= 2 && !solve_first) return finish(introspective2(J, wave, det));

    // Section 2.2 / Alg. 4.1 with i_max = 1: one solve gives K = s~_n.
    const int64_t *bdev = nullptr;
    std::vector<int64_t> bh(n);
    {
        SplitMix g(o.seed ^ 0xb5ull);
        const double l2S = rhs_range_log2(n, J.log2H);
        const uint64_t S = (uint64_t)std::exp2(std::floor(l2S));
        for (int64_t i = 0; i < n; ++i) bh[i] = (int64_t)(g.below(S)) - (int64_t)(S / 2);
        int64_t *bd = nullptr;
        IDET_TRY(ws.alloc_n(&bd, n));
        IDET_CUDA_TRY(cudaMemcpyAsync(bd, bh.data(), 8 * (size_t)n, cudaMemcpyHostToDevice, s));
        bdev = bd;
    }
    LiftResult lr;
    Timer tl(s);
    int rc = lif_common(J, bdev, bh, lr);
    J.st.ms_lift += tl.stop();
    J.st.lift_timed_out = lr.timed_out;
    if (spec) {
        J.during_rr = nullptr;
        if (J.during_rr_ran) {
            if (J.during_rr_rc != IDET_OK) return finish(J.during_rr_rc);
            if (spec_done) return finish(IDET_OK);
        } else {
            // the solve ended before its reconstruction: the wave now
            bool done = false;
            const int rc0 = det_first(J, k0, wave, false, det, &done);
            if (rc0 != IDET_OK || done) return finish(rc0);
        }
    }
    if (rc != IDET_OK && rc != IDET_ERR_SINGULAR) return finish(rc);
    J.st.lift_iters = lr.m;
    J.st.lift_timed_out = lr.timed_out;

    const bool K = rc == IDET_OK && lr.has_den;
    J.st.log2_K = K ? (int)std::floor(lr.log2K) : 0;
    return finish(det_over_K(J, K ? lr.Kbin : nullptr, K ? lr.Klen : 0, K ? lr.log2K : 0, wave,
                             det, solve_first));
}

int idet_int_det_mp(const uint32_t *A_limbs, const int8_t *A_sign, int64_t n, int32_t L,
                    int32_t on_device, const idet_opts *opts, void *stream, idet_int *det,
                    idet_stats *stats) {
    if (n < 0 || n > IDET_MAX_ORDER || L < 1 || L > 64 || (n > 0 && (!A_limbs || !A_sign)) ||
        !det) {
        set_last_error("invalid argument");
        return IDET_ERR_ARG;
    }
    const unsigned long long launches0 = g_launches;
    if (n == 0) {
        uint32_t one = 1;
        return write_int(det, 1, &one, 1);
    }
    idet_opts o;
    idet_default_opts(&o);
    if (opts) o = *opts;
    if (o.prime_bits != 0 && o.prime_bits != 21 && o.prime_bits != 31) {
        set_last_error("prime_bits must be 0, 21 or 31");
        return IDET_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    Workspace ws(s);
    Timer total(s);
    const size_t nn = (size_t)n * n;
    uint32_t *mag = nullptr;
    int8_t *sgn = nullptr;
    IDET_TRY(ws.alloc_n(&mag, nn * L));
    IDET_TRY(ws.alloc_n(&sgn, nn));
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    IDET_CUDA_TRY(cudaMemcpyAsync(mag, A_limbs, 4 * nn * L, kind, s));
    IDET_CUDA_TRY(cudaMemcpyAsync(sgn, A_sign, nn, kind, s));
    DevMatrix M;
    M.n = n;
    DetJob J(M, ws, o, o.prime_bits == 21 ? 21 : 31);
    J.mag = mag;
    J.sgn = sgn;
    J.L = L;
    auto finish = [&](int rc) {
        J.st.ms_total = total.stop();
        J.st.launches = g_launches - launches0;
        if (stats) *stats = J.st;
        return rc;
    };
    // Hadamard bound from row and column norms (log domain); colsq holds
    // log2 of the column norms here
    double *E = nullptr, *rl = nullptr, *cl = nullptr;
    unsigned int *mb = nullptr, abits = 0;
    IDET_TRY(ws.alloc_n(&E, nn));
    IDET_TRY(ws.alloc_n(&rl, n));
    IDET_TRY(ws.alloc_n(&cl, n));
    IDET_TRY(ws.alloc_n(&mb, 1));
    IDET_TRY(launch_mp_stats(mag, sgn, n, L, E, rl, cl, mb, s));
    std::vector<double> rlh(n), clh(n);
    IDET_CUDA_TRY(cudaMemcpyAsync(rlh.data(), rl, 8 * (size_t)n, cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaMemcpyAsync(clh.data(), cl, 8 * (size_t)n, cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaMemcpyAsync(&abits, mb, 4, cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaStreamSynchronize(s));
    double hr = 0, hc = 0;
    for (int64_t i = 0; i < n; ++i) {
        hr += rlh[i];
        hc += clh[i];
    }
    if (hr == -INFINITY || hc == -INFINITY || abits == 0) {  // a zero row or column
        J.st.et_stop = 2;
        return finish(write_int(det, 0, nullptr, 0));
    }
    // margin for the rounding of the norms (upper bound kept)
    J.log2H = std::min(hr, hc) * (1 + 1e-12) + 1e-6 * n;
    J.st.log2_H = J.log2H;
    J.colsq = clh;
    const bool certify = o.certify != 0;
    const int k0 = k_default(o.log2_epsilon, J.draw.pool(), J.log2H, J.draw.log2l());
    const int wave = default_wave(o, n, J.draw.bits, k0);
    bool done = false;
    const int rc0 = det_first(J, k0, wave, certify || !o.lif, det, &done);
    if (rc0 != IDET_OK || done) return finish(rc0);
    MpLift lr;
    Timer tl(s);
    int rc = mp_lift(J, abits, lr);
    J.st.ms_lift += tl.stop();
    if (rc != IDET_OK && rc != IDET_ERR_SINGULAR) return finish(rc);
    J.st.lift_iters = lr.m;
    uint32_t *Kbin = nullptr;
    int Klen = 0;
    double log2K = 0;
    if (rc == IDET_OK && !lr.den.empty())
        IDET_TRY(den_to_binary(ws, lr.den, lr.p, &Kbin, &Klen, &log2K));
    J.st.log2_K = (int)std::floor(log2K);
    return finish(det_over_K(J, Kbin, Klen, log2K, wave, det));
}

static int lif_common(DetJob &J, const int64_t *b_dev, const std::vector<int64_t> &bh,
                      LiftResult &lr) {
    const int64_t n = J.M.n;
    // projection vector u, entries in [0, 2^16)
    SplitMix g(J.o.seed ^ 0x9a11ull);
    std::vector<int32_t> uh(n);
    double u1 = 0;
    for (int64_t i = 0; i < n; ++i) {
        uh[i] = (int32_t)(g.next() & 0xffff);
        u1 += uh[i];
    }
    int32_t *ud = nullptr;
    IDET_TRY(J.ws.alloc_n(&ud, n));
    IDET_CUDA_TRY(cudaMemcpyAsync(ud, uh.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, J.s));
    return solve_and_denominator(J, b_dev, bh, ud, std::log2(std::max(u1, 1.0)), lr);
}

// A positive integer given by dlen radix-p digits on the device, written to
// out as base-2^32 limbs.
static int radix_to_int(Workspace &ws, const uint32_t *D, int dlen, uint32_t p, idet_int *out) {
    cudaStream_t s = ws.stream();
    const int bcap = dlen + 2;
    uint32_t *Db = nullptr;
    int32_t *len = nullptr;
    IDET_TRY(ws.alloc_n(&Db, bcap));
    IDET_TRY(ws.alloc_n(&len, 1));
    IDET_TRY(launch_radix_to_binary(D, dlen, p, Db, bcap, len, s));
    int32_t bl = 0;
    IDET_CUDA_TRY(cudaMemcpyAsync(&bl, len, 4, cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<uint32_t> host(bl > 0 ? bl : 1);
    if (bl > 0)
        IDET_CUDA_TRY(cudaMemcpyAsync(host.data(), Db, 4 * (size_t)bl, cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaStreamSynchronize(s));
    return write_int(out, 1, host.data(), (uint32_t)bl);
}

// The exact lcm D of the denominators of the entries of x, from its lifting
// digits (m x n, balanced) and their projections z_i = u . x_i (Section 2.2,
// s~_n for one right-hand side): the denominator of u . x by rational
// reconstruction (numerator below p^hN, denominator below p^hD), then every
// entry whose D x_j is not an integer (numerator bound p^hNe) is
// reconstructed itself and D replaced by lcm(D, d_j). *Dout: device buffer of
// radix-p digits (workspace), *dlen its length.
static int lcm_of_denominators(const int32_t *dig, int64_t n, int m, uint32_t p, const int64_t *z,
                               int hN, int hNe, int hD, Workspace &ws, uint32_t **Dout,
                               int *dlen_out) {
    cudaStream_t s = ws.stream();
    const int dcap = hD + 4;
    uint32_t *D = nullptr, *Dn = nullptr, *dj = nullptr, *cof = nullptr;
    int32_t *info = nullptr, *flags = nullptr, *len = nullptr;
    int64_t *zj = nullptr;
    IDET_TRY(ws.alloc_n(&D, dcap));
    IDET_TRY(ws.alloc_n(&Dn, dcap));
    IDET_TRY(ws.alloc_n(&dj, dcap));
    IDET_TRY(ws.alloc_n(&cof, dcap));
    IDET_TRY(ws.alloc_n(&info, 4));
    IDET_TRY(ws.alloc_n(&len, 1));
    IDET_TRY(ws.alloc_n(&flags, n));
    IDET_TRY(ws.alloc_n(&zj, m));
    int32_t hi[2] = {0, 0};
    IDET_TRY(launch_ratrecon(z, m, p, hN, hD, D, dcap, info, ws));
    IDET_CUDA_TRY(cudaMemcpyAsync(hi, info, 8, cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaStreamSynchronize(s));
    if (hi[0] != 0) {
        set_last_error("rational reconstruction of the projection failed (code %d)", hi[0]);
        return IDET_ERR_INTERNAL;
    }
    int dlen = hi[1];
    // every entry integral under D?  else D <- lcm(D, den(x_j))
    std::vector<int32_t> fl(n);
    int64_t nflag_first = 0, nflag_last = 0;
    for (int round = 0;; ++round) {
        IDET_TRY(launch_lif_check(dig, n, m, D, dlen, p, hNe, flags, s));
        IDET_CUDA_TRY(cudaMemcpyAsync(fl.data(), flags, 4 * (size_t)n, cudaMemcpyDeviceToHost, s));
        IDET_CUDA_TRY(cudaStreamSynchronize(s));
        int64_t bad = -1, nflag = 0;
        for (int64_t j = 0; j < n; ++j)
            if (fl[j]) {
                if (bad < 0) bad = j;
                ++nflag;
            }
        if (round == 0) nflag_first = nflag;
        nflag_last = nflag;
        if (bad < 0) break;
        if (round >= 64) {
            set_last_error("largest invariant factor: too many denominator updates (%lld entries "
                           "flagged at first, %lld after %d updates; D has %d digits, m = %d, "
                           "h = %d)",
                           (long long)nflag_first, (long long)nflag_last, round, dlen, m, hNe);
            return IDET_ERR_INTERNAL;
        }
        // d_j = den(x_j) by reconstruction of X_j
        IDET_TRY(launch_gather_col(dig, n, m, bad, zj, s));
        IDET_TRY(launch_ratrecon(zj, m, p, hNe, hD, dj, dcap, info, ws));
        IDET_CUDA_TRY(cudaMemcpyAsync(hi, info, 8, cudaMemcpyDeviceToHost, s));
        IDET_CUDA_TRY(cudaStreamSynchronize(s));
        if (hi[0] != 0) {
            set_last_error("rational reconstruction of an entry failed (code %d)", hi[0]);
            return IDET_ERR_INTERNAL;
        }
        const int djlen = hi[1];
        // D / gcd(D, d_j): cofactor of d_j at the zero remainder of Euclid(D, d_j)
        std::vector<uint32_t> djh(djlen);
        IDET_CUDA_TRY(cudaMemcpyAsync(djh.data(), dj, 4 * (size_t)djlen, cudaMemcpyDeviceToHost, s));
        IDET_CUDA_TRY(cudaStreamSynchronize(s));
        std::vector<int64_t> djz(djh.begin(), djh.end());
        IDET_CUDA_TRY(cudaMemcpyAsync(zj, djz.data(), 8 * (size_t)djlen, cudaMemcpyHostToDevice, s));
        IDET_TRY(launch_ratrecon(zj, djlen, p, 0, dcap, cof, dcap, info, ws, D, dlen));
        IDET_CUDA_TRY(cudaMemcpyAsync(hi, info, 8, cudaMemcpyDeviceToHost, s));
        IDET_CUDA_TRY(cudaStreamSynchronize(s));
        if (hi[0] != 0) {
            set_last_error("gcd of denominators failed (code %d)", hi[0]);
            return IDET_ERR_INTERNAL;
        }
        IDET_TRY(launch_mul_radix(dj, djlen, cof, hi[1], p, Dn, dcap, len, s));
        int32_t nl = 0;
        IDET_CUDA_TRY(cudaMemcpyAsync(&nl, len, 4, cudaMemcpyDeviceToHost, s));
        IDET_CUDA_TRY(cudaStreamSynchronize(s));
        std::swap(D, Dn);
        dlen = nl;
    }
    *Dout = D;
    *dlen_out = dlen;
    return IDET_OK;
}

int idet_largest_invariant_factor(const int64_t *A, int64_t n, int64_t lda, const int64_t *b,
                                  int32_t on_device, const idet_opts *opts, void *stream,
                                  idet_int *sout) {
    if (n < 0 || n > IDET_MAX_ORDER || lda < n || (n > 0 && (!A || !b)) || !sout) {
        set_last_error("invalid argument");
        return IDET_ERR_ARG;
    }
    if (n == 0) {
        uint32_t one = 1;
        return write_int(sout, 1, &one, 1);
    }
    idet_opts o;
    idet_default_opts(&o);
    if (opts) o = *opts;
    cudaStream_t s = (cudaStream_t)stream;
    Workspace ws(s);
    DevMatrix M;
    IDET_TRY(stage_matrix(A, n, lda, on_device, ws, M));
    DetJob J(M, ws, o);
    IDET_TRY(J.stats());
    if (J.log2H == -INFINITY) {
        set_last_error("A is singular (zero row or column)");
        return IDET_ERR_SINGULAR;
    }
    std::vector<int64_t> bh(n);
    int64_t *bd = nullptr;
    IDET_TRY(ws.alloc_n(&bd, n));
    IDET_CUDA_TRY(cudaMemcpyAsync(bd, b, 8 * (size_t)n,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    IDET_CUDA_TRY(cudaMemcpyAsync(bh.data(), bd, 8 * (size_t)n, cudaMemcpyDeviceToHost, s));
    IDET_CUDA_TRY(cudaStreamSynchronize(s));
    for (int64_t i = 0; i < n; ++i)
        if (bh[i] >= (1ll << 62) || bh[i] <= -(1ll << 62)) {
            set_last_error("right-hand side entries must satisfy |b_i| < 2^62");
            return IDET_ERR_ARG;
        }
    // lift with the digits kept, and the projection u . x
    SplitMix g(o.seed ^ 0x9a11ull);
    std::vector<int32_t> uh(n);
    double u1 = 0;
    for (int64_t i = 0; i < n; ++i) {
        uh[i] = (int32_t)(g.next() & 0xffff);
        u1 += uh[i];
    }
    int32_t *ud = nullptr;
    IDET_TRY(ws.alloc_n(&ud, n));
    IDET_CUDA_TRY(cudaMemcpyAsync(ud, uh.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, s));
    IDET_TRY(make_Anar(J.M, J.amax, ws, &J.Anar, &J.abytes, &J.ldl));
    int32_t *Cinv = nullptr;
    IDET_TRY(ws.alloc_n(&Cinv, (size_t)n * J.ldl));
    SplitMix gp(o.seed ^ 0x11f7ull);
    uint32_t p = 0;
    int rc = IDET_ERR_SINGULAR;
    for (int tries = 0; tries < 6 && rc == IDET_ERR_SINGULAR; ++tries) {
        p = random_prime31(gp);
        rc = inverse_mod_prime(J.M, p, J.nb, ws, Cinv, J.ldl);
    }
    if (rc == IDET_ERR_SINGULAR) {
        set_last_error("A is singular (singular modulo 6 random 31-bit primes)");
        return rc;
    }
    IDET_TRY(rc);
    double bb = 1.0, lc = 0, lcmin = INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        bb += (double)bh[i] * (double)bh[i];
        double c = 0.5 * std::log2(std::max(J.colsq[i], 1.0));
        lc += c;
        lcmin = std::min(lcmin, c);
    }
    const double log2Ne = 0.5 * std::log2(bb * (1 + 1e-12)) + lc - lcmin;  // |N_j|
    const double log2N = log2Ne + std::log2(std::max(u1, 1.0));             // |u . N|
    const double lp = std::log2((double)p);
    const int hN = (int)std::ceil((log2N + 1) / lp);
    const int hNe = (int)std::ceil((log2Ne + 1) / lp);
    const int hD = (int)std::ceil((J.log2H + 1) / lp);
    const int m = hN + hD + 2;
    int32_t *dig = nullptr;
    int64_t *z = nullptr, *r = nullptr;
    IDET_TRY(ws.alloc_n(&dig, (size_t)m * n));
    IDET_TRY(ws.alloc_n(&z, m));
    IDET_TRY(ws.alloc_n(&r, n));
    LiftArgs la{};
    la.Cinv = Cinv;
    la.b = bd;
    la.u = ud;
    la.n = n;
    la.m = m;
    la.mod = make_mod(p);
    la.pinv = inv_mod_2_64(p);
    la.digits = dig;
    la.zproj = z;
    la.r = r;
    la.amax = J.amax;
    int to = 0;
    IDET_TRY(launch_lift(la, J.Anar, J.abytes, J.ldl, ws, &to));
    uint32_t *D = nullptr;
    int dlen = 0;
    IDET_TRY(lcm_of_denominators(dig, n, m, p, z, hN, hNe, hD, ws, &D, &dlen));
    return radix_to_int(ws, D, dlen, p, sout);
}

// K given by len radix-p digits on the device: base-2^32 limbs on the
// device and log2 K (as den_to_binary).
static int radix_dev_to_binary(Workspace &ws, const uint32_t *dig, int len, uint32_t p,
                               uint32_t **Kbin, int *Klen, double *log2K) {
    std::vector<uint32_t> h(len);
    IDET_CUDA_TRY(cudaMemcpyAsync(h.data(), dig, 4 * (size_t)len, cudaMemcpyDeviceToHost,
                                  ws.stream()));
    IDET_CUDA_TRY(cudaStreamSynchronize(ws.stream()));
    return den_to_binary(ws, h, p, Kbin, Klen, log2K);
}

// Alg. 4.1 with i_min = i_max = 2 (the second column of Table 1), after the
// first CRA on det(A) did not terminate. The two solves of the inner loop
// run as one block lift (Section 6: solvings grouped into a block
// iteration). i = 1: pi~_1 = s~ of x_1, K = pi~_1, and the CRA of det/K
// resumes for no longer than one solve takes: with the second
// solve already done by the block lift, the time is spent better on it, so
// the resume checks the residues at hand for early termination and factors
// no new primes. i = 2: s~ = lcm of the
// denominators of x_1 and x_2, pi~_2 = s~^2 / gcd(det(R N), s~^2) for a
// random 2 x n matrix R (Section 3.2), K = lcm(K, pi~_2), and the CRA of
// det/K resumes until it stops. (With i_max = i_min the printed loop never
// raises k_done, so its rounds of solves would repeat without end; one round
// is made, and the last line of the algorithm, a determinant method of better
// worst-case cost, is read as the CRA of det/K run to its stop.)
static int introspective2(DetJob &J, int wave, idet_int *det) {
    const int64_t n = J.M.n;
    Workspace &ws = J.ws;
    cudaStream_t s = J.s;
    const idet_opts &o = J.o;
    if (!J.Anar) IDET_TRY(make_Anar(J.M, J.amax, ws, &J.Anar, &J.abytes, &J.ldl));
    int32_t *Cinv = nullptr;
    IDET_TRY(ws.alloc_n(&Cinv, (size_t)n * J.ldl));
    uint32_t p = 0;
    Timer tinv(s);
    const int rc = lift_prime_inverse(J, Cinv, J.ldl, &p);
    J.st.ms_inverse += tinv.stop();
    if (rc == IDET_ERR_SINGULAR) return det_over_K(J, nullptr, 0, 0, wave, det);
    IDET_TRY(rc);
    // b_1, b_2 and R from S contiguous integers (Alg. 4.1), u for the
    // projections
    SplitMix gb(o.seed ^ 0xb5ull), gu(o.seed ^ 0x9a11ull);
    const double l2S = rhs_range_log2(n, J.log2H);
    const uint64_t S = (uint64_t)std::exp2(std::floor(l2S));
    std::vector<int64_t> bh(2 * n), Rh(2 * n);
    std::vector<int32_t> uh(n);
    for (auto &v : bh) v = (int64_t)gb.below(S) - (int64_t)(S / 2);
    for (auto &v : Rh) v = (int64_t)gb.below(S) - (int64_t)(S / 2);
    double u1 = 0, lc = 0, lcmin = INFINITY, log2Ne = 0;
    for (int64_t i = 0; i < n; ++i) {
        uh[i] = (int32_t)(gu.next() & 0xffff);
        u1 += uh[i];
        const double c = 0.5 * std::log2(std::max(J.colsq[i], 1.0));
        lc += c;
        lcmin = std::min(lcmin, c);
    }
    for (int l = 0; l < 2; ++l) {
        double bb = 1.0;
        for (int64_t i = 0; i < n; ++i) bb += (double)bh[l * n + i] * (double)bh[l * n + i];
        log2Ne = std::max(log2Ne, 0.5 * std::log2(bb * (1 + 1e-12)) + lc - lcmin);
    }
    const double lp = std::log2((double)p);
    const int hNe = (int)std::ceil((log2Ne + 1) / lp);
    const int hN = (int)std::ceil((log2Ne + std::log2(std::max(u1, 1.0)) + 1) / lp);
    const int hD = (int)std::ceil((J.log2H + 1) / lp);
    const double log2RN = 1.0 + 2.0 * (std::log2((double)n) + std::log2((double)S) + log2Ne);
    const int m = std::max(hN + hD + 2, (int)std::ceil((log2RN + 2) / lp) + 1);
    int32_t *ud = nullptr, *dig = nullptr;
    int64_t *bd = nullptr, *Rd = nullptr, *z = nullptr;
    IDET_TRY(ws.alloc_n(&ud, n));
    IDET_TRY(ws.alloc_n(&bd, 2 * (size_t)n));
    IDET_TRY(ws.alloc_n(&Rd, 2 * (size_t)n));
    IDET_TRY(ws.alloc_n(&dig, 2 * (size_t)m * n));
    IDET_TRY(ws.alloc_n(&z, 2 * (size_t)m));
    IDET_CUDA_TRY(cudaMemcpyAsync(ud, uh.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, s));
    IDET_CUDA_TRY(cudaMemcpyAsync(bd, bh.data(), 16 * (size_t)n, cudaMemcpyHostToDevice, s));
    IDET_CUDA_TRY(cudaMemcpyAsync(Rd, Rh.data(), 16 * (size_t)n, cudaMemcpyHostToDevice, s));
    LiftArgs la{};
    la.Cinv = Cinv;
    la.b = bd;
    la.b2 = bd + n;
    la.u = ud;
    la.n = n;
    la.m = m;
    la.nrhs = 2;
    la.mod = make_mod(p);
    la.pinv = inv_mod_2_64(p);
    la.digits = dig;
    la.digits2 = dig + (size_t)m * n;
    la.zproj = z;
    la.zproj2 = z + m;
    la.amax = J.amax;
    Timer tl(s);
    int to = 0;
    float kms = 0;
    LiftInfo li{};
    IDET_TRY(launch_lift(la, J.Anar, J.abytes, J.ldl, ws, &to, &kms, &li));
    J.st.lift_timed_out = to;
    J.st.ms_lift_kernel += li.ms_steps;
    J.st.ms_lift_setup += li.ms_setup;
    J.st.lift_bytes += li.bytes;
    J.st.lift_path = li.path;
    J.st.lift_iters = m;
    uint32_t *D1 = nullptr, *D2 = nullptr;
    int l1 = 0, l2 = 0;
    Timer trr(s);
    IDET_TRY(lcm_of_denominators(dig, n, m, p, z, hN, hNe, hD, ws, &D1, &l1));
    IDET_TRY(lcm_of_denominators(dig + (size_t)m * n, n, m, p, z + m, hN, hNe, hD, ws, &D2, &l2));
    J.st.ms_rr += trr.stop();
    J.st.ms_lift += tl.stop();
    // i = 1: K = pi~_1 = s~(x_1); resume the CRA for the time of one solve
    uint32_t *Kbin = nullptr;
    int Klen = 0;
    double log2K = 0;
    IDET_TRY(radix_dev_to_binary(ws, D1, l1, p, &Kbin, &Klen, &log2K));
    J.st.log2_K = (int)std::floor(log2K);
    bool done = false;
    IDET_TRY(det_over_K(J, Kbin, Klen, log2K, wave, det, false, 0.0, &done));
    if (done) return IDET_OK;
    // i = 2: K = lcm(K, pi~_2)
    uint32_t *St = nullptr, *P2 = nullptr, *K2 = nullptr;
    int ls = 0, lp2 = 0, lk = 0;
    Timer tb(s);
    IDET_TRY(lcm_radix(D1, l1, D2, l2, p, ws, &St, &ls));
    IDET_TRY(bonus_pi2(dig, n, m, p, Rd, St, ls, ws, &P2, &lp2));
    IDET_TRY(lcm_radix(D1, l1, P2, lp2, p, ws, &K2, &lk));
    J.st.ms_rr += tb.stop();
    IDET_TRY(radix_dev_to_binary(ws, K2, lk, p, &Kbin, &Klen, &log2K));
    J.st.log2_K = (int)std::floor(log2K);
    return det_over_K(J, Kbin, Klen, log2K, wave, det);
}

int idet_extended_bonus(const int64_t *A, int64_t n, int64_t lda, const int64_t *B,
                        const int64_t *R, int32_t on_device, const idet_opts *opts, void *stream,
                        idet_int *pi, idet_int *s_tilde) {
    if (n <= 0 || n > IDET_MAX_ORDER || lda < n || !A || !B || !R || !pi || !s_tilde) {
        set_last_error("invalid argument");
        return IDET_ERR_ARG;
    }
    for (int64_t i = 0; i < 2 * n; ++i)
        if (B[i] >= (1ll << 62) || B[i] <= -(1ll << 62) || R[i] >= (1ll << 62) ||
            R[i] <= -(1ll << 62)) {
            set_last_error("entries of B and R must satisfy |v| < 2^62");
            return IDET_ERR_ARG;
        }
    idet_opts o;
    idet_default_opts(&o);
    if (opts) o = *opts;
    cudaStream_t s = (cudaStream_t)stream;
    Workspace ws(s);
    DevMatrix M;
    IDET_TRY(stage_matrix(A, n, lda, on_device, ws, M));
    DetJob J(M, ws, o);
    IDET_TRY(J.stats());
    if (J.log2H == -INFINITY) {
        set_last_error("A is singular (zero row or column)");
        return IDET_ERR_SINGULAR;
    }
    IDET_TRY(make_Anar(J.M, J.amax, ws, &J.Anar, &J.abytes, &J.ldl));
    int32_t *Cinv = nullptr;
    IDET_TRY(ws.alloc_n(&Cinv, (size_t)n * J.ldl));
    SplitMix gp(o.seed ^ 0x11f7ull);
    uint32_t p = 0;
    int rc = IDET_ERR_SINGULAR;
    for (int tries = 0; tries < 6 && rc == IDET_ERR_SINGULAR; ++tries) {
        p = random_prime31(gp);
        rc = inverse_mod_prime(J.M, p, J.nb, ws, Cinv, J.ldl);
    }
    if (rc == IDET_ERR_SINGULAR) {
        set_last_error("A is singular (singular modulo 6 random 31-bit primes)");
        return rc;
    }
    IDET_TRY(rc);
    // lengths: the denominators (below H), the numerators N_lj = s~ x_lj
    // (Cramer: |N_lj| <= |det A_j(b_l)| <= ||b_l|| prod_{k != j} ||col_k||)
    // and det(R N) <= 2 (n max|r| max|N|)^2
    SplitMix g(o.seed ^ 0x9a11ull);
    std::vector<int32_t> uh(n);
    double u1 = 0, lc = 0, lcmin = INFINITY, log2Ne = 0, rmax = 1;
    for (int64_t i = 0; i < n; ++i) {
        uh[i] = (int32_t)(g.next() & 0xffff);
        u1 += uh[i];
        const double c = 0.5 * std::log2(std::max(J.colsq[i], 1.0));
        lc += c;
        lcmin = std::min(lcmin, c);
    }
    for (int l = 0; l < 2; ++l) {
        double bb = 1.0;
        for (int64_t i = 0; i < n; ++i) bb += (double)B[l * n + i] * (double)B[l * n + i];
        log2Ne = std::max(log2Ne, 0.5 * std::log2(bb * (1 + 1e-12)) + lc - lcmin);
    }
    for (int64_t i = 0; i < 2 * n; ++i) rmax = std::max(rmax, std::fabs((double)R[i]));
    const double lp = std::log2((double)p);
    const int hNe = (int)std::ceil((log2Ne + 1) / lp);
    const int hN = (int)std::ceil((log2Ne + std::log2(std::max(u1, 1.0)) + 1) / lp);
    const int hD = (int)std::ceil((J.log2H + 1) / lp);
    const double log2RN = 1.0 + 2.0 * (std::log2((double)n) + std::log2(rmax) + log2Ne);
    const int m = std::max(hN + hD + 2, (int)std::ceil((log2RN + 2) / lp) + 1);
    int32_t *ud = nullptr, *dig = nullptr;
    int64_t *bd = nullptr, *Rd = nullptr, *z = nullptr, *r = nullptr;
    IDET_TRY(ws.alloc_n(&ud, n));
    IDET_TRY(ws.alloc_n(&bd, 2 * (size_t)n));
    IDET_TRY(ws.alloc_n(&Rd, 2 * (size_t)n));
    IDET_TRY(ws.alloc_n(&dig, 2 * (size_t)m * n));
    IDET_TRY(ws.alloc_n(&z, 2 * (size_t)m));
    IDET_TRY(ws.alloc_n(&r, 2 * (size_t)n));
    IDET_CUDA_TRY(cudaMemcpyAsync(ud, uh.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, s));
    IDET_CUDA_TRY(cudaMemcpyAsync(bd, B, 16 * (size_t)n, cudaMemcpyHostToDevice, s));
    IDET_CUDA_TRY(cudaMemcpyAsync(Rd, R, 16 * (size_t)n, cudaMemcpyHostToDevice, s));
    // both solves in one block lift
    LiftArgs la{};
    la.Cinv = Cinv;
    la.b = bd;
    la.b2 = bd + n;
    la.u = ud;
    la.n = n;
    la.m = m;
    la.nrhs = 2;
    la.mod = make_mod(p);
    la.pinv = inv_mod_2_64(p);
    la.digits = dig;
    la.digits2 = dig + (size_t)m * n;
    la.zproj = z;
    la.zproj2 = z + m;
    la.r = r;
    la.r2 = r + n;
    la.amax = J.amax;
    int to = 0;
    IDET_TRY(launch_lift(la, J.Anar, J.abytes, J.ldl, ws, &to));
    // s~ = lcm of the denominators of both solutions
    uint32_t *D1 = nullptr, *D2 = nullptr, *S = nullptr, *P = nullptr;
    int l1 = 0, l2 = 0, ls = 0, lpi = 0;
    IDET_TRY(lcm_of_denominators(dig, n, m, p, z, hN, hNe, hD, ws, &D1, &l1));
    IDET_TRY(lcm_of_denominators(dig + (size_t)m * n, n, m, p, z + m, hN, hNe, hD, ws, &D2, &l2));
    IDET_TRY(lcm_radix(D1, l1, D2, l2, p, ws, &S, &ls));
    IDET_TRY(bonus_pi2(dig, n, m, p, Rd, S, ls, ws, &P, &lpi));
    IDET_TRY(radix_to_int(ws, S, ls, p, s_tilde));
    return radix_to_int(ws, P, lpi, p, pi);
}

// ---------------------------------------------------------------------------
// Batched determinants: Alg. 4.1 (i_max = 1) for many independent matrices,
// advanced together phase by phase. The LUs of all (matrix, prime) pairs with
// n <= 192 run in one launch (one CTA each), the lifts of all matrices in one
// launch (one CTA each), and the reconstructions and Chinese remaindering of
// all matrices in one launch each; larger matrices use the blocked LU.

namespace {

struct BItem {
    DevMatrix M;
    int64_t n = 0;
    double log2H = 0;
    std::vector<double> rowsq, colsq;
    unsigned long long amax = 0;
    double *d_rowsq = nullptr, *d_colsq = nullptr;
    unsigned long long *d_amax = nullptr;
    bool done = false;
    int k0 = 0;
    std::vector<uint32_t> dets;  // det mod P[0..dets.size())
    // lift
    uint32_t p = 0;
    int m = 0, hN = 0, hD = 0;
    int32_t *A32 = nullptr, *Cinv = nullptr;
    int64_t ld4 = 0, *bd = nullptr, *z = nullptr, *r = nullptr;
    int32_t *ud = nullptr;
    uint32_t *den = nullptr, *Kbin = nullptr;
    int32_t *info = nullptr;
    int Klen = 0;
    double log2K = 0;
    bool have_K = false;
};

}  // namespace

int idet_int_det_batch(int32_t count, const int64_t *const *A, const int64_t *n,
                       const int64_t *lda, int32_t on_device, const idet_opts *opts, void *stream,
                       idet_int *dets, idet_stats *stats) {
    if (count < 0 || (count > 0 && (!A || !n || !lda || !dets))) {
        set_last_error("invalid argument");
        return IDET_ERR_ARG;
    }
    for (int i = 0; i < count; ++i)
        if (n[i] < 0 || n[i] > IDET_MAX_ORDER || lda[i] < n[i] || (n[i] > 0 && !A[i])) {
            set_last_error("invalid matrix %d", i);
            return IDET_ERR_ARG;
        }
    const unsigned long long launches0 = g_launches;
    idet_opts o;
    idet_default_opts(&o);
    if (opts) o = *opts;
    cudaStream_t s = (cudaStream_t)stream;
    Workspace ws(s);
    Timer total(s);
    idet_stats agg{};
    const double log2l = 20.0;
    const double pool = (double)pool21().size();
    std::vector<BItem> it(count);
    // stage, then the statistics of all matrices in one launch and one copy
    int64_t total_n = 0;
    for (int i = 0; i < count; ++i) {
        BItem &b = it[i];
        b.n = n[i];
        if (b.n == 0) continue;
        IDET_TRY(stage_matrix(A[i], b.n, lda[i], on_device, ws, b.M));
        total_n += b.n;
    }
    {
        double *d_sq = nullptr;
        unsigned long long *d_amax = nullptr;
        StatJob *d_jobs = nullptr;
        IDET_TRY(ws.alloc_n(&d_sq, 2 * (size_t)std::max<int64_t>(total_n, 1)));
        IDET_TRY(ws.alloc_n(&d_amax, std::max(count, 1)));
        IDET_TRY(ws.alloc_n(&d_jobs, std::max(count, 1)));
        IDET_CUDA_TRY(cudaMemsetAsync(d_amax, 0, 8 * (size_t)std::max(count, 1), s));
        std::vector<StatJob> sj;
        std::vector<int> sid;
        int64_t off = 0;
        for (int i = 0; i < count; ++i) {
            BItem &b = it[i];
            if (b.n == 0) continue;
            sj.push_back({b.M.A, b.n, d_sq + off, d_sq + total_n + off, d_amax + sj.size()});
            sid.push_back(i);
            off += b.n;
        }
        if (!sj.empty()) {
            IDET_CUDA_TRY(cudaMemcpyAsync(d_jobs, sj.data(), sizeof(StatJob) * sj.size(),
                                          cudaMemcpyHostToDevice, s));
            IDET_TRY(launch_stats_multi(d_jobs, (int)sj.size(), s));
        }
        std::vector<double> hsq(2 * (size_t)total_n);
        std::vector<unsigned long long> hmax(sj.size());
        if (total_n > 0) {
            IDET_CUDA_TRY(cudaMemcpyAsync(hsq.data(), d_sq, 16 * (size_t)total_n,
                                          cudaMemcpyDeviceToHost, s));
            IDET_CUDA_TRY(cudaMemcpyAsync(hmax.data(), d_amax, 8 * hmax.size(),
                                          cudaMemcpyDeviceToHost, s));
        }
        IDET_CUDA_TRY(cudaStreamSynchronize(s));
        off = 0;
        for (size_t q = 0; q < sid.size(); ++q) {
            BItem &b = it[sid[q]];
            b.rowsq.assign(hsq.begin() + off, hsq.begin() + off + b.n);
            b.colsq.assign(hsq.begin() + total_n + off, hsq.begin() + total_n + off + b.n);
            b.amax = hmax[q];
            off += b.n;
        }
    }
    for (int i = 0; i < count; ++i) {
        BItem &b = it[i];
        if (b.n == 0) {
            uint32_t one = 1;
            IDET_TRY(write_int(&dets[i], 1, &one, 1));
            b.done = true;
            continue;
        }
        if (!entry_range(b.amax, &b.amax)) {
            set_last_error("matrix %d: entries must lie in [-2^31, 2^31 - 1]", i);
            return IDET_ERR_ARG;
        }
        double hr = 0, hc = 0;
        for (double v : b.rowsq) hr += v > 0 ? 0.5 * std::log2(v) : -INFINITY;
        for (double v : b.colsq) hc += v > 0 ? 0.5 * std::log2(v) : -INFINITY;
        b.log2H = std::min(hr, hc);
        if (b.log2H > -INFINITY) b.log2H = b.log2H * (1 + 1e-12) + 1e-6 * (double)b.n;
        if (b.log2H == -INFINITY || b.amax == 0) {
            IDET_TRY(write_int(&dets[i], 0, nullptr, 0));
            b.done = true;
            continue;
        }
        b.k0 = std::max(1, k_default(o.log2_epsilon, pool, b.log2H, log2l));
    }
    // shared random prime sequence (Alg. 2.1), parameters on the device
    PrimeDraw draw(o.seed);
    std::vector<uint32_t> P;
    ModP *modsd = nullptr;
    uint32_t *Pd = nullptr;
    int mods_cap = 0;
    auto ensure_primes = [&](int need) -> int {
        if (need <= (int)P.size() && need <= mods_cap) return IDET_OK;
        while ((int)P.size() < need) {
            uint32_t q;
            if (!draw.take(q)) {
                set_last_error("prime pool exhausted");
                return IDET_ERR_INTERNAL;
            }
            P.push_back(q);
        }
        const int cap = std::max(need, 2 * mods_cap);
        while ((int)P.size() < cap) {
            uint32_t q;
            if (!draw.take(q)) break;
            P.push_back(q);
        }
        std::vector<ModP> mh(P.size());
        for (size_t k = 0; k < P.size(); ++k) mh[k] = make_mod(P[k]);
        IDET_TRY(ws.alloc_n(&modsd, P.size()));
        IDET_TRY(ws.alloc_n(&Pd, P.size()));
        IDET_CUDA_TRY(cudaMemcpyAsync(modsd, mh.data(), sizeof(ModP) * P.size(),
                                      cudaMemcpyHostToDevice, s));
        IDET_CUDA_TRY(cudaMemcpyAsync(Pd, P.data(), 4 * P.size(), cudaMemcpyHostToDevice, s));
        mods_cap = (int)P.size();
        return IDET_OK;
    };
    // det mod P[have .. need) for the listed items; results of all items in
    // one device array, copied back once
    auto factor = [&](const std::vector<std::pair<int, int>> &want) -> int {
        Timer t(s);
        std::vector<LUSmallJob> jobs;
        std::vector<ElimJob> ejobs;
        int maxn = 1, max_en = 1;
        size_t tot = 0;
        for (auto &wi : want) tot += (size_t)std::max(0, wi.second - (int)it[wi.first].dets.size());
        if (tot == 0) return IDET_OK;
        uint32_t *dd_all = nullptr;
        IDET_TRY(ws.alloc_n(&dd_all, tot));
        std::vector<size_t> off(want.size(), 0);
        size_t pos = 0;
        for (size_t q = 0; q < want.size(); ++q) {
            BItem &b = it[want[q].first];
            const int have = (int)b.dets.size(), need = want[q].second;
            if (need <= have) continue;
            IDET_TRY(ensure_primes(need));
            const int W = need - have;
            uint32_t *dd = dd_all + pos;
            off[q] = pos;
            pos += W;
            agg.lu_macs += (2.0 / 3.0) * (double)b.n * b.n * b.n * W;
            agg.primes_used += W;
            if (b.n > 192 && elim_cluster_fits((int)b.n)) {
                // one cluster per prime, reducing the int64 entries itself
                for (int w = 0; w < W; ++w) {
                    ElimJob e{};
                    e.A = b.M.A;
                    e.lda = b.n;
                    e.n = (int32_t)b.n;
                    e.ld = (int32_t)b.n;
                    e.mod = make_mod(P[have + w]);
                    e.det = dd + w;
                    ejobs.push_back(e);
                }
                max_en = std::max<int>(max_en, (int)b.n);
            } else if (b.n <= 192) {
                // the small LU reduces the int64 entries while loading them
                LUState *st = nullptr;
                IDET_TRY(ws.alloc_n(&st, W));
                for (int w = 0; w < W; ++w) {
                    LUSmallJob j{};
                    j.A64 = b.M.A;
                    j.n = (int32_t)b.n;
                    j.mod = make_mod(P[have + w]);
                    j.st = st + w;
                    j.det = dd + w;
                    jobs.push_back(j);
                }
                maxn = std::max<int>(maxn, (int)b.n);
            } else {
                int32_t *R = nullptr;
                IDET_TRY(ws.alloc_n(&R, (size_t)W * b.n * b.n));
                IDET_TRY(launch_reduce(b.M.A, b.n, b.n, modsd + have, W, R, s));
                std::vector<ModP> mh(W);
                for (int w = 0; w < W; ++w) mh[w] = make_mod(P[have + w]);
                IDET_TRY(lu_factor_batched(R, b.n, modsd + have, mh.data(), W, false, o.nb, nullptr,
                                           dd, o.update_path, ws));
            }
        }
        if (!jobs.empty() || !ejobs.empty()) {
            // one graph per shape: small LUs and cluster eliminations over
            // their job arrays
            const int nj = (int)jobs.size(), ne = (int)ejobs.size();
            const uint64_t key = 0x1000000000ull ^ ((uint64_t)maxn << 40) ^ ((uint64_t)max_en << 20);
            IDET_TRY(run_phase_graph(
                s, key,
                {{jobs.data(), sizeof(LUSmallJob) * jobs.size()},
                 {ejobs.data(), sizeof(ElimJob) * ejobs.size()}},
                [&](const std::vector<const void *> &d, cudaStream_t gs) -> int {
                    if (nj) IDET_TRY(lu_small_multi((const LUSmallJob *)d[0], nj, maxn, gs));
                    if (ne) IDET_TRY(launch_elim_cluster((const ElimJob *)d[1], ne, max_en, 0, gs));
                    return IDET_OK;
                }));
        }
        std::vector<uint32_t> hres(tot);
        IDET_CUDA_TRY(cudaMemcpyAsync(hres.data(), dd_all, 4 * tot, cudaMemcpyDeviceToHost, s));
        IDET_CUDA_TRY(cudaStreamSynchronize(s));
        for (size_t q = 0; q < want.size(); ++q) {
            BItem &b = it[want[q].first];
            const int have = (int)b.dets.size(), need = want[q].second;
            if (need <= have) continue;
            b.dets.insert(b.dets.end(), hres.begin() + off[q], hres.begin() + off[q] + (need - have));
        }
        agg.ms_lu += t.stop();
        return IDET_OK;
    };
    // Garner digits for each listed item: residues res[i] mod prs[i], all
    // items packed into one upload, one launch and one copy back
    auto cra = [&](const std::vector<int> &ids, const std::vector<std::vector<uint32_t>> &prs,
                   const std::vector<std::vector<uint32_t>> &res,
                   std::vector<std::vector<int32_t>> &dig) -> int {
        Timer t(s);
        size_t tot = 0;
        for (auto &v : prs) tot += v.size();
        std::vector<uint32_t> hp(tot + 1), hr(tot + 1);
        std::vector<size_t> off(ids.size());
        size_t pos = 0;
        for (size_t q = 0; q < ids.size(); ++q) {
            off[q] = pos;
            std::copy(prs[q].begin(), prs[q].end(), hp.begin() + pos);
            std::copy(res[q].begin(), res[q].end(), hr.begin() + pos);
            pos += prs[q].size();
        }
        uint32_t *dp = nullptr, *dr = nullptr;
        int32_t *dd = nullptr;
        CraJob *jd = nullptr;
        IDET_TRY(ws.alloc_n(&dp, tot + 1));
        IDET_TRY(ws.alloc_n(&dr, tot + 1));
        IDET_TRY(ws.alloc_n(&dd, tot + 1));
        IDET_TRY(ws.alloc_n(&jd, ids.size() + 1));
        IDET_CUDA_TRY(cudaMemcpyAsync(dp, hp.data(), 4 * tot, cudaMemcpyHostToDevice, s));
        IDET_CUDA_TRY(cudaMemcpyAsync(dr, hr.data(), 4 * tot, cudaMemcpyHostToDevice, s));
        std::vector<CraJob> jobs(ids.size());
        for (size_t q = 0; q < ids.size(); ++q) {
            jobs[q].primes = dp + off[q];
            jobs[q].residues = dr + off[q];
            jobs[q].digits = dd + off[q];
            jobs[q].count = (int32_t)prs[q].size();
        }
        IDET_CUDA_TRY(cudaMemcpyAsync(jd, jobs.data(), sizeof(CraJob) * jobs.size(),
                                      cudaMemcpyHostToDevice, s));
        IDET_TRY(launch_cra_multi(jd, (int)jobs.size(), s));
        std::vector<int32_t> hd(tot + 1);
        IDET_CUDA_TRY(cudaMemcpyAsync(hd.data(), dd, 4 * tot, cudaMemcpyDeviceToHost, s));
        IDET_CUDA_TRY(cudaStreamSynchronize(s));
        dig.assign(ids.size(), {});
        for (size_t q = 0; q < ids.size(); ++q)
            dig[q].assign(hd.begin() + off[q], hd.begin() + off[q] + prs[q].size());
        agg.ms_cra += t.stop();
        return IDET_OK;
    };
    // det_i = K_i * sum_{t<c} dig_t prod_{j<t} p_j for every finished item,
    // one launch per item and one copy back for all
    struct AsmReq {
        int i;
        std::vector<uint32_t> prs;
        std::vector<int32_t> dig;
        const uint32_t *K;
        int Klen;
    };
    std::vector<AsmReq> pending;
    auto flush_assemble = [&]() -> int {
        if (pending.empty()) return IDET_OK;
        Timer t(s);
        const size_t R = pending.size();
        std::vector<size_t> doff(R), boff(R);
        std::vector<int> cap(R);
        size_t dt = 0, bt = 0;
        for (size_t q = 0; q < R; ++q) {
            double bits = 64;
            for (uint32_t p : pending[q].prs) bits += std::log2((double)p);
            cap[q] = (int)(bits / 32) + (pending[q].K ? pending[q].Klen : 1) + 4;
            doff[q] = dt;
            boff[q] = bt;
            dt += pending[q].prs.size();
            bt += 2 * (size_t)cap[q];
        }
        std::vector<uint32_t> hp(dt + 1);
        std::vector<int32_t> hg(dt + 1);
        for (size_t q = 0; q < R; ++q) {
            std::copy(pending[q].prs.begin(), pending[q].prs.end(), hp.begin() + doff[q]);
            std::copy(pending[q].dig.begin(), pending[q].dig.end(), hg.begin() + doff[q]);
        }
        uint32_t *dp = nullptr, *buf = nullptr, *one = nullptr;
        int32_t *dg = nullptr, *info = nullptr;
        IDET_TRY(ws.alloc_n(&dp, dt + 1));
        IDET_TRY(ws.alloc_n(&dg, dt + 1));
        IDET_TRY(ws.alloc_n(&buf, bt));
        IDET_TRY(ws.alloc_n(&info, 4 * R));
        IDET_TRY(ws.alloc_n(&one, 1));
        const uint32_t h1 = 1;
        IDET_CUDA_TRY(cudaMemcpyAsync(one, &h1, 4, cudaMemcpyHostToDevice, s));
        IDET_CUDA_TRY(cudaMemcpyAsync(dp, hp.data(), 4 * dt, cudaMemcpyHostToDevice, s));
        IDET_CUDA_TRY(cudaMemcpyAsync(dg, hg.data(), 4 * dt, cudaMemcpyHostToDevice, s));
        for (size_t q = 0; q < R; ++q)
            IDET_TRY(launch_mixed_to_int(dp + doff[q], dg + doff[q], (int)pending[q].prs.size(),
                                         pending[q].K ? pending[q].K : one,
                                         pending[q].K ? pending[q].Klen : 1, buf + boff[q], cap[q],
                                         info + 4 * q, s));
        std::vector<int32_t> hinfo(4 * R);
        std::vector<uint32_t> hbuf(bt);
        IDET_CUDA_TRY(cudaMemcpyAsync(hinfo.data(), info, 16 * R, cudaMemcpyDeviceToHost, s));
        IDET_CUDA_TRY(cudaMemcpyAsync(hbuf.data(), buf, 4 * bt, cudaMemcpyDeviceToHost, s));
        IDET_CUDA_TRY(cudaStreamSynchronize(s));
        for (size_t q = 0; q < R; ++q) {
            if (hinfo[4 * q + 2]) {
                set_last_error("reconstruction buffer too small");
                return IDET_ERR_INTERNAL;
            }
            IDET_TRY(write_int(&dets[pending[q].i], hinfo[4 * q], hbuf.data() + boff[q],
                               (uint32_t)hinfo[4 * q + 1]));
        }
        pending.clear();
        agg.ms_cra += t.stop();
        return IDET_OK;
    };

    // Alg. 2.1 on det(A_i) for k0_i primes (Alg. 4.1, lines 1-4)
    {
        std::vector<std::pair<int, int>> want;
        for (int i = 0; i < count; ++i)
            if (!it[i].done) want.push_back({i, it[i].k0});
        IDET_TRY(factor(want));
        std::vector<int> ids;
        std::vector<std::vector<uint32_t>> prs, res;
        for (int i = 0; i < count; ++i)
            if (!it[i].done) {
                ids.push_back(i);
                prs.push_back(std::vector<uint32_t>(P.begin(), P.begin() + it[i].dets.size()));
                res.push_back(it[i].dets);
            }
        std::vector<std::vector<int32_t>> dig;
        if (!ids.empty()) IDET_TRY(cra(ids, prs, res, dig));
        for (size_t q = 0; q < ids.size(); ++q) {
            int why = 0;
            const int i = ids[q];
            const int stop = CraScan::scan(dig[q], prs[q], it[i].log2H, o.log2_epsilon, log2l, pool,
                                           o.certify != 0, &why);
            if (why == 3) return inconsistent_residues();
            if (stop >= 0) {
                pending.push_back({i, std::vector<uint32_t>(prs[q].begin(), prs[q].begin() + stop + 1),
                                   std::vector<int32_t>(dig[q].begin(), dig[q].begin() + stop + 1),
                                   nullptr, 0});
                it[i].done = true;
            }
        }
        IDET_TRY(flush_assemble());
    }
    // one Dixon solve per remaining matrix, all in one launch
    {
        Timer t(s);
        std::vector<int> ids;
        for (int i = 0; i < count; ++i)
            if (!it[i].done) ids.push_back(i);
        SplitMix gp(o.seed ^ 0x11f7ull);
        uint32_t p0 = random_prime31(gp);
        // A_i^{-1} mod p0 (and A_i narrowed to int32) for every matrix that
        // fits a cluster, in one launch
        std::vector<ElimJob> ej;
        std::vector<int> ejid;
        int max_en = 1;
        uint32_t *eflag = nullptr;
        IDET_TRY(ws.alloc_n(&eflag, std::max<size_t>(ids.size(), 1)));
        for (int i : ids) {
            BItem &b = it[i];
            b.ld4 = (b.n + 3) / 4 * 4;
            IDET_TRY(ws.alloc_n(&b.A32, (size_t)b.n * b.ld4));
            IDET_TRY(ws.alloc_n(&b.Cinv, (size_t)b.n * b.ld4));
            if (elim_cluster_fits((int)b.n)) {
                ElimJob e{};
                e.A = b.M.A;
                e.lda = b.n;
                e.n = (int32_t)b.n;
                e.ld = (int32_t)b.ld4;
                e.mod = make_mod(p0);
                e.Cinv = b.Cinv;
                e.A32 = b.A32;
                e.det = eflag + ej.size();
                ej.push_back(e);
                ejid.push_back(i);
                max_en = std::max<int>(max_en, (int)b.n);
            } else {
                IDET_TRY(launch_narrow(b.M.A, b.n, b.n, b.A32, b.ld4, 4, s));
            }
        }
        std::vector<uint32_t> einv(ids.size() + 1, 0);
        if (!ej.empty()) {
            ElimJob *ejd = nullptr;
            IDET_TRY(ws.alloc_n(&ejd, ej.size()));
            IDET_CUDA_TRY(cudaMemcpyAsync(ejd, ej.data(), sizeof(ElimJob) * ej.size(),
                                          cudaMemcpyHostToDevice, s));
            Timer ti(s);
            IDET_TRY(launch_elim_cluster(ejd, (int)ej.size(), max_en, 1, s));
            agg.ms_inverse += ti.stop();
            IDET_CUDA_TRY(cudaMemcpyAsync(einv.data(), eflag, 4 * ej.size(), cudaMemcpyDeviceToHost, s));
            IDET_CUDA_TRY(cudaStreamSynchronize(s));
        }
        std::vector<char> inv_ok(count, 0);
        for (size_t q = 0; q < ej.size(); ++q) inv_ok[ejid[q]] = einv[q] != 0;
        // right-hand sides, projections and lift lengths (host), then every
        // per-system vector in one device array each
        std::vector<int> lid;
        std::vector<int64_t> hb;
        std::vector<int32_t> hu;
        std::vector<size_t> voff, zoff, doff;
        size_t vt = 0, zt = 0, dt = 0;
        for (int i : ids) {
            BItem &b = it[i];
            uint32_t p = p0;
            int rc = inv_ok[i] ? IDET_OK : IDET_ERR_SINGULAR;
            if (!inv_ok[i] && elim_cluster_fits((int)b.n)) p = random_prime31(gp);
            for (int tries = 0; tries < 6 && rc == IDET_ERR_SINGULAR; ++tries) {
                rc = inverse_mod_prime(b.M, p, 32, ws, b.Cinv, b.ld4);
                if (rc == IDET_ERR_SINGULAR) p = random_prime31(gp);
            }
            if (rc != IDET_OK && rc != IDET_ERR_SINGULAR) return rc;
            if (rc != IDET_OK) {
                b.p = 0;  // no solve: the CRA alone finishes this matrix
                continue;
            }
            b.p = p;
            agg.inverse_macs += 2.0 * (double)b.n * b.n * b.n;
            // bounds as in the single-matrix path
            SplitMix g(o.seed ^ 0xb5ull ^ ((uint64_t)i << 20));
            const double l2S = rhs_range_log2(b.n, b.log2H);
            const uint64_t S = (uint64_t)std::exp2(std::floor(l2S));
            double bb = 1.0, u1 = 0, lc = 0, lcmin = INFINITY;
            for (int64_t k = 0; k < b.n; ++k) {
                const int64_t bk = (int64_t)(g.below(S)) - (int64_t)(S / 2);
                const int32_t uk = (int32_t)(g.next() & 0xffff);
                hb.push_back(bk);
                hu.push_back(uk);
                bb += (double)bk * (double)bk;
                u1 += uk;
                const double c = 0.5 * std::log2(std::max(b.colsq[k], 1.0));
                lc += c;
                lcmin = std::min(lcmin, c);
            }
            const double log2N = std::log2(std::max(u1, 1.0)) + 0.5 * std::log2(bb * (1 + 1e-12)) + lc - lcmin;
            const double lp = std::log2((double)p);
            b.hN = (int)std::ceil((log2N + 1) / lp);
            b.hD = (int)std::ceil((b.log2H + 1) / lp);
            b.m = b.hN + b.hD + 2;
            lid.push_back(i);
            voff.push_back(vt);
            zoff.push_back(zt);
            doff.push_back(dt);
            vt += b.n;
            zt += b.m;
            dt += b.hD + 4;
        }
        if (!lid.empty()) {
            int64_t *bd = nullptr, *z = nullptr, *r = nullptr;
            int32_t *ud = nullptr, *info = nullptr;
            uint32_t *den = nullptr;
            IDET_TRY(ws.alloc_n(&bd, vt));
            IDET_TRY(ws.alloc_n(&ud, vt));
            IDET_TRY(ws.alloc_n(&r, vt));
            IDET_TRY(ws.alloc_n(&z, zt));
            IDET_TRY(ws.alloc_n(&den, dt));
            IDET_TRY(ws.alloc_n(&info, 4 * lid.size()));
            IDET_CUDA_TRY(cudaMemcpyAsync(bd, hb.data(), 8 * vt, cudaMemcpyHostToDevice, s));
            IDET_CUDA_TRY(cudaMemcpyAsync(ud, hu.data(), 4 * vt, cudaMemcpyHostToDevice, s));
            std::vector<LiftJob> lj;
            std::vector<RRJob> rj;
            int max_ld = 4, max_m = 1;
            for (size_t q = 0; q < lid.size(); ++q) {
                BItem &b = it[lid[q]];
                b.den = den + doff[q];
                b.info = info + 4 * q;
                LiftJob j{};
                j.A = b.A32;
                j.C = b.Cinv;
                j.b = bd + voff[q];
                j.u = ud + voff[q];
                j.r = r + voff[q];
                j.z = z + zoff[q];
                j.n = (int32_t)b.n;
                j.ld = (int32_t)b.ld4;
                j.m = b.m;
                j.mod = make_mod(b.p);
                j.pinv = inv_mod_2_64(b.p);
                lj.push_back(j);
                RRJob rr{};
                rr.z = z + zoff[q];
                rr.m = b.m;
                rr.hN = b.hN;
                rr.hD = b.hD;
                rr.den_cap = b.hD + 4;
                rr.den = b.den;
                rr.info = b.info;
                rr.p = b.p;
                rj.push_back(rr);
                max_ld = std::max<int>(max_ld, (int)b.ld4);
                max_m = std::max(max_m, b.m);
                agg.lift_iters += b.m;
                agg.lift_bytes += (double)b.m * 8.0 * b.n * b.n;
            }
            // one graph per shape: the lift of every system, then the
            // reconstruction of every projection (timed together)
            const int nl = (int)lj.size();
            const uint64_t key = 0x2000000000ull ^ ((uint64_t)max_ld << 32) ^ (uint64_t)max_m;
            Timer tk(s);
            IDET_TRY(run_phase_graph(
                s, key,
                {{lj.data(), sizeof(LiftJob) * lj.size()}, {rj.data(), sizeof(RRJob) * rj.size()}},
                [&](const std::vector<const void *> &d, cudaStream_t gs) -> int {
                    IDET_TRY(launch_lift_multi((const LiftJob *)d[0], nl, max_ld, gs));
                    IDET_TRY(launch_ratrecon_multi((const RRJob *)d[1], nl, max_m, gs));
                    return IDET_OK;
                }));
            agg.ms_lift_kernel += tk.stop();
            // denominators: status and digits of all systems in two copies,
            // then K in base 2^32 for each, their lengths in one copy
            std::vector<int32_t> hinfo(4 * lid.size());
            std::vector<uint32_t> hden(dt);
            IDET_CUDA_TRY(cudaMemcpyAsync(hinfo.data(), info, 16 * lid.size(), cudaMemcpyDeviceToHost, s));
            IDET_CUDA_TRY(cudaMemcpyAsync(hden.data(), den, 4 * dt, cudaMemcpyDeviceToHost, s));
            IDET_CUDA_TRY(cudaStreamSynchronize(s));
            uint32_t *kb = nullptr;
            int32_t *kl = nullptr;
            size_t kt = 0;
            for (size_t q = 0; q < lid.size(); ++q)
                if (hinfo[4 * q] == 0 && hinfo[4 * q + 1] > 0) kt += hinfo[4 * q + 1] + 2;
            IDET_TRY(ws.alloc_n(&kb, kt + 1));
            IDET_TRY(ws.alloc_n(&kl, lid.size()));
            size_t kp = 0;
            for (size_t q = 0; q < lid.size(); ++q) {
                BItem &b = it[lid[q]];
                const int kd = hinfo[4 * q + 1];
                if (hinfo[4 * q] != 0 || kd <= 0) continue;  // no factor: K = 1
                b.Kbin = kb + kp;
                kp += kd + 2;
                IDET_TRY(launch_radix_to_binary(b.den, kd, b.p, b.Kbin, kd + 2, kl + q, s));
                const uint32_t *dh = hden.data() + doff[q];
                const double top = dh[kd - 1] + (kd > 1 ? dh[kd - 2] / (double)b.p : 0.0);
                b.log2K = std::log2(top) + (kd - 1) * std::log2((double)b.p);
            }
            std::vector<int32_t> hkl(lid.size());
            IDET_CUDA_TRY(cudaMemcpyAsync(hkl.data(), kl, 4 * lid.size(), cudaMemcpyDeviceToHost, s));
            IDET_CUDA_TRY(cudaStreamSynchronize(s));
            for (size_t q = 0; q < lid.size(); ++q) {
                BItem &b = it[lid[q]];
                if (!b.Kbin) continue;
                b.Klen = hkl[q];
                b.have_K = b.Klen > 0;
            }
        }
        agg.ms_lift += t.stop();
    }
    // Alg. 2.1 on det(A_i)/K_i reusing the residues; more primes as needed
    for (int round = 0;; ++round) {
        std::vector<int> ids;
        for (int i = 0; i < count; ++i)
            if (!it[i].done) ids.push_back(i);
        if (ids.empty()) break;
        if (round > 4096) {
            set_last_error("batched determinant did not terminate");
            return IDET_ERR_INTERNAL;
        }
        // d_k K^{-1} mod p_k for every item with a factor: one launch each,
        // inputs and outputs in one array each, one copy back
        std::vector<std::vector<uint32_t>> prs(ids.size()), res(ids.size());
        {
            Timer t(s);
            std::vector<size_t> off(ids.size(), 0);
            size_t tot = 0;
            for (size_t q = 0; q < ids.size(); ++q)
                if (it[ids[q]].have_K) {
                    off[q] = tot;
                    tot += it[ids[q]].dets.size();
                }
            if (tot > 0) {
                std::vector<uint32_t> hi(tot);
                for (size_t q = 0; q < ids.size(); ++q)
                    if (it[ids[q]].have_K)
                        std::copy(it[ids[q]].dets.begin(), it[ids[q]].dets.end(), hi.begin() + off[q]);
                uint32_t *di = nullptr, *dout = nullptr;
                int32_t *dsk = nullptr;
                IDET_TRY(ws.alloc_n(&di, tot));
                IDET_TRY(ws.alloc_n(&dout, tot));
                IDET_TRY(ws.alloc_n(&dsk, tot));
                IDET_CUDA_TRY(cudaMemcpyAsync(di, hi.data(), 4 * tot, cudaMemcpyHostToDevice, s));
                for (size_t q = 0; q < ids.size(); ++q) {
                    BItem &b = it[ids[q]];
                    if (!b.have_K) continue;
                    IDET_TRY(launch_div_by_K(b.Kbin, b.Klen, Pd, di + off[q], dout + off[q],
                                             dsk + off[q], (int)b.dets.size(), s));
                }
                std::vector<uint32_t> ho(tot);
                std::vector<int32_t> hs(tot);
                IDET_CUDA_TRY(cudaMemcpyAsync(ho.data(), dout, 4 * tot, cudaMemcpyDeviceToHost, s));
                IDET_CUDA_TRY(cudaMemcpyAsync(hs.data(), dsk, 4 * tot, cudaMemcpyDeviceToHost, s));
                IDET_CUDA_TRY(cudaStreamSynchronize(s));
                for (size_t q = 0; q < ids.size(); ++q) {
                    BItem &b = it[ids[q]];
                    if (!b.have_K) continue;
                    for (size_t k = 0; k < b.dets.size(); ++k)
                        if (!hs[off[q] + k]) {
                            prs[q].push_back(P[k]);
                            res[q].push_back(ho[off[q] + k]);
                        }
                }
            }
            for (size_t q = 0; q < ids.size(); ++q) {
                BItem &b = it[ids[q]];
                if (b.have_K) continue;
                prs[q].assign(P.begin(), P.begin() + b.dets.size());
                res[q] = b.dets;
            }
            agg.ms_cra += t.stop();
        }
        std::vector<std::vector<int32_t>> dig;
        IDET_TRY(cra(ids, prs, res, dig));
        std::vector<std::pair<int, int>> more;
        for (size_t q = 0; q < ids.size(); ++q) {
            const int i = ids[q];
            BItem &b = it[i];
            int why = 0;
            const double lh = b.have_K ? std::max(0.0, b.log2H - b.log2K) : b.log2H;
            const int stop = CraScan::scan(dig[q], prs[q], lh, o.log2_epsilon, log2l, pool, false, &why);
            if (why == 3) return inconsistent_residues();
            if (stop >= 0) {
                pending.push_back({i, std::vector<uint32_t>(prs[q].begin(), prs[q].begin() + stop + 1),
                                   std::vector<int32_t>(dig[q].begin(), dig[q].begin() + stop + 1),
                                   b.have_K ? b.Kbin : nullptr, b.have_K ? b.Klen : 0});
                b.done = true;
            } else {
                more.push_back({i, (int)b.dets.size() + std::max(4, b.k0 / 2)});
            }
        }
        IDET_TRY(flush_assemble());
        if (!more.empty()) IDET_TRY(factor(more));
    }
    agg.ms_total = total.stop();
    agg.launches = g_launches - launches0;
    if (stats) *stats = agg;
    return IDET_OK;
}

}  // extern "C"
