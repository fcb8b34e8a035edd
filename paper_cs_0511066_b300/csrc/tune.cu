// Autotuner for the multi-prime LU (Section 2.1): the trailing-update
// arithmetic (limb count: int64 / int8 limbs / bf16 limbs on mma.sync or on
// tcgen05), the panel width nb and the prime-batch width W (primes factored
// per wave). For an order n it times the reduction plus the LU of W primes
// on a random matrix generated on the device (a counter-based hash of the
// entry index, so nothing is copied from the host) for every candidate and
// keeps the fastest time per prime. Results live in a process-wide table
// keyed by (n bucket, prime bits), with buckets of a quarter octave of n;
// IDET_PATH_AUTO, nb = 0 and wave = 0 consult it (nearest bucket within one
// octave, else the built-in defaults). The table is saved and loaded as
// JSON:
//   {"version": 1, "entries": [{"bucket": b, "n": n, "prime_bits": 21,
//     "update_path": 5, "nb": 32, "wave": 16, "ms_per_prime": 3.5}, ...]}
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "idet_internal.cuh"

namespace idet {

namespace {

std::mutex g_tune_mu;
std::map<std::pair<int, int>, idet_tuned> g_table;  // (bucket, prime bits) -> choice

int bucket_of(int64_t n) { return (int)std::floor(4.0 * std::log2((double)std::max<int64_t>(n, 1))); }

// Entries uniform in [-2^(bits-1), 2^(bits-1)) from SplitMix64 of (seed, i).
__global__ void k_fill_random(int64_t *A, int64_t count, uint64_t seed, int bits) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + 0x9e3779b97f4a7c15ull * (uint64_t)(i + 1);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        z ^= z >> 31;
        A[i] = (int64_t)(z >> (64 - bits)) - ((int64_t)1 << (bits - 1));
    }
}

}  // namespace

bool tuned_lookup(int64_t n, int prime_bits, idet_tuned *out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (g_table.empty()) return false;
    const int b = bucket_of(n);
    int best = -1, bd = 1 << 30;
    for (const auto &kv : g_table) {
        if (kv.first.second != prime_bits) continue;
        const int d = std::abs(kv.first.first - b);
        if (d < bd) {
            bd = d;
            best = kv.first.first;
        }
    }
    if (best < 0 || bd > 4) return false;
    *out = g_table[{best, prime_bits}];
    return true;
}

}  // namespace idet

using namespace idet;

extern "C" {

int idet_autotune(int64_t n, int32_t prime_bits, int32_t entry_bits, void *stream, idet_tuned *out) {
    if (n < 1 || n > IDET_MAX_ORDER || (prime_bits != 21 && prime_bits != 31) || entry_bits < 2 ||
        entry_bits > 32) {
        set_last_error("autotune: invalid argument");
        return IDET_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    Workspace ws(s);
    int64_t *A = nullptr;
    IDET_TRY(ws.alloc_n(&A, (size_t)n * n));
    k_fill_random<<<592, 256, 0, s>>>(A, n * n, 0x7a11u + (uint64_t)n, entry_bits);
    count_launch();
    IDET_CUDA_TRY(cudaGetLastError());
    // primes of the class, spread over it
    std::vector<uint32_t> pr;
    for (uint32_t c = prime_bits == 21 ? (1u << 20) + 1 : (1u << 30) + 1; pr.size() < 16; c += 2) {
        bool ok = c > 2;
        for (uint32_t q = 3; ok && (uint64_t)q * q <= c; q += 2) ok = c % q != 0;
        if (ok) pr.push_back(c);
    }
    std::vector<int> paths = prime_bits == 21
                                 ? std::vector<int>{IDET_PATH_TC05, IDET_PATH_INT64, IDET_PATH_BF16,
                                                    IDET_PATH_I8}
                                 : std::vector<int>{IDET_PATH_TC05, IDET_PATH_INT64};
    const int nbs[2] = {16, 32};
    const int waves[3] = {4, 8, 16};
    idet_tuned best{};
    best.ms_per_prime = INFINITY;
    EventPair ev;
    IDET_CUDA_TRY(cudaEventCreate(&ev.a));
    IDET_CUDA_TRY(cudaEventCreate(&ev.b));
    cudaEvent_t e0 = ev.a, e1 = ev.b;
    int rc = IDET_OK;
    for (int path : paths)
        for (int nb : nbs)
            for (int W : waves) {
                if (rc != IDET_OK) break;
                Workspace w2(s);
                std::vector<ModP> mh(W);
                for (int i = 0; i < W; ++i) mh[i] = make_mod(pr[i]);
                ModP *md = nullptr;
                int32_t *R = nullptr;
                uint32_t *dd = nullptr;
                if ((rc = w2.alloc_n(&md, W)) != IDET_OK) break;
                if ((rc = w2.alloc_n(&R, (size_t)W * n * n)) != IDET_OK) break;
                if ((rc = w2.alloc_n(&dd, W)) != IDET_OK) break;
                cudaMemcpyAsync(md, mh.data(), sizeof(ModP) * W, cudaMemcpyHostToDevice, s);
                float best_ms = INFINITY;
                for (int rep = 0; rep < 2 && rc == IDET_OK; ++rep) {  // first run warms up
                    cudaEventRecord(e0, s);
                    rc = launch_reduce(A, n, n, md, W, R, s);
                    if (rc == IDET_OK)
                        rc = lu_factor_batched(R, n, md, mh.data(), W, prime_bits == 31, nb,
                                               nullptr, dd, path, w2);
                    cudaEventRecord(e1, s);
                    if (cudaEventSynchronize(e1) != cudaSuccess) {
                        cudaGetLastError();
                        rc = IDET_ERR_CUDA;
                    }
                    float ms = 0;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep > 0) best_ms = ms;
                }
                if (rc != IDET_OK) break;
                const double per = best_ms / W;
                if (per < best.ms_per_prime) {
                    best.update_path = path;
                    best.nb = nb;
                    best.wave = W;
                    best.ms_per_prime = per;
                }
            }
    if (rc != IDET_OK) return rc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_table[{bucket_of(n), prime_bits}] = best;
    }
    if (out) *out = best;
    return IDET_OK;
}

int idet_tuning_save(const char *path) {
    if (!path) {
        set_last_error("tuning: null path");
        return IDET_ERR_ARG;
    }
    FILE *f = fopen(path, "w");
    if (!f) {
        set_last_error("tuning: cannot write %s", path);
        return IDET_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    fprintf(f, "{\"version\": 1, \"entries\": [");
    bool first = true;
    for (const auto &kv : g_table) {
        const idet_tuned &t = kv.second;
        fprintf(f,
                "%s\n  {\"bucket\": %d, \"n\": %lld, \"prime_bits\": %d, \"update_path\": %d, "
                "\"nb\": %d, \"wave\": %d, \"ms_per_prime\": %.6f}",
                first ? "" : ",", kv.first.first,
                (long long)std::llround(std::exp2(kv.first.first / 4.0)), kv.first.second,
                t.update_path, t.nb, t.wave, t.ms_per_prime);
        first = false;
    }
    fprintf(f, "\n]}\n");
    fclose(f);
    return IDET_OK;
}

int idet_tuning_load(const char *path) {
    if (!path) {
        set_last_error("tuning: null path");
        return IDET_ERR_ARG;
    }
    FILE *f = fopen(path, "r");
    if (!f) {
        set_last_error("tuning: cannot read %s", path);
        return IDET_ERR_ARG;
    }
    std::string text;
    char buf[4096];
    size_t k;
    while ((k = fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, k);
    fclose(f);
    // one object per entry: read the numbers after each key
    auto num = [&](size_t from, size_t to, const char *key, double *v) {
        const std::string kq = std::string("\"") + key + "\"";
        const size_t p = text.find(kq, from);
        if (p == std::string::npos || p >= to) return false;
        const size_t c = text.find(':', p);
        if (c == std::string::npos || c >= to) return false;
        char *end = nullptr;
        *v = strtod(text.c_str() + c + 1, &end);
        return end != text.c_str() + c + 1;
    };
    std::map<std::pair<int, int>, idet_tuned> t;
    size_t pos = text.find("\"entries\"");
    if (pos == std::string::npos) {
        set_last_error("tuning: no entries in %s", path);
        return IDET_ERR_ARG;
    }
    while (true) {
        const size_t a = text.find('{', pos);
        if (a == std::string::npos) break;
        const size_t b = text.find('}', a);
        if (b == std::string::npos) break;
        double bucket, bits, up, nb, wave, ms;
        if (!num(a, b, "bucket", &bucket) || !num(a, b, "prime_bits", &bits) ||
            !num(a, b, "update_path", &up) || !num(a, b, "nb", &nb) || !num(a, b, "wave", &wave) ||
            !num(a, b, "ms_per_prime", &ms)) {
            set_last_error("tuning: malformed entry in %s", path);
            return IDET_ERR_ARG;
        }
        if ((bits != 21 && bits != 31) || up < 0 || up > IDET_PATH_TC05 || nb < 0 || nb > 32 ||
            wave < 1 || wave > 256) {
            set_last_error("tuning: entry out of range in %s", path);
            return IDET_ERR_ARG;
        }
        idet_tuned e{};
        e.update_path = (int32_t)up;
        e.nb = (int32_t)nb;
        e.wave = (int32_t)wave;
        e.ms_per_prime = ms;
        t[{(int)bucket, (int)bits}] = e;
        pos = b + 1;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto &kv : t) g_table[kv.first] = kv.second;
    return IDET_OK;
}

void idet_tuning_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_table.clear();
}

}  // extern "C"
