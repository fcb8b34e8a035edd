// Serving: a request loop over the determinant method (Alg. 4.1) with
// continuous batching.
//
// Requests are queued as they arrive (idet_submit copies the matrix). A pool
// of worker threads, each owning a CUDA stream, takes work whenever a slot
// and device memory are free: jobs are admitted first-in first-out against
// an HBM budget, using an estimate of each job's device footprint; a job
// that does not fit lets later ones that do fit go ahead (a skipped head
// job reserves the memory after a bounded number of overtakes, so it cannot
// starve). A worker that takes a job with n <= small_n also takes the other
// queued small jobs that fit (up to max_batch) and runs them as one batch
// through the batched path (idet_int_det_batch); a larger job runs alone
// (idet_int_det). Jobs on different workers overlap on the device. Results
// are read with idet_poll.
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "idet_internal.cuh"

namespace idet {
namespace {

using Clock = std::chrono::steady_clock;

struct SJob {
    uint64_t ticket = 0;
    std::vector<int64_t> A;  // n x n, row-major
    int64_t n = 0;
    size_t foot = 0;
    int status = -1;  // -1 while pending
    int sign = 0;
    std::vector<uint32_t> limbs;
    idet_stats st{};
    int batched = 0;
    int skipped = 0;
    int worker = -1;
    std::string err;
    Clock::time_point t_sub, t_start, t_end;
};

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

// Device bytes of one job (upper estimate): the staged matrix (8 n^2), the
// residues of the first prime wave (4 n^2 per prime, up to 24 primes), the
// LU and inverse modulo the lifting prime (8 n^2), A narrowed and A^{-1}
// mod p for the lift (8 n^2), plus a fixed allowance.
size_t job_footprint(int64_t n) {
    const double nn = (double)n * (double)n;
    return (size_t)(nn * (8.0 + 4.0 * 24 + 8.0 + 8.0)) + ((size_t)16 << 20);
}

size_t det_cap_limbs(const std::vector<int64_t> &A, int64_t n) {
    // |det| <= prod of the row norms <= (sqrt(n) max|a|)^n
    int64_t amax = 0;
    for (int64_t v : A) amax = std::max<int64_t>(amax, v < 0 ? -v : v);
    const double bits = (double)n * (std::log2((double)amax + 1.0) + 0.5 * std::log2((double)n + 1));
    return (size_t)(bits / 32.0) + 8;
}

}  // namespace
}  // namespace idet

using namespace idet;

struct idet_server {
    size_t budget = 0, in_use = 0;
    int slots = 1, small_n = 512, max_batch = 64, device = 0;
    int max_skips = 8;
    idet_opts opts{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<SJob *> queue;
    std::unordered_map<uint64_t, SJob *> jobs;
    uint64_t next_ticket = 1;
    bool stop = false;
    int running = 0, max_running = 0;
    uint64_t admitted = 0, completed = 0, groups = 0;
    std::vector<std::thread> workers;
};

namespace {

// The admission rule, under the lock. Picks the jobs to run next into take
// (removing them from the queue) and returns their total footprint.
size_t pick(idet_server *S, std::vector<SJob *> &take) {
    take.clear();
    if (S->queue.empty()) return 0;
    const size_t room = S->budget - S->in_use;
    size_t pos = S->queue.size();
    SJob *head = S->queue.front();
    if (head->foot <= room) {
        pos = 0;
    } else if (head->skipped < S->max_skips) {
        for (size_t i = 1; i < S->queue.size(); ++i)
            if (S->queue[i]->foot <= room) {
                pos = i;
                break;
            }
    }
    if (pos == S->queue.size()) return 0;
    SJob *first = S->queue[pos];
    size_t foot = first->foot;
    take.push_back(first);
    if (first->n <= S->small_n) {
        for (size_t i = pos + 1; i < S->queue.size() && (int)take.size() < S->max_batch; ++i) {
            SJob *j = S->queue[i];
            if (j->n <= S->small_n && foot + j->foot <= room) {
                take.push_back(j);
                foot += j->foot;
            }
        }
    }
    // the jobs left before the first taken one were overtaken
    for (size_t i = 0; i < pos; ++i) S->queue[i]->skipped++;
    std::deque<SJob *> rest;
    size_t t = 0;
    for (SJob *j : S->queue) {
        if (t < take.size() && j == take[t]) {
            ++t;
            continue;
        }
        rest.push_back(j);
    }
    S->queue.swap(rest);
    return foot;
}

bool can_admit(idet_server *S) {
    if (S->queue.empty()) return false;
    const size_t room = S->budget - S->in_use;
    SJob *head = S->queue.front();
    if (head->foot <= room) return true;
    if (head->skipped >= S->max_skips) return false;
    for (size_t i = 1; i < S->queue.size(); ++i)
        if (S->queue[i]->foot <= room) return true;
    return false;
}

void run_group(idet_server *S, std::vector<SJob *> &take, cudaStream_t st) {
    const int count = (int)take.size();
    std::vector<std::vector<uint32_t>> bufs(count);
    std::vector<idet_int> outs(count);
    for (int i = 0; i < count; ++i) {
        bufs[i].assign(det_cap_limbs(take[i]->A, take[i]->n), 0);
        outs[i].sign = 0;
        outs[i].nlimbs = 0;
        outs[i].cap = (uint32_t)bufs[i].size();
        outs[i].limbs = bufs[i].data();
    }
    idet_stats stats{};
    int rc;
    if (count == 1 && take[0]->n > S->small_n) {
        rc = idet_int_det(take[0]->A.data(), take[0]->n, take[0]->n, 0, &S->opts, st, &outs[0],
                          &stats);
    } else {
        std::vector<const int64_t *> ptr(count);
        std::vector<int64_t> ns(count);
        for (int i = 0; i < count; ++i) {
            ptr[i] = take[i]->A.data();
            ns[i] = take[i]->n;
        }
        rc = idet_int_det_batch(count, ptr.data(), ns.data(), ns.data(), 0, &S->opts, st,
                                outs.data(), &stats);
    }
    std::string err;
    if (rc != IDET_OK) {
        err = idet_last_error();
        cudaStreamSynchronize(st);
    }
    const auto now = Clock::now();
    std::lock_guard<std::mutex> lk(S->mu);
    for (int i = 0; i < count; ++i) {
        SJob *j = take[i];
        j->status = rc;
        j->err = err;
        if (rc == IDET_OK) {
            j->sign = outs[i].sign;
            j->limbs.assign(bufs[i].begin(), bufs[i].begin() + outs[i].nlimbs);
        }
        j->st = stats;
        j->batched = count;
        j->t_end = now;
    }
    S->completed += count;
}

void worker_main(idet_server *S, int w) {
    t_native_alloc = true;
    cudaSetDevice(S->device);
    cudaStream_t st = nullptr;
    bool own_stream = true;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        // no stream of its own: this thread's per-thread default stream,
        // which is still not ordered with the other workers' work
        cudaGetLastError();
        st = cudaStreamPerThread;
        own_stream = false;
    }
    std::vector<SJob *> take;
    while (true) {
        size_t foot = 0;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || can_admit(S); });
            if (S->stop) break;
            foot = pick(S, take);
            if (take.empty()) continue;
            S->in_use += foot;
            S->running++;
            S->max_running = std::max(S->max_running, S->running);
            S->admitted += take.size();
            S->groups++;
            const auto now = Clock::now();
            for (SJob *j : take) {
                j->t_start = now;
                j->worker = w;
            }
        }
        run_group(S, take, st);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->in_use -= foot;
            S->running--;
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
    cudaStreamSynchronize(st);
    if (own_stream) cudaStreamDestroy(st);
}

}  // namespace

extern "C" {

idet_server *idet_server_create(size_t hbm_budget, int32_t slots, int32_t small_n,
                                int32_t max_batch, const idet_opts *opts) {
    if (slots < 1 || slots > 64 || small_n < 0 || max_batch < 1) {
        set_last_error("server: invalid argument");
        return nullptr;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        set_last_error("server: no CUDA device");
        return nullptr;
    }
    if (hbm_budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            set_last_error("server: cudaMemGetInfo failed");
            return nullptr;
        }
        hbm_budget = fr / 10 * 8;
    }
    // keep freed workspace in the stream-ordered pool between jobs
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    idet_server *S = new idet_server();
    S->budget = hbm_budget;
    S->slots = slots;
    S->small_n = small_n;
    S->max_batch = max_batch;
    S->device = dev;
    S->max_skips = 2 * slots + 2;
    idet_default_opts(&S->opts);
    if (opts) S->opts = *opts;
    for (int w = 0; w < slots; ++w) S->workers.emplace_back(worker_main, S, w);
    return S;
}

int idet_submit(idet_server *S, const int64_t *A, int64_t n, int64_t lda, uint64_t *ticket) {
    if (!S || !ticket || n < 1 || n > IDET_MAX_ORDER || lda < n || !A) {
        set_last_error("submit: invalid argument");
        return IDET_ERR_ARG;
    }
    SJob *j = new SJob();
    j->n = n;
    j->A.resize((size_t)n * n);
    for (int64_t i = 0; i < n; ++i) memcpy(&j->A[(size_t)i * n], A + i * lda, 8 * (size_t)n);
    for (int64_t v : j->A)
        if (v > 0x7fffffffll || v < -0x80000000ll) {
            delete j;
            set_last_error("submit: entries must lie in [-2^31, 2^31 - 1]");
            return IDET_ERR_ARG;
        }
    j->foot = job_footprint(n);
    j->t_sub = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (j->foot > S->budget) {
            delete j;
            set_last_error("submit: the job needs about %zu bytes, more than the budget", job_footprint(n));
            return IDET_ERR_NOMEM;
        }
        j->ticket = S->next_ticket++;
        S->jobs[j->ticket] = j;
        S->queue.push_back(j);
        *ticket = j->ticket;
    }
    S->cv_work.notify_one();
    return IDET_OK;
}

int idet_poll(idet_server *S, uint64_t ticket, int32_t timeout_ms, idet_int *det,
              idet_job_info *info) {
    if (!S || !det) {
        set_last_error("poll: invalid argument");
        return IDET_ERR_ARG;
    }
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) {
        set_last_error("poll: unknown ticket %llu", (unsigned long long)ticket);
        return IDET_ERR_ARG;
    }
    // The job is looked up again after every wake-up: another thread polling
    // the same ticket may have collected (and freed) it meanwhile.
    auto ready = [&] {
        auto f = S->jobs.find(ticket);
        return f == S->jobs.end() || f->second->status != -1;
    };
    if (timeout_ms < 0) {
        S->cv_done.wait(lk, ready);
    } else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
        set_last_error("poll: job %llu not finished", (unsigned long long)ticket);
        return IDET_ERR_TIMEOUT;
    }
    it = S->jobs.find(ticket);
    if (it == S->jobs.end()) {
        set_last_error("poll: ticket %llu was collected by another call",
                       (unsigned long long)ticket);
        return IDET_ERR_ARG;
    }
    SJob *j = it->second;
    if (info) {
        info->status = j->status;
        info->batched = j->batched;
        info->worker = j->worker;
        info->ms_queue = ms_between(j->t_sub, j->t_start);
        info->ms_run = ms_between(j->t_start, j->t_end);
        info->ms_latency = ms_between(j->t_sub, j->t_end);
        info->t_start_ms = ms_between(Clock::time_point(), j->t_start);
        info->t_end_ms = ms_between(Clock::time_point(), j->t_end);
        info->stats = j->st;
    }
    if (j->status != IDET_OK) {
        const int rc = j->status;
        set_last_error("job %llu failed: %s", (unsigned long long)ticket, j->err.c_str());
        S->jobs.erase(it);
        delete j;
        S->cv_done.notify_all();  // other pollers of this ticket see it is gone
        return rc;
    }
    const uint32_t nl = (uint32_t)j->limbs.size();
    if (nl > det->cap || (nl > 0 && !det->limbs)) {
        det->nlimbs = nl;
        set_last_error("poll: det needs %u limbs", nl);
        return IDET_ERR_BUFFER;  // the job is kept: poll again with room
    }
    det->sign = j->sign;
    det->nlimbs = nl;
    if (nl) memcpy(det->limbs, j->limbs.data(), 4 * (size_t)nl);
    S->jobs.erase(it);
    delete j;
    S->cv_done.notify_all();  // other pollers of this ticket see it is gone
    return IDET_OK;
}

void idet_server_info(idet_server *S, idet_server_stats *out) {
    if (!S || !out) return;
    std::lock_guard<std::mutex> lk(S->mu);
    out->queued = (int32_t)S->queue.size();
    out->running = S->running;
    out->max_running = S->max_running;
    out->bytes_in_use = S->in_use;
    out->budget = S->budget;
    out->admitted = S->admitted;
    out->completed = S->completed;
    out->groups = S->groups;
}

void idet_server_destroy(idet_server *S) {
    if (!S) return;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        // finish what was submitted
        S->cv_done.wait(lk, [&] { return S->queue.empty() && S->running == 0; });
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto &t : S->workers) t.join();
    for (auto &kv : S->jobs) delete kv.second;
    delete S;
}

}  // extern "C"
