// Synchronisation pieces shared by the persistent lifting kernels (k_lift.cu,
// k_lifte.cu): a grid-wide barrier among the consumer warps of a cooperative
// launch, mbarrier waits for a ring of shared-memory slots filled by bulk
// asynchronous copies, and L2 cache policies for those copies.
//
// Every wait is bounded by a cycle limit passed in by the launcher (about two
// seconds of SM clock by default; idet_set_wait_limit lowers it for the
// failure-detection tests). A wait that gives up records the first failure in
// the GridBar (code and place) and returns false; the other warps see the
// recorded error at their next poll and leave too. A producer that has
// issued copies drains them with the default limit before its CTA exits, so
// no copy is ever in flight into the shared memory of an exited block.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace idet {
namespace lift {

constexpr long long kDefaultWaitCycles = 4000000000ll;  // ~2 s at 2 GHz

struct GridBar {
    unsigned int count;  // arrivals, monotone within one launch
    int err;             // first failure: 1 grid barrier, 2 mbarrier, 3 a
                         // consumer gave up, 4 issue wait
    int info[6];         // where it happened: block, warp, seq, slot, parity, it
};

// Record the first failure only.
__device__ __forceinline__ void fail_once(GridBar *gb, int code, int warp, long long seq, int slot,
                                          unsigned par, int it) {
    if (atomicCAS(&gb->err, 0, code) == 0) {
        gb->info[0] = blockIdx.x;
        gb->info[1] = warp;
        gb->info[2] = (int)seq;
        gb->info[3] = slot;
        gb->info[4] = (int)par;
        gb->info[5] = it;
    }
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t addr, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the completion of the phase of parity `parity`; false after the
// time limit or when another block has recorded an error.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, GridBar *gb,
                                          long long limit, long long seq = -1, int slot = -1,
                                          int it = -1) {
    const uint32_t addr = smem_u32(bar);
    const long long t0 = clock64();
    for (unsigned i = 0;; ++i) {
        if (mbar_test(addr, parity)) return true;
        if ((i & 255) == 255) {
            if (*((volatile int *)&gb->err)) return false;
            if (clock64() - t0 > limit) {
                fail_once(gb, 2, threadIdx.x >> 5, seq, slot, parity, it);
                return false;
            }
        }
    }
}

// Wait until the producer has issued sequence number seq. An mbarrier parity
// wait only tells the current phase from the previous one, so a consumer may
// wait on a slot's barrier only once the copy it needs has been issued (the
// slot's barrier is then at most one phase away from it).
__device__ __forceinline__ bool wait_issued(const volatile unsigned int *issued, long long seq,
                                            GridBar *gb, long long limit, int slot, int it) {
    const long long t0 = clock64();
    for (unsigned i = 0; (long long)*issued <= seq; ++i) {
        if ((i & 255) == 255) {
            if (*((volatile int *)&gb->err)) return false;
            if (clock64() - t0 > limit) {
                fail_once(gb, 4, threadIdx.x >> 5, seq, slot, 0, it);
                return false;
            }
        }
    }
    return true;
}

// The producer's last duty: wait (default limit) for the final phase of
// every slot it used, so that no copy is in flight when the block exits.
// seq = copies issued, S = slots.
__device__ __forceinline__ void drain_ring(uint64_t *full, int S, long long seq) {
    for (int s = 0; s < S && s < seq; ++s) {
        const long long q = seq - 1 - ((seq - 1 - s) % S);
        const uint32_t addr = smem_u32(&full[s]);
        const unsigned par = (unsigned)((q / S) & 1);
        const long long t0 = clock64();
        while (!mbar_test(addr, par) && clock64() - t0 <= kDefaultWaitCycles) {
        }
    }
}

// Bulk copy global -> shared completing on an mbarrier, with an L2 policy.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         uint64_t *bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
        "[%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// Named barrier among the first `threads` threads of the block.
template <int kThreads> __device__ __forceinline__ void cons_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(kThreads) : "memory");
}

// Grid-wide barrier among the consumer warps of all CTAs: the b-th barrier
// completes when count reaches b * gridDim.x.
template <int kThreads>
__device__ __forceinline__ bool grid_sync(GridBar *gb, unsigned target, long long limit) {
    cons_sync<kThreads>();
    if (threadIdx.x == 0) {
        // arrive with release semantics (cumulative over the consumer
        // threads' writes ordered before it by the CTA barrier), poll with
        // acquire loads and a short back-off
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&gb->count) : "memory");
        volatile int *ve = &gb->err;
        const long long t0 = clock64();
        while (true) {
            unsigned c;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(c) : "l"(&gb->count) : "memory");
            if (c >= target) break;
            if (*ve) break;
            if (clock64() - t0 > limit) {
                fail_once(gb, 1, 0, target, -1, 0, -1);
                break;
            }
            __nanosleep(20);
        }
    }
    cons_sync<kThreads>();
    return *((volatile int *)&gb->err) == 0;
}

__device__ __forceinline__ int64_t warp_sum64(int64_t v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace lift

// Cycle limit of the lifting kernels' waits (idet_set_wait_limit; 0 = the
// default). Defined in k_lift.cu.
long long lift_wait_cycles();

}  // namespace idet
