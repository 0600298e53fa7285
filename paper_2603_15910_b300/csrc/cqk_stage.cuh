// cqk_stage.cuh -- bulk-copy (TMA) staging of contiguous tiles into shared memory.
//
// A block walks its tiles (tile c = blockIdx.x + i*gridDim.x) with a ring of kStages shared
// memory stages.  Thread 0 issues one cp.async.bulk per array and tile, completing on the
// stage's mbarrier; the block computes on tile i while tile i + kStages - 1 is in flight.
// This keeps the memory system busy during the long double-float compute phase of the
// general map-reduce, which plain loads (consumed right after issue) could not.
//
// Rules kept here: every bulk copy starts and ends on 16-byte boundaries (arrays must be
// 16-byte aligned; a tile's tail that is not a multiple of 16 bytes is read with ordinary
// loads by the consumer); every mbarrier wait is bounded by a time limit, after which the
// error flag is raised and the wait continues (bounded again) so that no bulk copy is still
// writing into shared memory when the block leaves.
#pragma once

#include "cqk_device.cuh"

namespace cqk {

constexpr int kStages = 2;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the completion of phase `parity` of `bar`.  On expiry the error flag is
// set and the wait goes on for up to another `limit_ns` (the copies of this block must land
// before it can leave); returns false if the barrier never completed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int* error, unsigned long long limit_ns,
                                          int timeout_code) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    bool flagged = false;
    while (!mbar_try_wait(bar, parity)) {
        const unsigned long long dt = globaltimer_ns() - t0;
        if (!flagged && dt > limit_ns) {
            atomicExch(error, timeout_code);
            flagged = true;
        }
        if (dt > 2 * limit_ns) return false;
    }
    return true;
}

// The tiles of one block over n elements of NA arrays of T, tile = TT elements.
template <typename T, int NA, int TT>
struct TileRing {
    T* buf;              // dynamic shared memory: [kStages][NA][TT]
    uint64_t* bar;       // kStages mbarriers
    unsigned parity;     // bit s: parity of the next completion of stage s
    int64_t n, ntiles, first, step, count;

    __device__ __forceinline__ void setup(int64_t n_, T* buf_, uint64_t* bar_) {
        buf = buf_;
        bar = bar_;
        n = n_;
        ntiles = (n + TT - 1) / TT;
        first = blockIdx.x;
        step = gridDim.x;
        count = first < ntiles ? (ntiles - first + step - 1) / step : 0;
    }
    __device__ __forceinline__ int64_t tile(int64_t i, bool rev) const { return first + (rev ? count - 1 - i : i) * step; }
    __device__ __forceinline__ T* stage(int s, int a) const { return buf + ((size_t)s * NA + a) * TT; }
    // number of leading elements of tile c delivered by the bulk copy (a multiple of 16 bytes)
    __device__ __forceinline__ int staged(int64_t c) const {
        const int64_t cnt = n - c * TT < TT ? n - c * TT : TT;
        return (int)((cnt * (int64_t)sizeof(T)) / 16 * 16 / (int64_t)sizeof(T));
    }
    // thread 0: start the copies of tile c into stage s
    __device__ __forceinline__ void issue(int64_t c, int s, const T* const* src) const {
        const int m = staged(c);
        const uint32_t bytes = (uint32_t)m * sizeof(T);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(&bar[s], bytes * NA);
        if (bytes)
#pragma unroll
            for (int a = 0; a < NA; a++) bulk_g2s(stage(s, a), src[a] + c * TT, bytes, &bar[s]);
    }
};

}  // namespace cqk
