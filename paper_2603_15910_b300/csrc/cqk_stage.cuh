// cqk_stage.cuh -- bulk-copy (TMA) staging of contiguous tiles into shared memory.
//
// A block of a group walks its tiles (tile c = first tile of the span + member + i*g) with a
// ring of shared-memory stages.  One thread issues one cp.async.bulk per array and tile,
// completing on the stage's mbarrier; the block computes on tile i while the next tiles are
// in flight.  This keeps the memory system busy during the long double-float compute phase
// of the general map-reduce, the scan of the Alg. 2 start and the simplex adjoint, which
// plain loads (consumed right after issue, held in registers) could not.
//
// Rules kept here: every bulk copy starts and ends on 16-byte boundaries (arrays must be
// 16-byte aligned; a tile's tail that is not a multiple of 16 bytes is read with ordinary
// loads by the consumer); every mbarrier wait is bounded by a time limit, after which the
// error flag is raised and the wait continues (bounded again) so that no bulk copy is still
// writing into shared memory when the block leaves.
#pragma once

#include "cqk_block.cuh"

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
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_cnt(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
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

// try_wait with a suspend-time hint: the thread may be suspended until the phase completes or
// about `hint_ns` pass, instead of polling (a polling warp takes issue slots from the warps of
// its SM sub-partition)
__device__ __forceinline__ bool mbar_try_wait_suspend(uint64_t* bar, unsigned parity, unsigned hint_ns) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
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
    while (!mbar_try_wait_suspend(bar, parity, 1000u)) {
        const unsigned long long dt = globaltimer_ns() - t0;
        if (!flagged && dt > limit_ns) {
            atomicExch(error, timeout_code);
            flagged = true;
        }
        if (dt > 2 * limit_ns) return false;
    }
    return true;
}

// The tiles of one group member over a span of NA arrays of T (16-byte aligned at element
// 0): tile c holds the global elements [c*TT, (c+1)*TT); the span's tiles are shared out
// round-robin among the g members.  The bulk copy of tile c delivers the elements
// [b0, b1) = [c*TT, (c+1)*TT) intersected with the span rounded inwards to 16 bytes; smem
// position of element e is e - c*TT.  Other elements of the span are read directly.
template <typename T, int NA, int TT>
struct TileRing {
    T* buf;              // dynamic shared memory: [kStages][NA][TT]
    uint64_t* bar;       // kStages mbarriers
    unsigned parity;     // bit s: parity of the next completion of stage s
    int64_t slo, shi;    // the span rounded inwards to 16-byte boundaries
    int64_t first, step, count;

    __device__ __forceinline__ void setup(int64_t lo, int64_t hi, T* buf_, uint64_t* bar_, int member, int g) {
        constexpr int64_t E = 16 / sizeof(T);
        buf = buf_;
        bar = bar_;
        slo = (lo + E - 1) / E * E;
        shi = hi / E * E;
        if (shi < slo) shi = slo;
        const int64_t c0 = lo / TT, c1 = (hi + TT - 1) / TT;
        first = c0 + member;
        step = g;
        count = first < c1 ? (c1 - first + step - 1) / step : 0;
    }
    __device__ __forceinline__ int64_t tile(int64_t i, bool rev) const { return first + (rev ? count - 1 - i : i) * step; }
    __device__ __forceinline__ T* stage(int s, int a) const { return buf + ((size_t)s * NA + a) * TT; }
    __device__ __forceinline__ int64_t b0(int64_t c) const { return c * TT > slo ? c * TT : slo; }
    __device__ __forceinline__ int64_t b1(int64_t c) const { return (c + 1) * TT < shi ? (c + 1) * TT : shi; }
    // called by every thread: lane 0 of warp w starts the copies of arrays w, w + NWARP, ... of
    // tile c into stage s (warp 0 also registers the stage's bytes), so that the issue cost is
    // spread over the warps instead of delaying one
    __device__ __forceinline__ void issue_by_warps(int64_t c, int s, const T* const* src) const {
        const int w = threadIdx.x >> 5;
        if ((threadIdx.x & 31) != 0 || w >= NA) return;
        const int64_t lo = b0(c), hi = b1(c);
        const uint32_t bytes = hi > lo ? (uint32_t)((hi - lo) * (int64_t)sizeof(T)) : 0u;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (w == 0) mbar_arrive_expect_tx(&bar[s], bytes * NA);
        if (bytes)
            for (int a = w; a < NA; a += NWARP) bulk_g2s(stage(s, a) + (lo - c * TT), src[a] + lo, bytes, &bar[s]);
    }
    // thread 0: start the copies of tile c into stage s
    __device__ __forceinline__ void issue(int64_t c, int s, const T* const* src) const {
        const int64_t lo = b0(c), hi = b1(c);
        const uint32_t bytes = hi > lo ? (uint32_t)((hi - lo) * (int64_t)sizeof(T)) : 0u;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(&bar[s], bytes * NA);
        if (bytes)
#pragma unroll
            for (int a = 0; a < NA; a++) bulk_g2s(stage(s, a) + (lo - c * TT), src[a] + lo, bytes, &bar[s]);
    }
};

}  // namespace cqk
