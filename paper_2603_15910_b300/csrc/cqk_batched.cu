// cqk_batched.cu -- planning of batched calls: every instance gets a group of blocks and the
// instances are queued longest first (cqk_batch.cuh describes the queue).
#include "cqk_batch.cuh"

namespace cqk {
namespace {

constexpr int kPlanThreads = 1024;

// inclusive warp scan of v; returns the warp total in `total`
__device__ __forceinline__ long long warp_incl_scan(long long v, long long& total) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    total = __shfl_sync(0xffffffffu, v, 31);
    return v;
}

// One block.  Buckets instances by floor(log2(length)) (longest first; the order inside a
// bucket only affects scheduling, never a result), gives each a group of
// clamp(ceil(length / per_block), 1, gmax) blocks, and writes the slot prefix sums.
// Instances shorter than 2^small_log2 (small_log2 > 0) are not given block groups: they form
// a suffix of the plan order and are handed out in packs of kWarpPack, one per warp.
__global__ void __launch_bounds__(kPlanThreads) plan_kernel(const int64_t* __restrict__ offsets, int64_t B,
                                                            int64_t per_block, int gmax, int small_log2,
                                                            BatchRefs R) {
    __shared__ unsigned hist[64], start[64], fill[64];
    __shared__ long long warp_tot[kPlanThreads / 32];
    __shared__ long long s_base, s_nlarge;
    const int tid = threadIdx.x;
    if (tid < 64) {
        hist[tid] = 0;
        fill[tid] = 0;
    }
    __syncthreads();
    for (int64_t i = tid; i < B; i += kPlanThreads) {
        const long long len = offsets[i + 1] - offsets[i];
        const int bk = len > 0 ? 63 - __clzll(len) : 0;
        atomicAdd(&hist[bk], 1u);
    }
    __syncthreads();
    if (tid == 0) {
        unsigned acc = 0;
        long long nl = 0;
        for (int b = 63; b >= 0; b--) {
            start[b] = acc;
            acc += hist[b];
            if (small_log2 <= 0 || b >= small_log2) nl += hist[b];
        }
        s_nlarge = nl;
    }
    __syncthreads();
    for (int64_t i = tid; i < B; i += kPlanThreads) {
        const long long len = offsets[i + 1] - offsets[i];
        const int bk = len > 0 ? 63 - __clzll(len) : 0;
        R.order[start[bk] + atomicAdd(&fill[bk], 1u)] = (int)i;
    }
    __syncthreads();
    if (tid == 0) s_base = 0;
    __syncthreads();
    const long long NL = s_nlarge;
    for (int64_t c = 0; c < NL; c += kPlanThreads) {
        const int64_t p = c + tid;
        long long g = 0;
        if (p < NL) {
            const int i = R.order[p];
            const long long len = offsets[i + 1] - offsets[i];
            g = (len + per_block - 1) / per_block;
            if (g < 1) g = 1;
            if (g > gmax) g = gmax;
            R.gsize[p] = (int)g;
        }
        long long wt;
        const long long incl = warp_incl_scan(g, wt);
        if ((tid & 31) == 31) warp_tot[tid >> 5] = wt;
        __syncthreads();
        long long before = 0;
        for (int w = 0; w < (tid >> 5); w++) before += warp_tot[w];
        if (p < NL) {
            const long long first = s_base + before + incl - g;
            R.prefix[p] = first;
            for (long long m = 0; m < g; m++) R.slots[first + m] = (int)p;
        }
        __syncthreads();
        if (tid == kPlanThreads - 1) {
            long long all = 0;
            for (int w = 0; w < kPlanThreads / 32; w++) all += warp_tot[w];
            s_base += all;
        }
        __syncthreads();
    }
    if (tid == 0) {
        R.prefix[NL] = s_base;
        R.bh->large = (unsigned long long)s_base;
        R.bh->nlarge = NL;
        R.bh->total = (unsigned long long)s_base + (unsigned long long)((B - NL + kWarpPack - 1) / kWarpPack);
        R.bh->cursor = 0ull;
    }
}

}  // namespace

#ifndef CQK_BATCH_ONLY
size_t batch_ws_bytes(int64_t B) { return batch_layout(B).total; }
#endif

int CQK_VFN(plan_batch)(const int64_t* offsets_dev, int64_t B, int64_t per_block, int gmax, void* ws, cudaStream_t s,
               int small_log2) {
    const BatchLayout L = batch_layout(B);
    cudaError_t e = cudaMemsetAsync(ws, 0, L.order, s);  // batch header + per-instance headers
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return CQK_CUDA_ERROR;
    }
    if (gmax > kMaxGroup) gmax = kMaxGroup;
    if (gmax < 1) gmax = 1;
    plan_kernel<<<1, kPlanThreads, 0, s>>>(offsets_dev, B, per_block, gmax, small_log2, BatchRefs::at(ws, B));
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return CQK_CUDA_ERROR;
    }
    return CQK_OK;
}

}  // namespace cqk
