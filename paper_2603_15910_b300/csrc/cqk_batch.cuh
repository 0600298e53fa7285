// cqk_batch.cuh -- the work queue of the batched persistent kernels.
//
// A batch of B instances lives back to back in the same arrays (instance i = elements
// [offsets[i], offsets[i+1])).  A planning kernel gives instance i a group of g_i blocks
// (about one block per `per_block` elements, at most kMaxGroup) and lists the instances
// longest first; the flattened list of (instance, member) slots is then handed out by one
// atomic cursor.  Slots are taken in order, so at any time only the most recently opened
// group can be waiting for members, and every block of the co-resident grid eventually takes
// one of its slots: with g_i <= grid size the groups cannot deadlock.  Every wait is bounded
// anyway (grid_barrier).
#pragma once

#include "cqk_block.cuh"

namespace cqk {

constexpr int kMaxGroup = 32;
constexpr size_t kInstPartBytes = 2ull * kPartialQ * kMaxGroup * sizeof(double);  // per instance

// Workspace of a batched call (all offsets from the workspace start, 256-byte aligned):
//   [0, 256)                 BatchHeader
//   inst headers             B x WsHeader (zeroed with the batch header before each launch)
//   plan                     order[B] (int32), gsize[B] (int32), prefix[B+1] (int64)
//   slot table               B x kMaxGroup int32: the plan position of every slot
//   partials                 B x kInstPartBytes
struct BatchHeader {
    unsigned long long cursor;  // next slot to hand out
    unsigned long long total;   // number of slots (written by the planner)
    unsigned long long large;   // slots of block groups; the slots after them are warp packs
    long long nlarge;           // instances solved by block groups (plan positions [0, nlarge))
    unsigned pad[56];
};
static_assert(sizeof(BatchHeader) == 256, "batch header must be 256 bytes");

struct BatchLayout {
    size_t hdr, inst_hdr, order, gsize, prefix, slots, part, total;
};
__host__ __device__ inline size_t align256(size_t x) { return (x + 255) / 256 * 256; }
__host__ __device__ inline BatchLayout batch_layout(int64_t B) {
    BatchLayout L;
    L.hdr = 0;
    L.inst_hdr = 256;
    L.order = align256(L.inst_hdr + (size_t)B * sizeof(WsHeader));
    L.gsize = align256(L.order + (size_t)B * 4);
    L.prefix = align256(L.gsize + (size_t)B * 4);
    L.slots = align256(L.prefix + (size_t)(B + 1) * 8);
    L.part = align256(L.slots + (size_t)B * kMaxGroup * 4);
    L.total = align256(L.part + (size_t)B * kInstPartBytes);
    return L;
}

struct BatchRefs {
    BatchHeader* bh;
    WsHeader* inst_hdr;
    int* order;
    int* gsize;
    long long* prefix;
    int* slots;
    double* part;
    __host__ __device__ static BatchRefs at(void* ws, int64_t B) {
        const BatchLayout L = batch_layout(B);
        char* p = static_cast<char*>(ws);
        BatchRefs R;
        R.bh = reinterpret_cast<BatchHeader*>(p + L.hdr);
        R.inst_hdr = reinterpret_cast<WsHeader*>(p + L.inst_hdr);
        R.order = reinterpret_cast<int*>(p + L.order);
        R.gsize = reinterpret_cast<int*>(p + L.gsize);
        R.prefix = reinterpret_cast<long long*>(p + L.prefix);
        R.slots = reinterpret_cast<int*>(p + L.slots);
        R.part = reinterpret_cast<double*>(p + L.part);
        return R;
    }
};

// One slot of the queue: the instance, this block's member index and the group size; or a
// pack of up to kWarpPack small instances, one per warp (plan positions pack_first + warp).
constexpr int kWarpPack = NWARP;
struct Slot {
    int inst, member, g;
    long long pack_first;  // -1 unless the slot is a warp pack
};

// Called by all threads of a block: the next slot, or inst = -1 when the queue is empty.
__device__ __forceinline__ Slot next_slot(const BatchRefs& R, int64_t B) {
    __shared__ Slot s_slot;
    if (threadIdx.x == 0) {
        const unsigned long long slot = atomicAdd(&R.bh->cursor, 1ull);
        const unsigned long long total = *(volatile unsigned long long*)&R.bh->total;
        const unsigned long long large = *(volatile unsigned long long*)&R.bh->large;
        Slot sl{-1, 0, 0, -1};
        if (slot < large) {
            const int p = R.slots[slot];  // plan position of the slot's instance
            sl.inst = R.order[p];
            sl.member = (int)(slot - (unsigned long long)R.prefix[p]);
            sl.g = R.gsize[p];
        } else if (slot < total) {
            sl.pack_first = *(volatile long long*)&R.bh->nlarge + (long long)(slot - large) * kWarpPack;
        }
        s_slot = sl;
    }
    __syncthreads();
    const Slot sl = s_slot;
    __syncthreads();
    return sl;
}

__device__ __forceinline__ Grp slot_group(const BatchRefs& R, const int64_t* offsets, const Slot& sl) {
    Grp gp;
    gp.member = sl.member;
    gp.g = sl.g;
    gp.sp = Span{offsets[sl.inst], offsets[sl.inst + 1]};
    gp.hdr = R.inst_hdr + sl.inst;
    gp.part = R.part + (size_t)sl.inst * (kInstPartBytes / sizeof(double));
    return gp;
}

// The info of an instance that is not solved (empty, or invalid per-instance arguments).
__device__ __forceinline__ void write_plain_info(cqk_info* info, int status, int stop, double r) {
    cqk_info inf;
    inf.lambda = 0.0;
    inf.residual = -r;
    inf.abs_bx = 0.0;
    inf.slope = 0.0;
    inf.lambda0 = 0.0;
    inf.nfree = 0;
    inf.iters = 0;
    inf.status = status;
    inf.passes = 0;
    inf.stop = stop;
    inf.nchunks = 0;
    inf.tile = 0;
    *info = inf;
}

}  // namespace cqk
