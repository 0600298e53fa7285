// cqk_internal.h -- host-side declarations shared by the libcqk translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cqk.h"

// Kernel variants.  The batched kernels are compiled more than once, each build with its own
// block size (CQK_NT threads per block) or per-lane unroll (CQK_UNROLL_HALF: half of the
// vectors in flight per lane of the streaming loops); a variant build defines CQK_VARIANT to
// the suffix of its launchers (launch_general_batched_t512, ...) and CQK_BATCH_ONLY, which
// leaves out the single-instance kernels.  The default build (no suffix) has every kernel.
#ifndef CQK_NT
#define CQK_NT 256
#endif
#ifndef CQK_VARIANT
#define CQK_VARIANT
#endif
#define CQK_CAT2(a, b) a##b
#define CQK_CAT(a, b) CQK_CAT2(a, b)
#define CQK_VFN(name) CQK_CAT(name, CQK_VARIANT)

namespace cqk {

// machine epsilon^{3/4} of the stopping criteria (Sec. 4)
constexpr double kEps34F64 = 1.8189894035458565e-12;  // (2^-52)^{3/4}
constexpr double kEps34F32 = 6.4155306680183660e-06;  // (2^-23)^{3/4}

// Workspace header, at offset 0 of every workspace (zeroed before each launch).
struct WsHeader {
    unsigned bar_count;  // grid-barrier arrivals
    unsigned ticket;     // last-block-done ticket of the final pass
    int error;           // device-side error code (CQK_TIMEOUT) or 0
    unsigned flags;      // validation flags (bit 0: bad input)
    unsigned pad[60];
};
static_assert(sizeof(WsHeader) == 256, "header must be 256 bytes");

constexpr int kBlockThreads = CQK_NT;
static_assert(kBlockThreads == 128 || kBlockThreads == 256 || kBlockThreads == 512, "block size");
// blocks per SM the kernels are compiled for: 512 threads per SM (16 warps) at every block size,
// so every variant has the register budget of the 256-thread build (128 per thread)
constexpr int kMinBlocksPerSM = 512 / kBlockThreads;
constexpr int kMaxBlocks = 148 * 8;  // upper bound of any persistent grid
constexpr int kPartialQ = 8;         // doubles per block per pass
constexpr unsigned kFlagBadInput = 1u;

// bytes of workspace used by one persistent solve: header + 2 x kPartialQ x kMaxBlocks doubles
constexpr size_t kSingleWsBytes = sizeof(WsHeader) + 2ull * kPartialQ * kMaxBlocks * sizeof(double);

// Resolved options (defaults applied).
struct Opts {
    int max_iter;
    int init;
    double lambda0;
    int validate;
    int final_step;
    unsigned long long limit_ns;
    int max_blocks;
    int fault_inject;
    int64_t group_elems;   // batched calls: one block of an instance's group per this many elements
    int64_t condat_chunk;  // CQK_INIT_CONDAT: minimum elements per chunk
    const void* xbar;      // CQK_INIT_WARM: primal estimate
    int warp_log2;         // batched projections: instances shorter than 2^warp_log2 take one warp (0: none)
    int scan_warps;        // pipelined Alg. 2: chunks (scan warps) per block; 0 = automatic
    int block_threads;     // batched kernels: threads per block (128, 256 or 512)
    int unroll_half;       // batched kernels: 1 = the half-unroll build
};

Opts resolve_options(const cqk_options* opt, int dtype, int default_init);
void set_last_cuda_error(cudaError_t e);

// Launchers.  Each is defined by the default build; the batched ones (and the adjoint) also by
// the variant builds under the suffixes listed in CQK_FOR_VARIANTS.
int launch_simplex(int64_t n, int dtype, const void* y, double r, int l1, void* x, uint32_t* mask,
                   cqk_info* info, const Opts& o, void* ws, cudaStream_t s);
int launch_general(int64_t n, int dtype, const void* a, const void* b, const void* d, const void* l,
                   const void* u, double r, void* x, uint32_t* mask, cqk_info* info, const Opts& o,
                   void* ws, cudaStream_t s);
int launch_phi(int64_t n, int dtype, const void* a, const void* b, const void* d, const void* l,
               const void* u, double lambda, void* x, double* out, void* ws, cudaStream_t s);

// batched calls: default elements per block of an instance's group (at most kMaxGroup blocks)
constexpr int64_t kSimplexGroupElems = 1 << 20;
constexpr int64_t kGeneralGroupElems = 1 << 16;
constexpr int64_t kCondatChunkElems = 512;
constexpr int64_t kBackwardGroupElems = 1 << 15;  // general adjoint (projections: kSimplexGroupElems)
size_t batch_ws_bytes(int64_t B);

// Batched launchers and the adjoint, declared for the default build (suffix empty) and every
// variant build: _t128 and _t512 (128 / 512 threads per block; general batches and adjoints),
// _u (256 threads, half unroll; every batched kernel).  The planner is built with each, since
// the warp packs of small instances hold one instance per warp of the block.
#define CQK_DECLARE_BATCHED(sfx)                                                                                   \
    int plan_batch##sfx(const int64_t* offsets_dev, int64_t B, int64_t per_block, int gmax, void* ws,               \
                        cudaStream_t s, int small_log2 = 0);                                                        \
    int launch_simplex_batched##sfx(int64_t B, const int64_t* offsets, int dtype, const void* y, const double* r,  \
                                    int l1, void* x, uint32_t* mask, cqk_info* info, const Opts& o, void* ws,       \
                                    cudaStream_t s);                                                                \
    int launch_general_batched##sfx(int64_t B, const int64_t* offsets, int dtype, const void* a, const void* b,     \
                                    const void* d, const void* l, const void* u, const double* r, void* x,          \
                                    uint32_t* mask, cqk_info* info, const Opts& o, void* ws, cudaStream_t s);      \
    /* backward (kind 0 general, 1 simplex, 2 l1 ball); offsets == nullptr: one instance of n */                   \
    int launch_backward##sfx(int kind, int64_t B, const int64_t* offsets, int64_t n, int dtype, const void* g,     \
                             const void* x, const void* a, const void* b, const void* d, const void* l,            \
                             const void* u, const uint32_t* mask, const cqk_info* info, void* ga, void* gb,        \
                             void* gd, void* gl, void* gu, double* gr, int32_t* status, const Opts& o, void* ws,   \
                             cudaStream_t s);
CQK_DECLARE_BATCHED()
CQK_DECLARE_BATCHED(_t128)
CQK_DECLARE_BATCHED(_t512)
CQK_DECLARE_BATCHED(_u)

// number of co-resident blocks for a cooperative kernel, capped by max_blocks and by the work
int persistent_grid(const void* kernel, int threads, size_t smem, int64_t work_items, int max_blocks);

}  // namespace cqk
