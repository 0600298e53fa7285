// cqk_internal.h -- host-side declarations shared by the libcqk translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cqk.h"

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

constexpr int kBlockThreads = 256;
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
};

Opts resolve_options(const cqk_options* opt, int dtype, int default_init);
void set_last_cuda_error(cudaError_t e);

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
int plan_batch(const int64_t* offsets_dev, int64_t B, int64_t per_block, int gmax, void* ws, cudaStream_t s,
               int small_log2 = 0);
int launch_simplex_batched(int64_t B, const int64_t* offsets, int dtype, const void* y, const double* r, int l1,
                           void* x, uint32_t* mask, cqk_info* info, const Opts& o, void* ws, cudaStream_t s);
int launch_general_batched(int64_t B, const int64_t* offsets, int dtype, const void* a, const void* b,
                           const void* d, const void* l, const void* u, const double* r, void* x, uint32_t* mask,
                           cqk_info* info, const Opts& o, void* ws, cudaStream_t s);

// backward (kind 0 general, 1 simplex, 2 l1 ball); offsets == nullptr: one instance of n
int launch_backward(int kind, int64_t B, const int64_t* offsets, int64_t n, int dtype, const void* g, const void* x,
                    const void* a, const void* b, const void* d, const void* l, const void* u, const uint32_t* mask,
                    const cqk_info* info, void* ga, void* gb, void* gd, void* gl, void* gu, double* gr,
                    int32_t* status, const Opts& o, void* ws, cudaStream_t s);

// number of co-resident blocks for a cooperative kernel, capped by max_blocks and by the work
int persistent_grid(const void* kernel, int threads, size_t smem, int64_t work_items, int max_blocks);

}  // namespace cqk
