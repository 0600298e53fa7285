// cqk_api.cu -- the extern "C" entry points of libcqk (declared in include/cqk.h): host-side
// argument checks, option defaults, workspace sizing and grid sizing.  All compute is in the
// kernels of cqk_simplex.cu and cqk_general.cu.
#include <string.h>

#include "cqk_internal.h"

#include <stddef.h>

static_assert(sizeof(cqk_options) == 72, "cqk_options layout is part of the ABI");
static_assert(offsetof(cqk_options, xbar) == 48, "cqk_options layout is part of the ABI");
static_assert(sizeof(cqk_info) == 72, "cqk_info layout is part of the ABI");

namespace cqk {

static thread_local int g_last_cuda_error = 0;
void set_last_cuda_error(cudaError_t e) { g_last_cuda_error = (int)e; }

Opts resolve_options(const cqk_options* opt, int dtype, int default_init) {
    (void)dtype;
    cqk_options d;
    cqk_default_options(&d);
    if (opt) d = *opt;
    Opts o;
    o.max_iter = d.max_iter > 0 ? d.max_iter : 100;
    o.init = d.init >= 0 ? d.init : default_init;
    o.lambda0 = d.lambda0;
    o.validate = d.validate != 0;
    o.final_step = d.final_step != 0;
    o.limit_ns = (unsigned long long)(d.spin_limit_us > 0 ? d.spin_limit_us : 2000000) * 1000ull;
    o.max_blocks = d.max_blocks > 0 ? d.max_blocks : 0;
    o.fault_inject = d.fault_inject;
    o.group_elems = d.group_elems > 0 ? d.group_elems : 0;
    o.condat_chunk = d.condat_chunk > 0 ? d.condat_chunk : kCondatChunkElems;
    o.xbar = d.xbar;
    // warp_elems: 0 -> 16384 (default), < 0 -> no warp-level instances, else rounded down to 2^k
    if (d.warp_elems < 0) {
        o.warp_log2 = 0;
    } else {
        const long long we = d.warp_elems > 0 ? d.warp_elems : 16384;
        int lg = 0;
        while ((2ll << lg) <= we && lg < 30) lg++;
        o.warp_log2 = lg;
    }
    // scan_warps: 0 (automatic) or 1, 2, 4 (other positive values round down to one of these)
    o.scan_warps = d.scan_warps >= 4 ? 4 : d.scan_warps >= 2 ? 2 : d.scan_warps >= 1 ? 1 : 0;
    o.block_threads = d.block_threads == 0 ? 256 : d.block_threads;  // checked by the entry points
    o.unroll_half = d.unroll;
    return o;
}

int persistent_grid(const void* kernel, int threads, size_t smem, int64_t work_items, int max_blocks) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { set_last_cuda_error(e); return -1; }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) { set_last_cuda_error(e); return -1; }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (e != cudaSuccess) { set_last_cuda_error(e); return -1; }
    if (per_sm < 1) return -1;
    int64_t g = (int64_t)sms * per_sm;
    if (g > kMaxBlocks) g = kMaxBlocks;
    // at least ~8 vectors per thread and pass before another block is added
    int64_t want = (work_items + (int64_t)threads * 8 - 1) / ((int64_t)threads * 8);
    if (want < 1) want = 1;
    if (g > want) g = want;
    if (max_blocks > 0 && g > max_blocks) g = max_blocks;
    return (int)g;
}

}  // namespace cqk

using namespace cqk;

// Single-instance calls have one build of each kernel (256 threads, full unroll).
static bool single_variant_ok(const Opts& o) { return o.block_threads == 256 && o.unroll_half == 0; }

// The build of the batched kernels selected by (block_threads, unroll): the default build, the
// 128- and 512-thread builds (general batches and adjoints only) or the half-unroll build.
enum Variant { kVarDefault, kVarT128, kVarT512, kVarHalf, kVarNone };
static Variant pick_variant(const Opts& o, bool projection_forward) {
    if (o.unroll_half == 0 && o.block_threads == 256) return kVarDefault;
    if (o.unroll_half == 1 && o.block_threads == 256) return kVarHalf;
    if (o.unroll_half == 0 && !projection_forward && o.block_threads == 128) return kVarT128;
    if (o.unroll_half == 0 && !projection_forward && o.block_threads == 512) return kVarT512;
    return kVarNone;
}

static bool ws_ok(const void* ws, size_t bytes, size_t need) { return ws && bytes >= need && ((uintptr_t)ws % 256) == 0; }

extern "C" {

void cqk_default_options(cqk_options* opt) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->max_iter = 100;
    opt->init = -1;
    opt->lambda0 = 0.0;
    opt->validate = 1;
    opt->final_step = 1;
    opt->spin_limit_us = 2000000;
    opt->max_blocks = 0;
    opt->fault_inject = 0;
}

size_t cqk_workspace_bytes(int64_t n_total, int32_t batch, int32_t dtype) {
    if (n_total < 0 || batch < 1 || (dtype != CQK_F64 && dtype != CQK_F32)) return 0;
    const size_t bb = batch_ws_bytes(batch);
    return bb > kSingleWsBytes ? bb : kSingleWsBytes;
}

int cqk_solve(int64_t n, int32_t dtype, const void* a, const void* b, const void* d, const void* l, const void* u,
              double r, void* x, uint32_t* free_mask, cqk_info* info_dev, const cqk_options* opt, void* workspace,
              size_t ws_bytes, void* stream) {
    if (n < 0 || (dtype != CQK_F64 && dtype != CQK_F32) || !info_dev) return CQK_BAD_ARG;
    if (n > 0 && (!a || !b || !d || !l || !u || !x)) return CQK_BAD_ARG;
    if (!ws_ok(workspace, ws_bytes, kSingleWsBytes)) return CQK_BAD_ARG;
    if (r != r) return CQK_BAD_ARG;
    Opts o = resolve_options(opt, dtype, CQK_INIT_FORMULA);
    if (!single_variant_ok(o)) return CQK_BAD_ARG;
    if (o.init != CQK_INIT_FORMULA && o.init != CQK_INIT_GIVEN && o.init != CQK_INIT_WARM) return CQK_BAD_ARG;
    if (o.init == CQK_INIT_WARM && !o.xbar && n > 0) return CQK_BAD_ARG;
    if (n == 0) {
        cqk_info inf;
        memset(&inf, 0, sizeof(inf));
        inf.status = (r == 0.0) ? CQK_OK : CQK_INFEASIBLE;
        inf.residual = -r;
        cudaError_t e = cudaMemcpyAsync(info_dev, &inf, sizeof(inf), cudaMemcpyHostToDevice, (cudaStream_t)stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) { set_last_cuda_error(e); return CQK_CUDA_ERROR; }
        return CQK_OK;
    }
    return launch_general(n, dtype, a, b, d, l, u, r, x, free_mask, info_dev, o, workspace, (cudaStream_t)stream);
}

int cqk_phi(int64_t n, int32_t dtype, const void* a, const void* b, const void* d, const void* l, const void* u,
            double lambda, void* x, double* out_dev, void* workspace, size_t ws_bytes, void* stream) {
    if (n <= 0 || (dtype != CQK_F64 && dtype != CQK_F32) || !out_dev) return CQK_BAD_ARG;
    if (!a || !b || !d || !l || !u) return CQK_BAD_ARG;
    if (!ws_ok(workspace, ws_bytes, kSingleWsBytes)) return CQK_BAD_ARG;
    return launch_phi(n, dtype, a, b, d, l, u, lambda, x, out_dev, workspace, (cudaStream_t)stream);
}

static int project(int64_t n, int32_t dtype, const void* y, double r, void* x, uint32_t* mask, cqk_info* info,
                   const cqk_options* opt, void* ws, size_t ws_bytes, void* stream, int l1) {
    if (n <= 0 || (dtype != CQK_F64 && dtype != CQK_F32) || !y || !x || !info) return CQK_BAD_ARG;
    if (!(r > 0.0) || !(r < INFINITY)) return CQK_BAD_ARG;
    if (x == y) return CQK_BAD_ARG;
    if (!ws_ok(ws, ws_bytes, kSingleWsBytes)) return CQK_BAD_ARG;
    Opts o = resolve_options(opt, dtype, CQK_INIT_CONDAT);
    if (!single_variant_ok(o)) return CQK_BAD_ARG;
    if (o.init != CQK_INIT_FORMULA && o.init != CQK_INIT_CONDAT && o.init != CQK_INIT_GIVEN && o.init != CQK_INIT_WARM)
        return CQK_BAD_ARG;
    if (o.init == CQK_INIT_WARM && !o.xbar) return CQK_BAD_ARG;
    return launch_simplex(n, dtype, y, r, l1, x, mask, info, o, ws, (cudaStream_t)stream);
}

int cqk_project_simplex(int64_t n, int32_t dtype, const void* y, double r, void* x, uint32_t* free_mask,
                        cqk_info* info_dev, const cqk_options* opt, void* workspace, size_t ws_bytes, void* stream) {
    return project(n, dtype, y, r, x, free_mask, info_dev, opt, workspace, ws_bytes, stream, 0);
}

int cqk_project_l1(int64_t n, int32_t dtype, const void* y, double r, void* x, uint32_t* free_mask,
                   cqk_info* info_dev, const cqk_options* opt, void* workspace, size_t ws_bytes, void* stream) {
    return project(n, dtype, y, r, x, free_mask, info_dev, opt, workspace, ws_bytes, stream, 1);
}

static int batched(int32_t B, const int64_t* offsets, int32_t dtype, const void* a, const void* b, const void* d,
                   const void* l, const void* u, const double* r, void* x, uint32_t* mask, cqk_info* info,
                   const cqk_options* opt, void* ws, size_t ws_bytes, void* stream, int kind) {
    // kind: 0 general, 1 simplex, 2 l1 ball
    if (B < 0 || (dtype != CQK_F64 && dtype != CQK_F32)) return CQK_BAD_ARG;
    if (B == 0) return CQK_OK;
    if (!offsets || !a || !r || !x || !info) return CQK_BAD_ARG;
    if (kind == 0 && (!b || !d || !l || !u)) return CQK_BAD_ARG;
    if (kind != 0 && x == a) return CQK_BAD_ARG;
    if (!ws_ok(ws, ws_bytes, batch_ws_bytes(B))) return CQK_BAD_ARG;
    Opts o = resolve_options(opt, dtype, kind == 0 ? CQK_INIT_FORMULA : CQK_INIT_CONDAT);
    if (o.init == CQK_INIT_WARM && !o.xbar) return CQK_BAD_ARG;
    const Variant v = pick_variant(o, kind != 0);
    if (v == kVarNone) return CQK_BAD_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (kind == 0) {
        if (o.init != CQK_INIT_FORMULA && o.init != CQK_INIT_GIVEN && o.init != CQK_INIT_WARM) return CQK_BAD_ARG;
        switch (v) {
            case kVarT128: return launch_general_batched_t128(B, offsets, dtype, a, b, d, l, u, r, x, mask, info, o, ws, s);
            case kVarT512: return launch_general_batched_t512(B, offsets, dtype, a, b, d, l, u, r, x, mask, info, o, ws, s);
            case kVarHalf: return launch_general_batched_u(B, offsets, dtype, a, b, d, l, u, r, x, mask, info, o, ws, s);
            default: return launch_general_batched(B, offsets, dtype, a, b, d, l, u, r, x, mask, info, o, ws, s);
        }
    }
    if (o.init != CQK_INIT_FORMULA && o.init != CQK_INIT_CONDAT && o.init != CQK_INIT_GIVEN && o.init != CQK_INIT_WARM)
        return CQK_BAD_ARG;
    if (v == kVarHalf) return launch_simplex_batched_u(B, offsets, dtype, a, r, kind == 2, x, mask, info, o, ws, s);
    return launch_simplex_batched(B, offsets, dtype, a, r, kind == 2, x, mask, info, o, ws, s);
}

int cqk_solve_batched(int32_t B, const int64_t* offsets_dev, int32_t dtype, const void* a, const void* b,
                      const void* d, const void* l, const void* u, const double* r_dev, void* x, uint32_t* free_mask,
                      cqk_info* info_dev, const cqk_options* opt, void* workspace, size_t ws_bytes, void* stream) {
    if (!b && !d && !l && !u)  // simplex batch on y = a (b = d = 1, l = 0, u = +inf)
        return batched(B, offsets_dev, dtype, a, b, d, l, u, r_dev, x, free_mask, info_dev, opt, workspace, ws_bytes,
                       stream, 1);
    return batched(B, offsets_dev, dtype, a, b, d, l, u, r_dev, x, free_mask, info_dev, opt, workspace, ws_bytes, stream,
                   0);
}

int cqk_project_simplex_batched(int32_t B, const int64_t* offsets_dev, int32_t dtype, const void* y,
                                const double* r_dev, void* x, uint32_t* free_mask, cqk_info* info_dev,
                                const cqk_options* opt, void* workspace, size_t ws_bytes, void* stream) {
    return batched(B, offsets_dev, dtype, y, nullptr, nullptr, nullptr, nullptr, r_dev, x, free_mask, info_dev, opt,
                   workspace, ws_bytes, stream, 1);
}

int cqk_project_l1_batched(int32_t B, const int64_t* offsets_dev, int32_t dtype, const void* y, const double* r_dev,
                           void* x, uint32_t* free_mask, cqk_info* info_dev, const cqk_options* opt, void* workspace,
                           size_t ws_bytes, void* stream) {
    return batched(B, offsets_dev, dtype, y, nullptr, nullptr, nullptr, nullptr, r_dev, x, free_mask, info_dev, opt,
                   workspace, ws_bytes, stream, 2);
}

static int backward(int kind, int32_t B, const int64_t* offsets, int64_t n, int32_t dtype, const void* g,
                    const void* x, const void* a, const void* b, const void* d, const void* l, const void* u,
                    const uint32_t* mask, const cqk_info* info, void* ga, void* gb, void* gd, void* gl, void* gu,
                    double* gr, int32_t* status, const cqk_options* opt, void* ws, size_t ws_bytes, void* stream) {
    if (B < 0 || (dtype != CQK_F64 && dtype != CQK_F32) || !info) return CQK_BAD_ARG;
    if (!offsets && (B != 1 || n < 0)) return CQK_BAD_ARG;
    if (B == 0 || (!offsets && n == 0)) return CQK_OK;
    if (!g || !x) return CQK_BAD_ARG;
    if (kind == 0 && (!b || !d)) return CQK_BAD_ARG;
    if (kind == 0 && (!mask || gl || gu) && (!l || !u)) return CQK_BAD_ARG;
    const size_t need = offsets ? batch_ws_bytes(B) : kSingleWsBytes;
    if (!ws_ok(ws, ws_bytes, need)) return CQK_BAD_ARG;
    Opts o = resolve_options(opt, dtype, CQK_INIT_FORMULA);
    const Variant v = offsets ? pick_variant(o, false) : (single_variant_ok(o) ? kVarDefault : kVarNone);
    cudaStream_t s = (cudaStream_t)stream;
    switch (v) {
        case kVarNone: return CQK_BAD_ARG;
        case kVarT128:
            return launch_backward_t128(kind, B, offsets, n, dtype, g, x, a, b, d, l, u, mask, info, ga, gb, gd, gl,
                                        gu, gr, status, o, ws, s);
        case kVarT512:
            return launch_backward_t512(kind, B, offsets, n, dtype, g, x, a, b, d, l, u, mask, info, ga, gb, gd, gl,
                                        gu, gr, status, o, ws, s);
        case kVarHalf:
            return launch_backward_u(kind, B, offsets, n, dtype, g, x, a, b, d, l, u, mask, info, ga, gb, gd, gl, gu,
                                     gr, status, o, ws, s);
        default:
            return launch_backward(kind, B, offsets, n, dtype, g, x, a, b, d, l, u, mask, info, ga, gb, gd, gl, gu,
                                   gr, status, o, ws, s);
    }
}

int cqk_backward(int32_t B, const int64_t* offsets_dev, int64_t n, int32_t dtype, const void* g, const void* x,
                 const void* a, const void* b, const void* d, const void* l, const void* u,
                 const uint32_t* free_mask, const cqk_info* info_dev, void* ga, void* gb, void* gd, void* gl,
                 void* gu, double* gr_dev, int32_t* status_dev, const cqk_options* opt, void* workspace,
                 size_t ws_bytes, void* stream) {
    return backward(0, B, offsets_dev, n, dtype, g, x, a, b, d, l, u, free_mask, info_dev, ga, gb, gd, gl, gu, gr_dev,
                    status_dev, opt, workspace, ws_bytes, stream);
}

int cqk_backward_simplex(int32_t B, const int64_t* offsets_dev, int64_t n, int32_t dtype, const void* g,
                         const void* x, const uint32_t* free_mask, const cqk_info* info_dev, void* gy,
                         double* gr_dev, int32_t* status_dev, const cqk_options* opt, void* workspace,
                         size_t ws_bytes, void* stream) {
    return backward(1, B, offsets_dev, n, dtype, g, x, nullptr, nullptr, nullptr, nullptr, nullptr, free_mask,
                    info_dev, gy, nullptr, nullptr, nullptr, nullptr, gr_dev, status_dev, opt, workspace, ws_bytes,
                    stream);
}

int cqk_backward_l1(int32_t B, const int64_t* offsets_dev, int64_t n, int32_t dtype, const void* g, const void* x,
                    const uint32_t* free_mask, const cqk_info* info_dev, void* gy, double* gr_dev,
                    int32_t* status_dev, const cqk_options* opt, void* workspace, size_t ws_bytes, void* stream) {
    return backward(2, B, offsets_dev, n, dtype, g, x, nullptr, nullptr, nullptr, nullptr, nullptr, free_mask,
                    info_dev, gy, nullptr, nullptr, nullptr, nullptr, gr_dev, status_dev, opt, workspace, ws_bytes,
                    stream);
}

const char* cqk_status_string(int status) {
    switch (status) {
        case CQK_OK: return "ok";
        case CQK_INFEASIBLE: return "infeasible";
        case CQK_MAXITER: return "maxiter";
        case CQK_BAD_INPUT: return "bad_input";
        case CQK_NONDIFF: return "nondiff";
        case CQK_TIMEOUT: return "timeout";
        case CQK_CUDA_ERROR: return "cuda_error";
        case CQK_BAD_ARG: return "bad_arg";
        default: return "unknown";
    }
}

int cqk_last_cuda_error(void) { return g_last_cuda_error; }

int cqk_version(void) { return 300; }  // 0.3.0: options block_threads and unroll

}  // extern "C"
