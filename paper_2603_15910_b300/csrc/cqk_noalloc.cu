// cqk_noalloc.cu -- simplex projection for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc when they need a projection: a plugin whose host
// application owns the device allocator, or a real-time loop whose device memory is fixed at
// start-up and may not grow.  They cannot provide the workspace that cqk_project_simplex
// takes.  cqk_project_simplex_noalloc runs the same projection kernel with its scratch (grid
// barrier counter, error flag and per-block partial sums) in the file-scope device array
// below.  The array exists on every GPU that loads the library, for the life of the
// process; it is shared by every call on that device.
#include <mutex>

#include "cqk_internal.h"

namespace {

// Scratch for one projection: the 256-byte header plus two parities of kPartialQ doubles
// for at most kNoAllocMaxBlocks blocks (76,032 bytes).
constexpr int kNoAllocMaxBlocks = CQK_NOALLOC_MAX_BLOCKS;
constexpr size_t kNoAllocBytes = sizeof(cqk::WsHeader) + 2ull * cqk::kPartialQ * kNoAllocMaxBlocks * sizeof(double);
static_assert(kNoAllocBytes == CQK_NOALLOC_SCRATCH_BYTES, "header constant out of date");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch per CUDA context.  In host code the array's name is
// only a host-side stand-in, so the address is looked up (cudaGetSymbolAddress) with the
// device current, once per context -- normally once per device, in its primary context --
// and passed to the kernel.  Keying on the context rather than the device ordinal keeps the
// address right for a host that runs its own context on the device.  The current context is
// read through the driver's cuCtxGetCurrent, reached via the runtime's entry-point query so
// that the library does not link the driver library directly.
typedef int (*CtxGetCurrentFn)(void**);
struct Entry {
    void* ctx;
    int dev;
    void* addr;
};
constexpr int kMaxEntries = 64;
std::mutex g_mu;
Entry g_tab[kMaxEntries];
int g_count = 0, g_next = 0;
CtxGetCurrentFn g_ctx_get = nullptr;
bool g_ctx_resolved = false;

void* current_context() {
    if (!g_ctx_resolved) {
        g_ctx_resolved = true;
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get = reinterpret_cast<CtxGetCurrentFn>(fn);
    }
    void* ctx = nullptr;
    if (g_ctx_get && g_ctx_get(&ctx) != 0) ctx = nullptr;
    return ctx;
}

int scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cqk::set_last_cuda_error(e);
        return CQK_CUDA_ERROR;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    void* ctx = current_context();
    if (ctx)
        for (int i = 0; i < g_count; i++)
            if (g_tab[i].ctx == ctx && g_tab[i].dev == dev) {
                *out = g_tab[i].addr;
                return CQK_OK;
            }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
        cqk::set_last_cuda_error(e);
        return CQK_CUDA_ERROR;
    }
    if (!ctx) ctx = current_context();  // the lookup made the device's primary context current
    if (ctx) {  // without a context handle the address is looked up on every call
        Entry& slot = g_count < kMaxEntries ? g_tab[g_count++] : g_tab[g_next++ % kMaxEntries];
        slot = Entry{ctx, dev, p};
    }
    *out = p;
    return CQK_OK;
}

}  // namespace

extern "C" int cqk_project_simplex_noalloc(int64_t n, int32_t dtype, const void* y, double r, void* x,
                                           uint32_t* free_mask, cqk_info* info_dev, const cqk_options* opt,
                                           void* stream) {
    if (n <= 0 || (dtype != CQK_F64 && dtype != CQK_F32) || !y || !x || !info_dev) return CQK_BAD_ARG;
    if (!(r > 0.0) || !(r < INFINITY) || x == y) return CQK_BAD_ARG;
    cqk::Opts o = cqk::resolve_options(opt, dtype, CQK_INIT_CONDAT);
    if (o.init != CQK_INIT_FORMULA && o.init != CQK_INIT_CONDAT && o.init != CQK_INIT_GIVEN) return CQK_BAD_ARG;
    if (o.block_threads != 256 || o.unroll_half != 0) return CQK_BAD_ARG;  // one build of the kernel
    // the static scratch holds partial sums for at most kNoAllocMaxBlocks blocks
    if (o.max_blocks > kNoAllocMaxBlocks) return CQK_BAD_ARG;
    if (o.max_blocks == 0) o.max_blocks = kNoAllocMaxBlocks;
    void* ws = nullptr;
    const int rc = scratch_address(&ws);
    if (rc != CQK_OK) return rc;
    // launch_simplex clears the scratch header (barrier counter, ticket, flags) on `stream`
    // before the kernel; the partial sums are written before they are read.
    return cqk::launch_simplex(n, dtype, y, r, 0, x, free_mask, info_dev, o, ws, (cudaStream_t)stream);
}
