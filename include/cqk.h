/*
 * cqk.h -- C ABI of libcqk, a B300 (sm_103a) solver for the continuous quadratic
 * knapsack problem (CQK) by the semismooth Newton method of Secchin & Silva,
 * "Parallel Newton methods for the continuous quadratic knapsack problem: A
 * Jacobi and Gauss-Seidel tale" (arXiv 2603.15910).
 *
 *   (CQK)   min  1/2 x'Dx - a'x   s.t.  b'x = r,  l <= x <= u,
 *           D = diag(d), d > 0, b > 0 (Sec. 1, eq. (CQK)); l_i may be -inf and
 *           u_i may be +inf.
 *
 * The dual multiplier lambda parametrises x_i(lambda) = clip((a_i + lambda b_i)/d_i,
 * l_i, u_i) (Sec. 2.1, eq. (xopt)); x(lambda*) is optimal iff
 * phi(lambda*) = b'x(lambda*) = r (eq. (opt)).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every array argument (a, b, d, l, u, y, x, g, gradients, masks, offsets, info,
 *    workspace) is a DEVICE pointer of the current CUDA device, owned by the
 *    caller.  The library allocates no memory and keeps no pointer after the call
 *    returns.  16-byte alignment of the arrays enables 128-bit loads; unaligned
 *    arrays are accepted and read with scalar loads.
 *  - dtype selects the storage of every floating-point array of the call:
 *    CQK_F64 (double) or CQK_F32 (float).  Scalars (r, lambda, sums) are always
 *    double; with CQK_F32 the multiplier is still kept and updated in double.
 *  - stream is a cudaStream_t passed as void*; NULL means the legacy default
 *    stream.  Every call is asynchronous on that stream and does not synchronise
 *    the host (except cqk_solve with n = 0, which writes info synchronously).
 *  - workspace/ws_bytes: caller-provided device scratch of at least
 *    cqk_workspace_bytes(...) bytes, 256-byte aligned.  It is overwritten; calls
 *    that may run concurrently need distinct workspaces.
 *  - Two levels of error reporting:
 *      return value   host-detectable problems: CQK_BAD_ARG (n < 0, NULL where
 *                     an array is required, bad dtype, workspace too small or
 *                     misaligned, r not usable) or CQK_CUDA_ERROR (a launch
 *                     failed; cqk_last_cuda_error() gives the cudaError_t).
 *                     Nothing is launched when the return value is not CQK_OK.
 *      info_dev       the outcome of the solve, written on the device at the
 *                     end of the call (status CQK_OK, CQK_INFEASIBLE,
 *                     CQK_MAXITER, CQK_BAD_INPUT, CQK_TIMEOUT).  Read it after
 *                     synchronising the stream.
 */
#ifndef CQK_H
#define CQK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { CQK_F64 = 0, CQK_F32 = 1 } cqk_dtype;

typedef enum {
    CQK_OK = 0,          /* solved                                                         */
    CQK_INFEASIBLE = 1,  /* r outside [b'l, b'u]: no breakpoint in the needed direction    */
                         /* (Alg. 1, the zero-derivative branches)                         */
    CQK_MAXITER = 2,     /* max_iter phi evaluations without meeting a stopping test       */
    CQK_BAD_INPUT = 3,   /* d <= 0, b <= 0, l > u, or a NaN in the data (sanity checks of  */
                         /* Sec. 5.1.1)                                                    */
    CQK_NONDIFF = 4,     /* backward: the free set is empty, lambda is not differentiable  */
    CQK_TIMEOUT = 5,     /* a device-wide wait exceeded spin_limit_us; results invalid     */
    CQK_CUDA_ERROR = 6,  /* a CUDA call failed (return value only)                         */
    CQK_BAD_ARG = 7      /* invalid host argument (return value only)                      */
} cqk_status;

typedef enum {
    CQK_INIT_FORMULA = 0, /* eq. (CQKlambda0) with J = all variables; for the simplex and    */
                          /* l1 ball also line 1 of Alg. 4 (lambda_0 >= min_i(-y_i))         */
    CQK_INIT_CONDAT = 1,  /* simplex / l1 only: Alg. 2 run independently on every chunk of a */
                          /* fixed partition, lambda_0 from eq. (lambdaJ) on the union of the */
                          /* J's (Sec. 4); the partition is reported in cqk_info             */
    CQK_INIT_WARM = 2,    /* from a primal estimate options.xbar (device array of the data's  */
                          /* dtype and length).  cqk_solve: eq. (CQKlambda0) over J = {l <    */
                          /* xbar < u}, all variables if J is empty (Sec. 2).  Projections:  */
                          /* Alg. 2 per chunk (as CQK_INIT_CONDAT) on the support of xbar    */
                          /* (xbar > 0; l1 ball: xbar != 0) (Sec. 3.3); lambda_0 =           */
                          /* max{r/n, -y_1} (l1 ball: -|y_1|) when no chunk keeps an element */
    CQK_INIT_GIVEN = 3    /* lambda_0 = options.lambda0                                      */
} cqk_init;

/* Which test ended the Newton loop (cqk_info.stop). */
typedef enum {
    CQK_STOP_NONE = 0,
    CQK_STOP_EXACT = 1,    /* phi(lambda_k) == r                                (Alg. 1, Alg. 4) */
    CQK_STOP_RESIDUAL = 2, /* |phi - r| < eps^{3/4}(sum|b_i x_i| + |r|)        (Sec. 4, crit. 1) */
    CQK_STOP_STEP = 3,     /* |(phi - r)/phi'| < eps^{3/4}                      (Sec. 4, crit. 2) */
    CQK_STOP_SAME = 4,     /* lambda_{k+1} == lambda_k                          (Sec. 4, crit. 2) */
    CQK_STOP_BRACKET = 5,  /* upper - lower < eps^{3/4} max(|upper|, |lower|)   (Sec. 4, crit. 3) */
    CQK_STOP_BELOW = 6,    /* phi(lambda_k) <= r, k >= 1                        (Alg. 4)          */
    CQK_STOP_INSIDE = 7    /* l1 ball: sum |y_i| <= r, x = y                    (Sec. 3.2)        */
} cqk_stop;

typedef struct cqk_options {
    int32_t max_iter;       /* cap on phi evaluations; default 100                              */
    int32_t init;           /* cqk_init; -1 (default): FORMULA for cqk_solve, CONDAT for the    */
                            /* projections                                                      */
    double lambda0;         /* start for CQK_INIT_GIVEN                                         */
    int32_t validate;       /* 1 (default): flag d <= 0, b <= 0, l > u, NaN as CQK_BAD_INPUT    */
    int32_t final_step;     /* 1 (default): after a stop by stopping criterion 1 or 2, form x   */
                            /* at lambda_k plus the Newton step already computed from lambda_k  */
                            /* (when it stays inside the bracket); 0: x = x(lambda_k)           */
    int64_t spin_limit_us;  /* bound on every device-wide wait, microseconds; default 2000000    */
    int32_t max_blocks;     /* 0 = automatic grid size; otherwise an upper bound                */
    int32_t fault_inject;   /* testing only: 1 = make every device-wide wait unsatisfiable so   */
                            /* that the call ends with CQK_TIMEOUT after spin_limit_us; 2 =     */
                            /* (simplex / l1, CQK_INIT_CONDAT, block chunks of 64 tiles or      */
                            /* more) the split Alg. 2 scan's queue is never published, so the   */
                            /* scanning warp's wait ends with CQK_TIMEOUT after spin_limit_us   */
    int32_t group_elems;    /* batched calls: an instance of length m is solved by a group of    */
                            /* min(32, ceil(m / group_elems)) blocks; 0 (default): 1048576 for  */
                            /* simplex / l1 batches, 65536 for general ones                     */
    int32_t condat_chunk;   /* CQK_INIT_CONDAT: the partition has min(warps, ceil(n /            */
                            /* condat_chunk)) chunks; 0 (default): 512                          */
    const void* xbar;       /* CQK_INIT_WARM: the primal estimate (device; NULL otherwise)       */
    int32_t warp_elems;     /* batched projections: instances shorter than warp_elems (rounded  */
                            /* down to a power of two) are solved by one warp each; 0 (default): */
                            /* 16384; negative: never                                           */
    int32_t scan_warps;     /* CQK_INIT_CONDAT projections on 16-byte aligned data: each block   */
                            /* deals its tiles to scan_warps chunks (1, 2 or 4; other positive   */
                            /* values round down to one of these), scanned by as                */
                            /* many warps side by side (the partition then has nchunks =         */
                            /* blocks * scan_warps, a looser union start); 0 (default): 1        */
    int32_t block_threads;  /* batched calls: threads per block of the persistent kernel.  0       */
                            /* (default) = 256; 128 or 512 for cqk_solve_batched (general) and   */
                            /* the batched adjoints; the batched projections and every single-   */
                            /* instance call run 256 (other values: CQK_BAD_ARG)                 */
    int32_t unroll;         /* batched calls: 16-byte vectors in flight per lane of the streaming */
                            /* loops.  0 (default): the full setting (projections 8, adjoints    */
                            /* 4-6, general 2 and two vectors per thread of a bulk-copy stage);  */
                            /* 1: half of that, with 256 threads per block.  Single-instance     */
                            /* calls: 0 only (other values: CQK_BAD_ARG)                         */
} cqk_options;

/* Written on the device by every solve. */
typedef struct cqk_info {
    double lambda;    /* final multiplier; x = x(lambda)                                       */
    double residual;  /* sum b_i x_i - r of the stored x (l1 ball: sum |x_i| - r)               */
    double abs_bx;    /* sum |b_i x_i| of the stored x (the scale of stopping criterion 1)       */
    double slope;     /* lateral derivative used in the last Newton step                        */
    double lambda0;   /* initial multiplier actually used                                       */
    int64_t nfree;    /* |{i : l_i < x_i < u_i}| (simplex / l1: number of nonzero x_i)           */
    int32_t iters;    /* phi evaluations (Newton iterations)                                    */
    int32_t status;   /* cqk_status                                                             */
    int32_t passes;   /* passes over the data, all phases                                       */
    int32_t stop;     /* cqk_stop                                                               */
    int32_t nchunks;  /* CQK_INIT_CONDAT: number of chunks of the partition (0 otherwise)        */
    int32_t tile;     /* CQK_INIT_CONDAT: elements per tile of the chunk partition.  A single   */
                      /* call: variable i is in chunk (i / tile) % nchunks.  With scan_warps =  */
                      /* s > 1, nchunks = blocks * s and block m deals its tiles m, m + blocks, */
                      /* m + 2 blocks, ... in turn to its s chunks, which is the same rule.     */
                      /* Batched calls shift the tiles by the instance's start: element         */
                      /* offsets[k] + i of instance k is in chunk                               */
                      /* ((i + offsets[k] % tile) / tile) % nchunks                             */
} cqk_info;

/* Fills *opt with the defaults listed above. */
void cqk_default_options(cqk_options* opt);

/* Workspace size, in bytes, for one call on n_total variables split into `batch` instances
 * (batch = 1 for cqk_solve / cqk_phi / cqk_project_*).  Returns 0 for invalid arguments. */
size_t cqk_workspace_bytes(int64_t n_total, int32_t batch, int32_t dtype);

/*
 * Solve one general CQK instance (Alg. 1 with the stopping tests of Sec. 4).
 *   n              number of variables, n >= 0 (n = 0: nothing is launched; info_dev
 *                  receives status CQK_OK if r == 0, else CQK_INFEASIBLE)
 *   a, b, d, l, u  device arrays of n elements of `dtype`; l may hold -inf, u +inf
 *   r              right-hand side of b'x = r
 *   x              device output, n elements of `dtype`: x(lambda*) (eq. (xopt))
 *   free_mask      nullable device output of ceil(n/32) uint32 words: bit i%32 of word
 *                  i/32 is set iff l_i < x_i < u_i
 *   info_dev       device pointer to one cqk_info
 *   opt            nullable; NULL means cqk_default_options()
 * Every Newton iteration is one Jacobi map-reduce pass over a, b, d, l, u (Sec. 4)
 * producing phi, phi'_+, phi'_- and sum|b_i x_i| (eq. (opt), eq. (phideriv)); the
 * multiplier update (Newton step, secant step, closest breakpoint) runs on the device with
 * no host synchronisation.
 */
int cqk_solve(int64_t n, int32_t dtype, const void* a, const void* b, const void* d,
              const void* l, const void* u, double r, void* x, uint32_t* free_mask,
              cqk_info* info_dev, const cqk_options* opt, void* workspace, size_t ws_bytes,
              void* stream);

/*
 * One map-reduce pass at a given lambda (eq. (opt) and eq. (phideriv)); writes 4 doubles
 * to out_dev (device): phi(lambda), phi'_+(lambda), phi'_-(lambda), sum |b_i x_i(lambda)|.
 * x (nullable) receives x(lambda).  Same array conventions as cqk_solve; n >= 1.
 */
int cqk_phi(int64_t n, int32_t dtype, const void* a, const void* b, const void* d,
            const void* l, const void* u, double lambda, void* x, double* out_dev,
            void* workspace, size_t ws_bytes, void* stream);

/*
 * Project y onto the r-simplex {x >= 0, sum x = r} (eq. (proj_Delta); r > 0, n >= 1) by
 * Alg. 4 from the start selected in opt->init (default CQK_INIT_CONDAT).
 *   y, x       device arrays of n elements of `dtype` (x may not alias y)
 *   free_mask  nullable, ceil(n/32) words, bit set iff x_i > 0
 */
int cqk_project_simplex(int64_t n, int32_t dtype, const void* y, double r, void* x,
                        uint32_t* free_mask, cqk_info* info_dev, const cqk_options* opt,
                        void* workspace, size_t ws_bytes, void* stream);

/*
 * Project y onto the l1 ball {sum |x_i| <= r} (Sec. 3.2; r > 0, n >= 1): x = y when
 * sum |y_i| <= r; otherwise x_i = sgn(y_i) max{0, |y_i| + lambda*} with lambda* <= 0
 * solving the simplex dual for |y| (Lemma 3.2), found by Alg. 4; with CQK_INIT_CONDAT the
 * Alg. 2 test is the strengthened min{|y|, |y| + lambda} > 0.  Arguments as
 * cqk_project_simplex; free_mask bit set iff x_i != 0.
 */
int cqk_project_l1(int64_t n, int32_t dtype, const void* y, double r, void* x,
                   uint32_t* free_mask, cqk_info* info_dev, const cqk_options* opt,
                   void* workspace, size_t ws_bytes, void* stream);

/*
 * A batch of B independent instances in one persistent launch (the paper solves one
 * instance at a time; the batch is a throughput convenience of this library: every
 * instance is solved exactly as the single call would, by Alg. 1 or Alg. 4).
 *   B              number of instances (B = 0: nothing is launched)
 *   offsets_dev    device array of B + 1 int64: instance k is the element range
 *                  [offsets_dev[k], offsets_dev[k+1]) of every array (non-decreasing;
 *                  empty instances allowed; read on the device only, so a decreasing pair
 *                  is reported as status CQK_BAD_ARG in that instance's info)
 *   a, b, d, l, u  device arrays of offsets_dev[B] elements; b, d, l, u all NULL selects
 *                  the simplex batch on y = a (b = d = 1, l = 0, u = +inf), the same as
 *                  cqk_project_simplex_batched
 *   r_dev          device array of B doubles: the right-hand side of each instance
 *   x, free_mask   as for the single calls, over the concatenated elements (mask bit i%32
 *                  of word i/32 for global element index i)
 *   info_dev       device array of B cqk_info; instance k's outcome in info_dev[k].
 *                  An empty instance gets CQK_OK if r == 0, else CQK_INFEASIBLE (general);
 *                  CQK_INFEASIBLE (simplex); CQK_OK with stop CQK_STOP_INSIDE (l1 ball).
 *                  An instance whose r is NaN (projections: not in (0, inf)) gets
 *                  CQK_BAD_ARG and its x is not written.
 *   workspace      at least cqk_workspace_bytes(n_total, B, dtype) bytes, 256-byte aligned
 * Instances are handed, longest first, to groups of co-resident blocks (a group of
 * min(32, ceil(m / group_elems)) blocks for an instance of m elements).  With
 * CQK_INIT_CONDAT, element offsets_dev[k] + i of instance k lies in chunk
 * ((i + offsets_dev[k] % tile) / tile) % nchunks, tile and nchunks as in info_dev[k].
 */
int cqk_solve_batched(int32_t B, const int64_t* offsets_dev, int32_t dtype, const void* a,
                      const void* b, const void* d, const void* l, const void* u,
                      const double* r_dev, void* x, uint32_t* free_mask, cqk_info* info_dev,
                      const cqk_options* opt, void* workspace, size_t ws_bytes, void* stream);

/* B simplex projections (cqk_project_simplex per instance); arguments as cqk_solve_batched. */
int cqk_project_simplex_batched(int32_t B, const int64_t* offsets_dev, int32_t dtype,
                                const void* y, const double* r_dev, void* x,
                                uint32_t* free_mask, cqk_info* info_dev,
                                const cqk_options* opt, void* workspace, size_t ws_bytes,
                                void* stream);

/* B l1-ball projections (cqk_project_l1 per instance); arguments as cqk_solve_batched. */
int cqk_project_l1_batched(int32_t B, const int64_t* offsets_dev, int32_t dtype, const void* y,
                           const double* r_dev, void* x, uint32_t* free_mask,
                           cqk_info* info_dev, const cqk_options* opt, void* workspace,
                           size_t ws_bytes, void* stream);

/*
 * Adjoint of the solution map (the paper has no backward pass: the formulas below follow
 * from differentiating its optimality conditions, eq. (xopt) on the free set and
 * b'x = r).  Given the forward's x, free mask and lambda (info_dev) and an upstream
 * gradient g, with F the free set, Q = sum_F b_i^2/d_i and mu = sum_F b_i g_i/d_i / Q:
 *   ga_i = (g_i - mu b_i)/d_i on F, else 0      gd_i = -x_i ga_i
 *   gb_i = lambda ga_i - mu x_i                 gr   = mu
 *   gl_i = g_i - mu b_i where x_i sits at l_i, gu_i likewise at u_i, else 0
 * A variable with l_i = u_i counts as at its lower bound when (a_i + lambda b_i)/d_i <= l_i
 * (needs a; with a NULL it counts as at the lower bound).
 *   B, offsets_dev   offsets_dev NULL: one instance of n elements (B must be 1); otherwise
 *                    B instances as in cqk_solve_batched (n is ignored)
 *   g, x, b, d       device arrays (required); a nullable; l, u required when free_mask is
 *                    NULL (F = {l < x < u}) or when gl / gu is requested
 *   free_mask        nullable: the forward's mask
 *   info_dev         the forward's info (one per instance): lambda, and for the l1 ball stop
 *   ga, gb, gd, gl, gu  nullable device outputs (same dtype and length as x)
 *   gr_dev           nullable device output, one double per instance
 *   status_dev       nullable device output, one int32 per instance: CQK_OK, CQK_NONDIFF
 *                    (F empty: mu = 0), CQK_TIMEOUT, or CQK_BAD_ARG (decreasing offsets)
 *   workspace        cqk_workspace_bytes(n_total, B, dtype) bytes, 256-byte aligned
 * Two passes over the data: a reduction for (sum_F b g/d, Q) and the map.  Arithmetic: the
 * sums and mu in FP64; per element double-float (a pair of floats, about 2^-44 relative) for
 * values in [2^-60, 2^60] and exact FP64 outside that range; FP64 results rounded once.
 */
int cqk_backward(int32_t B, const int64_t* offsets_dev, int64_t n, int32_t dtype, const void* g,
                 const void* x, const void* a, const void* b, const void* d, const void* l,
                 const void* u, const uint32_t* free_mask, const cqk_info* info_dev, void* ga,
                 void* gb, void* gd, void* gl, void* gu, double* gr_dev, int32_t* status_dev,
                 const cqk_options* opt, void* workspace, size_t ws_bytes, void* stream);

/* Simplex projection adjoint: with F = {x > 0} (or the mask), gy_i = g_i - mean_F(g) on F,
 * else 0; gr = mean_F(g).  Arguments as cqk_backward. */
int cqk_backward_simplex(int32_t B, const int64_t* offsets_dev, int64_t n, int32_t dtype,
                         const void* g, const void* x, const uint32_t* free_mask,
                         const cqk_info* info_dev, void* gy, double* gr_dev, int32_t* status_dev,
                         const cqk_options* opt, void* workspace, size_t ws_bytes, void* stream);

/* l1-ball projection adjoint (Lemma 3.2): y inside the ball (info stop CQK_STOP_INSIDE):
 * gy = g, gr = 0; otherwise, with s = sgn(x) and F = {x != 0} (or the mask),
 * gy_i = g_i - s_i mean_F(s g) on F, else 0; gr = mean_F(s g). */
int cqk_backward_l1(int32_t B, const int64_t* offsets_dev, int64_t n, int32_t dtype, const void* g,
                    const void* x, const uint32_t* free_mask, const cqk_info* info_dev, void* gy,
                    double* gr_dev, int32_t* status_dev, const cqk_options* opt, void* workspace,
                    size_t ws_bytes, void* stream);

/*
 * Allocation-free variant of cqk_project_simplex (the paper has no counterpart: this is a
 * calling convenience of this library).
 *
 * Some callers cannot allocate device memory when they need a projection -- for instance a
 * plugin whose host application owns the device allocator, or a real-time loop whose device
 * memory is fixed at start-up -- and so cannot pass the workspace that cqk_project_simplex
 * takes.  This entry point takes the same arguments without the workspace and runs the same
 * kernel with its scratch in a static device array of CQK_NOALLOC_SCRATCH_BYTES bytes that
 * every GPU loading the library holds until the process exits.  It calls no allocator.
 *   - The array holds partial sums for at most CQK_NOALLOC_MAX_BLOCKS blocks, so the grid is
 *     capped there; options->max_blocks above that limit is rejected with CQK_BAD_ARG.
 *   - The first call in a CUDA context (normally: the first call on a device, in its primary
 *     context) looks up the array's device address (cudaGetSymbolAddress) with that device
 *     current and remembers it for that context; make that first call before any stream
 *     capture.
 *   - Every call on a device shares the one array, and each call clears the part that must
 *     start at zero.  Calls whose executions overlap on the GPU (different streams, or
 *     several host threads) race on it: issue them in order on one stream.
 */
#define CQK_NOALLOC_MAX_BLOCKS 592
#define CQK_NOALLOC_SCRATCH_BYTES 76032
int cqk_project_simplex_noalloc(int64_t n, int32_t dtype, const void* y, double r, void* x,
                                uint32_t* free_mask, cqk_info* info_dev, const cqk_options* opt,
                                void* stream);

/* Name of a cqk_status value (static string). */
const char* cqk_status_string(int status);

/* The cudaError_t of the last failed CUDA call made by this library in this thread. */
int cqk_last_cuda_error(void);

/* ABI version: 10000 * major + 100 * minor + patch. */
int cqk_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CQK_H */
