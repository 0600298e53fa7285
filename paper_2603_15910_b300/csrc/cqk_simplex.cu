// cqk_simplex.cu -- projection onto the r-simplex and onto the l1 ball (Sec. 3).
//
// One cooperative launch per projection.  Every block streams its share of y with
// coalesced 128-bit loads; after each pass the per-block partial sums go to the workspace,
// a bounded grid barrier follows, and EVERY block reduces the partials in the same fixed
// order and runs the same scalar update (Alg. 4), so all blocks hold bit-identical
// multipliers without a second synchronisation.
//
//   pass 0   start:  CQK_INIT_FORMULA  sum y and max y (l1: |y|) -> lambda_0 of
//                                      eq. (CQKlambda0), clamped by line 1 of Alg. 4
//                    CQK_INIT_CONDAT   Alg. 2 on every warp's chunk (exact, see
//                                      condat_chunk); lambda_0 from eq. (lambdaJ) on the
//                                      union of the J's (Sec. 4)
//   pass k   phi(lambda_k) = sum_{y_i > -lambda_k} (y_i + lambda_k),
//            phi'_- = #{y_i > -lambda_k}, phi'_+ = #{y_i >= -lambda_k}
//            (eq. (opt), eq. (phideriv) specialised as in the proof of Theorem 3.1)
//   final    x_i = max{0, y_i + lambda*} (l1: sgn(y_i) max{0, |y_i| + lambda*}), free mask,
//            sum x - r of the stored x (Sec. 4: the primal recovery is a map)
//
// The tests y_i > -lambda are exact (bit patterns for FP64 data, a directed rounding of
// the threshold for FP32 data); the selected terms y_i + lambda are formed exactly rounded
// in FP64 (FP64 data, few elements once lambda is near lambda*) or in double-float (FP32
// data).
#include "cqk_block.cuh"

namespace cqk {
namespace {

constexpr int kCondatVecsPerLane = 4;  // vectors per lane in one Alg. 2 tile

struct SimplexArgs {
    int64_t n;
    const void* y;
    void* x;
    uint32_t* mask;
    cqk_info* info;
    double r;
    int init;
    double lambda0;
    int max_iter;
    double eps34;
    int validate;
    int final_step;
    int aligned;
    unsigned long long limit_ns;
    int fault_inject;
    WsHeader* hdr;
    double* part;  // [2][kPartialQ][gridDim.x]
};

// ---- Alg. 2 on one warp's chunk -----------------------------------------------------------
// The chunk of warp w (of W) is the set of tiles t = w, w + W, w + 2W, ...; tile t holds
// elements [t*TILE, (t+1)*TILE), TILE = 32 * K * V, scanned in increasing index order.
// Lane L holds vectors t*32*K + k*32 + L (k < K), so the index order in a tile is (k, L, j).
//
// Exactness: both branches of the first loop of Alg. 2 lower lambda (adding j with
// y_j + lambda > 0 gives lambda - (y_j + lambda)/(|J|+1); a restart gives r - y_j, below the
// rejected lambda_{J u {j}}), so once J is started an element that fails the test fails it
// for the rest of the scan.  The warp therefore tests a whole slab at once, processes the
// first passing element in index order with the scalar update (the same FP64 operations as
// a sequential scan), and re-tests only the later elements of the slab.  The final loop of
// Alg. 2 over J~ visits, in order, the elements of J~ that pass the test with the current
// lambda; every element before the last restart that is not in J~ failed the test with a
// larger lambda and fails it again, so that loop is a re-scan of the chunk prefix before
// the last restart with the same test.
template <typename T, bool L1>
__device__ __forceinline__ bool condat_test(T v, const GtThreshold& g, float rd) {
    if constexpr (sizeof(T) == 8) {
        unsigned long long b = bits_of((double)v);
        if (L1) b &= 0x7FFFFFFFFFFFFFFFull;
        return gt_bits(b, g);
    } else {
        float f = L1 ? fabsf((float)v) : (float)v;
        return f > rd;
    }
}

// threshold c of the test "y + lambda > 0" (l1: "min{|y|, |y| + lambda} > 0", i.e. |y| > c)
template <bool L1>
__device__ __forceinline__ double condat_c(double lam) { return L1 ? fmax(0.0, -lam) : -lam; }

template <typename T, bool L1>
__device__ __forceinline__ void condat_slab(const T (&vals)[VecOf<T>::V], const bool (&okv)[VecOf<T>::V],
                                            int64_t eidx0, int64_t before, bool first_loop, double r,
                                            double& lam, double& S, long long& nJ, int64_t& rs) {
    constexpr int V = VecOf<T>::V;
    const int lane = threadIdx.x & 31;
    bool pass[V];
    if (first_loop && nJ == 0) {
        // the first element of the chunk starts J unconditionally (first line of Alg. 2)
        unsigned any_ok = __ballot_sync(0xffffffffu, okv[0]);
        if (!any_ok) return;
        const int L0 = __ffs(any_ok) - 1;
        double y0 = (double)__shfl_sync(0xffffffffu, vals[0], L0);
        if (L1) y0 = fabs(y0);
        S = y0;
        nJ = 1;
        lam = r - y0;
        rs = __shfl_sync(0xffffffffu, eidx0, L0);
        const double c = condat_c<L1>(lam);
        const GtThreshold g = make_gt(c);
        const float rd = f32_rd(c);
#pragma unroll
        for (int j = 0; j < V; j++) {
            const bool after = (lane > L0) || (lane == L0 && j > 0);
            pass[j] = okv[j] && after && condat_test<T, L1>(vals[j], g, rd);
        }
    } else {
        const double c = condat_c<L1>(lam);
        const GtThreshold g = make_gt(c);
        const float rd = f32_rd(c);
#pragma unroll
        for (int j = 0; j < V; j++) pass[j] = okv[j] && (eidx0 + j < before) && condat_test<T, L1>(vals[j], g, rd);
    }
    while (true) {
        unsigned m[V];
        unsigned any = 0;
#pragma unroll
        for (int j = 0; j < V; j++) {
            m[j] = __ballot_sync(0xffffffffu, pass[j]);
            any |= m[j];
        }
        if (!any) break;
        const int Lf = __ffs(any) - 1;
        int jf = 0;
#pragma unroll
        for (int j = V - 1; j >= 0; j--)
            if ((m[j] >> Lf) & 1u) jf = j;
        T mine = vals[0];
#pragma unroll
        for (int j = 1; j < V; j++)
            if (j == jf) mine = vals[j];
        double yv = (double)__shfl_sync(0xffffffffu, mine, Lf);
        if (L1) yv = fabs(yv);
        const int64_t e = __shfl_sync(0xffffffffu, eidx0, Lf) + jf;
        if (first_loop) {
            const double lamn = (r - S - yv) / (double)(nJ + 1);
            if (lamn < r - yv) {
                S += yv;
                nJ += 1;
                lam = lamn;
            } else {  // restart: J~ <- J~ u J, J <- {j}
                rs = e;
                S = yv;
                nJ = 1;
                lam = r - yv;
            }
        } else {
            lam = (r - S - yv) / (double)(nJ + 1);
            S += yv;
            nJ += 1;
        }
        const double c = condat_c<L1>(lam);
        const GtThreshold g = make_gt(c);
        const float rd = f32_rd(c);
#pragma unroll
        for (int j = 0; j < V; j++) {
            const bool after = (lane > Lf) || (lane == Lf && j > jf);
            pass[j] = pass[j] && after && condat_test<T, L1>(vals[j], g, rd);
        }
    }
}

template <typename T, bool L1>
__device__ void condat_chunk(const T* __restrict__ y, int64_t n, bool aligned, double r, int64_t w, int64_t W,
                             double& S_out, long long& nJ_out) {
    constexpr int V = VecOf<T>::V;
    constexpr int K = kCondatVecsPerLane;
    constexpr int TILE = 32 * K * V;
    const int lane = threadIdx.x & 31;
    const int64_t ntiles = (n + TILE - 1) / TILE;
    double lam = 0.0, S = 0.0;
    long long nJ = 0;
    int64_t rs = -1;
    for (int64_t t = w; t < ntiles; t += W) {
        T vals[K][V];
        bool okv[K][V];
#pragma unroll
        for (int k = 0; k < K; k++) load_vec<T>(y, n, t * 32 * K + k * 32 + lane, aligned, vals[k], okv[k]);
#pragma unroll
        for (int k = 0; k < K; k++)
            condat_slab<T, L1>(vals[k], okv[k], (t * 32 * K + k * 32 + lane) * V, INT64_MAX, true, r, lam, S, nJ, rs);
    }
    // final loop of Alg. 2: re-scan the chunk prefix before the last restart
    if (nJ > 0 && rs >= 0) {
        const int64_t tlast = rs / TILE;
        for (int64_t t = w; t <= tlast; t += W) {
            T vals[K][V];
            bool okv[K][V];
#pragma unroll
            for (int k = 0; k < K; k++) load_vec<T>(y, n, t * 32 * K + k * 32 + lane, aligned, vals[k], okv[k]);
#pragma unroll
            for (int k = 0; k < K; k++)
                condat_slab<T, L1>(vals[k], okv[k], (t * 32 * K + k * 32 + lane) * V, rs, false, r, lam, S, nJ, rs);
        }
    }
    S_out = S;
    nJ_out = nJ;
}

// ---- the persistent kernel ----------------------------------------------------------------
template <typename T, bool L1>
__global__ void __launch_bounds__(NT) simplex_kernel(SimplexArgs A) {
    constexpr int V = VecOf<T>::V;
    __shared__ double sh[kPartialQ][NWARP];
    __shared__ double bc[kPartialQ];
    const T* __restrict__ y = static_cast<const T*>(A.y);
    const int64_t n = A.n;
    const int64_t nv = (n + V - 1) / V;
    const int lane = threadIdx.x & 31;
    const int G = gridDim.x;
    const int64_t gwarp = (int64_t)blockIdx.x * NWARP + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)G * NWARP;
    const bool aligned = A.aligned != 0;
    unsigned bar_target = (unsigned)G + (A.fault_inject ? 1u : 0u);
    unsigned* bar = &A.hdr->bar_count;
    int* err = &A.hdr->error;
    const double r = A.r;

    // ------------------------------------------------------------------ pass 0: start
    double lam0 = 0.0, abs_sum = 0.0;
    int passes = 0, nchunks = 0, tile = 0;
    {
        double q[4] = {0.0, 0.0, 0.0, -INFINITY};  // sum y (l1: |y|), union sum, union size, max y (l1: |y|)
        const bool condat = A.init == CQK_INIT_CONDAT;
        const bool sum_pass = L1 || !condat;
        bool bad = false;
        if (sum_pass) {
            df acc = df_make(0.0f);
            double acc_wide = 0.0;  // FP64 values outside the df operating range
            double mx = -INFINITY;
            for (int64_t qw = gwarp * 32; qw < nv; qw += nwarps * 32) {
                T v[V];
                bool ok[V];
                load_vec<T>(y, n, qw + lane, aligned, v, ok);
#pragma unroll
                for (int j = 0; j < V; j++) {
                    if (!ok[j]) continue;
                    const T t = L1 ? (T)fabs((double)v[j]) : v[j];
                    if constexpr (sizeof(T) == 8) {
                        if (df_in_range((double)t, false)) acc = df_add(acc, split_f64((double)t));
                        else acc_wide += (double)t;
                    } else {
                        acc = df_add_f(acc, (float)t);
                    }
                    mx = fmax(mx, (double)t);
                    bad |= (v[j] != v[j]);
                }
            }
            q[0] = df_to_f64(acc) + acc_wide;
            q[3] = mx;
            passes++;
        }
        if (condat) {
            double Sw = 0.0;
            long long nJw = 0;
            condat_chunk<T, L1>(y, n, aligned, r, gwarp, nwarps, Sw, nJw);
            q[1] = lane == 0 ? Sw : 0.0;
            q[2] = lane == 0 ? (double)nJw : 0.0;
            passes++;
        }
        const int wid = threadIdx.x >> 5;
        const double s0 = warp_sum(q[0]), s1 = warp_sum(q[1]), s2 = warp_sum(q[2]), m = warp_max(q[3]);
        const unsigned badw = __ballot_sync(0xffffffffu, bad);
        if (lane == 0) {
            sh[0][wid] = s0;
            sh[1][wid] = s1;
            sh[2][wid] = s2;
            sh[3][wid] = m;
            if (badw && A.validate) atomicOr(&A.hdr->flags, kFlagBadInput);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double t0 = 0, t1 = 0, t2 = 0, t3 = -INFINITY;
            for (int w = 0; w < NWARP; w++) {
                t0 += sh[0][w];
                t1 += sh[1][w];
                t2 += sh[2][w];
                t3 = fmax(t3, sh[3][w]);
            }
            const double pv[4] = {t0, t1, t2, t3};
            write_partials<4>(A.part, 0, pv);
        }
        __syncthreads();
        if (!grid_barrier(bar, bar_target, err, A.limit_ns, CQK_TIMEOUT)) {
            if (threadIdx.x == 0) A.info->status = CQK_TIMEOUT;
            return;
        }
        bar_target += (unsigned)G;
        double red[4];
        grid_reduce<4>(A.part, 0, 3, red, sh, bc);
        abs_sum = red[0];
        if (condat) {
            lam0 = (r - red[1]) / red[2];  // eq. (lambdaJ) on the union of the chunks' J
            nchunks = (int)nwarps;
            tile = 32 * kCondatVecsPerLane * V;
        } else if (A.init == CQK_INIT_GIVEN) {
            lam0 = fmax(A.lambda0, -red[3]);  // Alg. 4, line 1
        } else {
            lam0 = fmax((r - red[0]) / (double)n, -red[3]);  // eq. (CQKlambda0) with b = d = 1; Alg. 4 line 1
        }
    }
    bool bad_input = A.validate && (__ldcg(&A.hdr->flags) & kFlagBadInput);

    // ------------------------------------------------------------------ Newton loop (Alg. 4)
    double lam = lam0, lower = -INFINITY, upper = INFINITY, slope = 0.0, final_lam = lam0;
    int status = CQK_OK, stop = CQK_STOP_NONE, k = 0;
    bool copy = false;  // l1 ball, y inside
    if (bad_input) {
        status = CQK_BAD_INPUT;
    } else if (L1 && abs_sum <= r) {
        copy = true;
        stop = CQK_STOP_INSIDE;
        lam = final_lam = 0.0;
    } else {
        int par = 1;
        for (k = 0;; k++) {
            if (k >= A.max_iter) {
                status = CQK_MAXITER;
                break;
            }
            double acc64 = 0.0;
            df acc32 = df_make(0.0f);
            long long cm = 0, ct = 0;
            bool nan_seen = false;
            const double c = -lam;
            if constexpr (sizeof(T) == 8) {
                const GtThreshold g = make_gt(c);
                const unsigned long long cb = g.bits;
                for (int64_t qw = gwarp * 32; qw < nv; qw += nwarps * 32) {
                    T v[V];
                    bool ok[V];
                    load_vec<T>(y, n, qw + lane, aligned, v, ok);
#pragma unroll
                    for (int j = 0; j < V; j++) {
                        unsigned long long b = bits_of((double)v[j]);
                        if (L1) b &= 0x7FFFFFFFFFFFFFFFull;
                        const bool sel = ok[j] && gt_bits(b, g);
                        const bool tie = ok[j] && !sel && (b == cb || ((b | cb) << 1) == 0ull);
                        if (sel) {
                            acc64 += __longlong_as_double((long long)b) + lam;
                            cm++;
                        }
                        ct += tie;
                        nan_seen |= ok[j] && ((b & 0x7FFFFFFFFFFFFFFFull) > 0x7FF0000000000000ull);
                    }
                }
            } else {
                const float rd = f32_rd(c), ru = f32_ru(c);
                const df Lm = df_from_f64(lam);
                for (int64_t qw = gwarp * 32; qw < nv; qw += nwarps * 32) {
                    T v[V];
                    bool ok[V];
                    load_vec<T>(y, n, qw + lane, aligned, v, ok);
#pragma unroll
                    for (int j = 0; j < V; j++) {
                        const float f = L1 ? fabsf((float)v[j]) : (float)v[j];
                        const bool sel = ok[j] && f > rd;
                        const bool tie = ok[j] && !sel && f >= ru;
                        if (sel) {
                            acc32 = df_add(acc32, df_add_f(Lm, f));
                            cm++;
                        }
                        ct += tie;
                        nan_seen |= ok[j] && (f != f);
                    }
                }
                acc64 = df_to_f64(acc32);
            }
            passes++;
            if (A.validate && __any_sync(0xffffffffu, nan_seen) && lane == 0) atomicOr(&A.hdr->flags, kFlagBadInput);
            double pv[3] = {acc64, (double)cm, (double)(cm + ct)};
            block_sum<3>(pv, sh);
            write_partials<3>(A.part, par, pv);
            if (!grid_barrier(bar, bar_target, err, A.limit_ns, CQK_TIMEOUT)) {
                if (threadIdx.x == 0) A.info->status = CQK_TIMEOUT;
                return;
            }
            bar_target += (unsigned)G;
            double red[3];
            grid_reduce<3>(A.part, par, -1, red, sh, bc);
            par ^= 1;
            if (A.validate && (__ldcg(&A.hdr->flags) & kFlagBadInput)) {
                bad_input = true;
                status = CQK_BAD_INPUT;
                k++;
                break;
            }
            const double phi = red[0], dminus = red[1], dplus = red[2];
            const double gk = phi - r;
            double step = 0.0;
            bool done = false;
            final_lam = lam;
            if (k == 0) {
                if (gk == 0.0) {
                    stop = CQK_STOP_EXACT;
                    done = true;
                } else if (gk < 0.0) {
                    lower = lam;
                    slope = dplus;
                    step = -gk / dplus;
                } else {
                    upper = lam;
                    slope = dminus;
                    step = -gk / dminus;
                }
            } else if (gk <= 0.0) {
                stop = CQK_STOP_BELOW;
                done = true;
            } else {
                upper = lam;
                slope = dminus;
                step = -gk / dminus;
            }
            if (!done && upper - lower < A.eps34 * fmax(fabs(upper), fabs(lower))) {
                stop = CQK_STOP_BRACKET;
                done = true;
            }
            if (!done && fabs(step) < A.eps34) {
                stop = CQK_STOP_STEP;
                done = true;
                if (A.final_step) final_lam = lam + step;  // the Newton step already computed
            }
            if (!done) {
                const double next = lam + step;
                if (next == lam) {
                    stop = CQK_STOP_SAME;
                    done = true;
                } else {
                    lam = next;
                }
            }
            if (done) {
                k++;
                break;
            }
        }
    }

    // ------------------------------------------------------------------ final pass: x, mask
    double sx = 0.0;
    df sx32 = df_make(0.0f);
    long long nz = 0;
    T* __restrict__ x = static_cast<T*>(A.x);
    if (!bad_input) {
        const double lamf = final_lam;
        const GtThreshold g = make_gt(-lamf);
        const float rd = f32_rd(-lamf);
        const df Lm = df_from_f64(lamf);
        for (int64_t qw = gwarp * 32; qw < nv; qw += nwarps * 32) {
            const int64_t q = qw + lane;
            T v[V];
            bool ok[V];
            load_vec<T>(y, n, q, aligned, v, ok);
            T o[V];
            bool sel[V];
#pragma unroll
            for (int j = 0; j < V; j++) {
                if (copy) {
                    o[j] = v[j];
                    sel[j] = ok[j] && v[j] != T(0);
                } else if constexpr (sizeof(T) == 8) {
                    const unsigned long long b = bits_of((double)v[j]);
                    const unsigned long long ab = L1 ? (b & 0x7FFFFFFFFFFFFFFFull) : b;
                    sel[j] = ok[j] && gt_bits(ab, g);
                    double xv = sel[j] ? (__longlong_as_double((long long)ab) + lamf) : 0.0;
                    if (L1 && (b >> 63)) xv = -xv;
                    o[j] = (T)xv;
                } else {
                    const float f = (float)v[j];
                    const float af = L1 ? fabsf(f) : f;
                    sel[j] = ok[j] && af > rd;
                    float xv = 0.0f;
                    if (sel[j]) {
                        const df t = df_add_f(Lm, af);
                        xv = __fadd_rn(t.hi, t.lo);
                    }
                    if (L1 && f < 0.0f) xv = -xv;
                    o[j] = (T)xv;
                }
                if (sel[j]) {
                    nz++;
                    if constexpr (sizeof(T) == 8) sx += fabs((double)o[j]);
                    else sx32 = df_add_f(sx32, fabsf((float)o[j]));
                }
            }
            store_vec<T>(x, n, q, aligned, o);
            if (A.mask) store_mask<V>(A.mask, n, qw, sel);
        }
    }
    if constexpr (sizeof(T) == 4) sx = df_to_f64(sx32);
    double pv[2] = {sx, (double)nz}, tot[2];
    if (last_block_sums<2>(A.part, &A.hdr->ticket, pv, tot, sh) && threadIdx.x == 0) {
        cqk_info inf;
        inf.lambda = final_lam;
        inf.residual = tot[0] - r;
        inf.abs_bx = tot[0];
        inf.slope = slope;
        inf.lambda0 = lam0;
        inf.nfree = (int64_t)tot[1];
        inf.iters = k;
        const int e = *(volatile int*)&A.hdr->error;
        inf.status = e ? e : status;
        inf.passes = passes + (bad_input ? 0 : 1);
        inf.stop = stop;
        inf.nchunks = nchunks;
        inf.tile = tile;
        *A.info = inf;
    }
}

}  // namespace

int launch_simplex(int64_t n, int dtype, const void* y, double r, int l1, void* x, uint32_t* mask,
                   cqk_info* info, const Opts& o, void* ws, cudaStream_t s) {
    SimplexArgs A;
    A.n = n;
    A.y = y;
    A.x = x;
    A.mask = mask;
    A.info = info;
    A.r = r;
    A.init = o.init;
    A.lambda0 = o.lambda0;
    A.max_iter = o.max_iter;
    A.eps34 = kEps34F64;
    A.validate = o.validate;
    A.final_step = o.final_step;
    A.limit_ns = o.limit_ns;
    A.fault_inject = o.fault_inject;
    A.hdr = static_cast<WsHeader*>(ws);
    A.part = reinterpret_cast<double*>(static_cast<char*>(ws) + sizeof(WsHeader));
    A.aligned = ((((uintptr_t)y) | ((uintptr_t)x)) % 16 == 0) ? 1 : 0;
    const void* kern;
    if (dtype == CQK_F64)
        kern = l1 ? (const void*)simplex_kernel<double, true> : (const void*)simplex_kernel<double, false>;
    else
        kern = l1 ? (const void*)simplex_kernel<float, true> : (const void*)simplex_kernel<float, false>;
    const int64_t vec = dtype == CQK_F64 ? 2 : 4;
    const int grid = persistent_grid(kern, NT, 0, (n + vec - 1) / vec, o.max_blocks);
    if (grid <= 0) return CQK_CUDA_ERROR;
    cudaError_t e = cudaMemsetAsync(ws, 0, sizeof(WsHeader), s);
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return CQK_CUDA_ERROR;
    }
    void* args[] = {&A};
    e = cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(NT), args, 0, s);
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return CQK_CUDA_ERROR;
    }
    return CQK_OK;
}

}  // namespace cqk
