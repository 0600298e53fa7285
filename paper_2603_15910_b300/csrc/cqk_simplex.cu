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
#include <string.h>

#include "cqk_batch.cuh"

namespace cqk {
namespace {

constexpr int kStreamU = 8;  // 16-byte vectors in flight per lane in the streaming passes

// vectors per lane in one Alg. 2 tile: a tile is 512 elements for FP64 and FP32 data
template <typename T>
__host__ __device__ constexpr int condat_k() { return 512 / (32 * VecOf<T>::V); }

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
    int64_t condat_chunk;  // minimum elements per chunk of the parallel Alg. 2 start
    const void* xbar;      // CQK_INIT_WARM: primal estimate
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
    // exact test "y > c" (l1: "|y| > c") on the bit pattern / against the rounded-down threshold
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

// Warp-uniform state of one chunk's scan: lambda_J, sum_J y, |J|, the index of the last
// restart, and the test threshold derived from lambda (recomputed only when lambda changes,
// which keeps FP64 instructions off the per-slab path).
struct CondatState {
    double lam, S;
    long long nJ;
    int64_t rs;
    GtThreshold g;
    float rd;
};

template <bool L1>
__device__ __forceinline__ void condat_set_lam(CondatState& st, double lam) {
    st.lam = lam;
    const double c = condat_c<L1>(lam);
    st.g = make_gt(c);
    st.rd = f32_rd(c);
}

template <typename T, bool L1>
__device__ __forceinline__ void condat_slab(const T (&vals)[VecOf<T>::V], const bool (&okv)[VecOf<T>::V],
                                            int64_t eidx0, int64_t before, bool first_loop, double r,
                                            CondatState& st) {
    constexpr int V = VecOf<T>::V;
    const int lane = threadIdx.x & 31;
    bool pass[V];
    if (first_loop && st.nJ == 0) {
        // the first element of the chunk (in (lane, j) order; a span may start inside a
        // vector) starts J unconditionally (first line of Alg. 2)
        unsigned any_ok = 0, mo[V];
#pragma unroll
        for (int j = 0; j < V; j++) {
            mo[j] = __ballot_sync(0xffffffffu, okv[j]);
            any_ok |= mo[j];
        }
        if (!any_ok) return;
        const int L0 = __ffs(any_ok) - 1;
        int j0 = 0;
#pragma unroll
        for (int j = V - 1; j >= 0; j--)
            if ((mo[j] >> L0) & 1u) j0 = j;
        double y0 = (double)__shfl_sync(0xffffffffu, pick(vals, j0), L0);
        if (L1) y0 = fabs(y0);
        st.S = y0;
        st.nJ = 1;
        st.rs = __shfl_sync(0xffffffffu, eidx0, L0) + j0;
        condat_set_lam<L1>(st, r - y0);
#pragma unroll
        for (int j = 0; j < V; j++) {
            const bool after = (lane > L0) || (lane == L0 && j > j0);
            pass[j] = okv[j] && after && condat_test<T, L1>(vals[j], st.g, st.rd);
        }
    } else {
#pragma unroll
        for (int j = 0; j < V; j++)
            pass[j] = okv[j] && (eidx0 + j < before) && condat_test<T, L1>(vals[j], st.g, st.rd);
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
        double yv = (double)__shfl_sync(0xffffffffu, pick(vals, jf), Lf);
        if (L1) yv = fabs(yv);
        const int64_t e = __shfl_sync(0xffffffffu, eidx0, Lf) + jf;
        if (first_loop) {
            const double lamn = (r - st.S - yv) / (double)(st.nJ + 1);
            if (lamn < r - yv) {
                st.S += yv;
                st.nJ += 1;
                condat_set_lam<L1>(st, lamn);
            } else {  // restart: J~ <- J~ u J, J <- {j}
                st.rs = e;
                st.S = yv;
                st.nJ = 1;
                condat_set_lam<L1>(st, r - yv);
            }
        } else {
            const double lamn = (r - st.S - yv) / (double)(st.nJ + 1);
            st.S += yv;
            st.nJ += 1;
            condat_set_lam<L1>(st, lamn);
        }
#pragma unroll
        for (int j = 0; j < V; j++) {
            const bool after = (lane > Lf) || (lane == Lf && j > jf);
            pass[j] = pass[j] && after && condat_test<T, L1>(vals[j], st.g, st.rd);
        }
    }
}

// xb (nullable): a primal estimate; the chunk then keeps only the elements of its support
// (x_i > 0; l1 ball: x_i != 0), the warm start of Sec. 3.3.
template <typename T, bool L1>
__device__ __forceinline__ void support_mask(const T* __restrict__ xb, const Span& sp, int64_t q, bool aligned,
                                             bool (&okv)[VecOf<T>::V]) {
    if (!xb) return;
    constexpr int V = VecOf<T>::V;
    T xv[V];
    bool xok[V];
    load_vec<T>(xb, sp, q, aligned, xv, xok);
#pragma unroll
    for (int j = 0; j < V; j++) okv[j] = okv[j] && (L1 ? xv[j] != T(0) : xv[j] > T(0));
}

template <typename T, bool L1>
__device__ void condat_chunk(const T* __restrict__ y, const T* __restrict__ xb, const Span& sp, bool aligned,
                             double r, int64_t w, int64_t W, double& S_out, long long& nJ_out) {
    constexpr int V = VecOf<T>::V;
    constexpr int K = condat_k<T>();
    constexpr int TILE = 32 * K * V;
    const int lane = threadIdx.x & 31;
    const int64_t t0 = sp.lo / TILE, ntiles = (sp.hi + TILE - 1) / TILE;
    CondatState st;
    st.S = 0.0;
    st.nJ = 0;
    st.rs = -1;
    condat_set_lam<L1>(st, 0.0);
    for (int64_t t = t0 + w; t < ntiles; t += W) {
        T vals[K][V];
        bool okv[K][V];
#pragma unroll
        for (int k = 0; k < K; k++) load_vec<T>(y, sp, t * 32 * K + k * 32 + lane, aligned, vals[k], okv[k]);
#pragma unroll
        for (int k = 0; k < K; k++) support_mask<T, L1>(xb, sp, t * 32 * K + k * 32 + lane, aligned, okv[k]);
#pragma unroll
        for (int k = 0; k < K; k++)
            condat_slab<T, L1>(vals[k], okv[k], (t * 32 * K + k * 32 + lane) * V, INT64_MAX, true, r, st);
    }
    // final loop of Alg. 2: re-scan the chunk prefix before the last restart
    if (st.nJ > 0 && st.rs >= 0) {
        const int64_t tlast = st.rs / TILE;
        const int64_t before = st.rs;
        for (int64_t t = t0 + w; t <= tlast; t += W) {
            T vals[K][V];
            bool okv[K][V];
#pragma unroll
            for (int k = 0; k < K; k++) load_vec<T>(y, sp, t * 32 * K + k * 32 + lane, aligned, vals[k], okv[k]);
#pragma unroll
            for (int k = 0; k < K; k++) support_mask<T, L1>(xb, sp, t * 32 * K + k * 32 + lane, aligned, okv[k]);
#pragma unroll
            for (int k = 0; k < K; k++)
                condat_slab<T, L1>(vals[k], okv[k], (t * 32 * K + k * 32 + lane) * V, before, false, r, st);
        }
    }
    S_out = st.S;
    nJ_out = st.nJ;
}

// ---- one Newton pass (Alg. 4 evaluation) over all elements --------------------------------
// phi(lambda) = sum over y_i > -lambda of (y_i + lambda), phi'_- = #{y_i > -lambda} and, in the
// first pass only (FIRST), the ties #{y_i = -lambda} for phi'_+ and the NaN check.  The test
// is one 64-bit integer compare (FP64 data; NEG = sign of the threshold) or one float
// compare (FP32 data); y_i + lambda is formed only for the selected elements.
struct PassAcc {
    double acc64;
    df acc32;
    unsigned cm, ct;
    bool nan;
};

template <typename T, bool L1, bool NEG, bool FIRST>
__device__ __forceinline__ void newton_sweep(const T* __restrict__ y, const Span& sp, const Grp& gp, bool aligned,
                                             bool rev, unsigned long long tb, float rd, float ru, double lam, df Lm,
                                             PassAcc& pa) {
    constexpr int V = VecOf<T>::V;
    constexpr int U = kStreamU;
    using VT = typename VecOf<T>::type;
    const int lane = threadIdx.x & 31;
    const WarpSweep sw(span_qlo<V>(sp), span_qhi<V>(sp), U, gp.member, gp.g);
    for (int64_t it = 0; it < sw.count; it++) {
        const int64_t base = sw.base(it, rev);
        const bool full = aligned && base * V >= sp.lo && (base + 32 * U) * V <= sp.hi;  // warp-uniform
        T vv[U][V];
        bool okk[U][V];
        if (full) {
#pragma unroll
            for (int u = 0; u < U; u++) {
                const VT w = __ldg(reinterpret_cast<const VT*>(y) + base + u * 32 + lane);
                const T* s = reinterpret_cast<const T*>(&w);
#pragma unroll
                for (int j = 0; j < V; j++) {
                    vv[u][j] = s[j];
                    okk[u][j] = true;
                }
            }
        } else {
#pragma unroll
            for (int u = 0; u < U; u++) load_vec<T>(y, sp, base + u * 32 + lane, aligned, vv[u], okk[u]);
        }
        unsigned selm = 0;
#pragma unroll
        for (int uj = 0; uj < U * V; uj++) {
            const int u = uj / V, j = uj % V;
            bool sel, tie = false, nan = false;
            if constexpr (sizeof(T) == 8) {
                unsigned long long b = bits_of((double)vv[u][j]);
                if (L1) b &= 0x7FFFFFFFFFFFFFFFull;
                sel = NEG ? (b < tb) : ((long long)b > (long long)tb);
                if (FIRST) {
                    tie = !sel && (b == tb || ((b | tb) << 1) == 0ull);
                    nan = u64_is_nan(b);
                }
            } else {
                const float f = L1 ? fabsf((float)vv[u][j]) : (float)vv[u][j];
                sel = f > rd;
                if (FIRST) {
                    tie = !sel && f >= ru;
                    nan = f != f;
                }
            }
            sel = sel && okk[u][j];
            selm |= (sel ? 1u : 0u) << uj;
            if (FIRST) {
                pa.ct += (tie && okk[u][j]) ? 1u : 0u;
                pa.nan |= nan && okk[u][j];
            }
        }
        pa.cm += __popc(selm);
        // y_i + lambda, one loop trip per selected element: B300's FP64 pipe takes ~20 cycles
        // per warp instruction, so none may sit on the path of the unselected elements
        for (unsigned m = selm; m; m &= m - 1) {
            const T tv = pick2(vv, __ffs(m) - 1);
            if constexpr (sizeof(T) == 8) {
                // |y| by clearing the sign bit (an integer operation, not an FP64 one)
                const double ya = L1 ? __longlong_as_double((long long)(bits_of(tv) & 0x7FFFFFFFFFFFFFFFull)) : (double)tv;
                pa.acc64 += ya + lam;
            } else {
                pa.acc32 = df_add(pa.acc32, df_add_f(Lm, L1 ? fabsf((float)tv) : (float)tv));
            }
        }
    }
}

// per-block totals of a pass (fixed order) -> partials slot `par`
__device__ __forceinline__ void write_pass_partials(const Grp& gp, int par, double acc, unsigned cm, unsigned ct,
                                                    double* sh_d, unsigned* sh_u) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    acc = warp_sum(acc);
    cm = __reduce_add_sync(0xffffffffu, cm);
    ct = __reduce_add_sync(0xffffffffu, ct);
    if (lane == 0) {
        sh_d[wid] = acc;
        sh_u[wid] = cm;
        sh_u[NWARP + wid] = ct;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        unsigned long long c0 = 0, c1 = 0;
        for (int w = 0; w < NWARP; w++) {
            t += sh_d[w];
            c0 += sh_u[w];
            c1 += sh_u[NWARP + w];
        }
        const double pv[3] = {t, (double)c0, (double)(c0 + c1)};
        write_partials<3>(gp.part, gp.member, gp.g, par, pv);
    }
}

// grid totals of slot `par` by warp 0 (fixed order); valid in lane 0 of warp 0
__device__ __forceinline__ void warp0_grid_sums(const double* part, int G, int par, double (&out)[3]) {
    const int lane = threadIdx.x & 31;
    double v[3] = {0.0, 0.0, 0.0};
    for (int bI = lane; bI < G; bI += 32)
#pragma unroll
        for (int q = 0; q < 3; q++) v[q] += ld_cg(part + ((size_t)par * kPartialQ + q) * G + bI);
#pragma unroll
    for (int q = 0; q < 3; q++) out[q] = warp_sum(v[q]);
}

// ---- one projection by one group of blocks ------------------------------------------------
// A supplies the arrays, r, the options and the info slot; gp the group (member, size, span,
// header and partial sums).  The instance is the span [gp.sp.lo, gp.sp.hi) of y and x.
template <typename T, bool L1>
__device__ __forceinline__ void simplex_solve(const SimplexArgs& A, const Grp& gp) {
    constexpr int V = VecOf<T>::V;
    __shared__ double sh[kPartialQ][NWARP];
    __shared__ double bc[kPartialQ];
    __shared__ double sh_d[NWARP];
    __shared__ unsigned sh_u[2 * NWARP];
    // loop state written by thread 0 after each update, read by all threads
    __shared__ double s_lam, s_final;
    __shared__ int s_done, s_bad;
    const T* __restrict__ y = static_cast<const T*>(A.y);
    const Span sp = gp.sp;
    const int64_t n = sp.hi - sp.lo;
    const int64_t qlo = span_qlo<V>(sp), qhi = span_qhi<V>(sp);
    const int lane = threadIdx.x & 31;
    const int G = gp.g;
    const int64_t gwarp = (int64_t)gp.member * NWARP + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)G * NWARP;
    const bool aligned = A.aligned != 0;
    unsigned bar_target = (unsigned)G + (A.fault_inject ? 1u : 0u);
    const double r = A.r;

    // ------------------------------------------------------------------ pass 0: start
    double lam0 = 0.0, abs_sum = 0.0;
    int passes = 0, nchunks = 0, tile = 0;
    {
        double q[4] = {0.0, 0.0, 0.0, -INFINITY};  // sum y (l1: |y|), union sum, union size, max y (l1: |y|)
        const bool warm = A.init == CQK_INIT_WARM;
        const bool condat = A.init == CQK_INIT_CONDAT || warm;
        const bool sum_pass = L1 || !condat;
        bool bad = false;
        if (sum_pass) {
            df acc = df_make(0.0f);       // FP32 data
            LazyDf lz{0.0f, 0.0f};        // FP64 data in the df operating range, flushed into acc64
            double acc64 = 0.0;
            double acc_wide = 0.0;  // FP64 values outside the df operating range
            long long mxk = order_key(-INFINITY);
            float mxf = -INFINITY;
            const WarpSweep sw(qlo, qhi, kStreamU, gp.member, gp.g);
            for (int64_t it = 0; it < sw.count; it++) {
                const int64_t base = sw.base(it, false);
                T vv[kStreamU][V];
                bool okk[kStreamU][V];
#pragma unroll
                for (int u = 0; u < kStreamU; u++) load_vec<T>(y, sp, base + u * 32 + lane, aligned, vv[u], okk[u]);
                unsigned widem = 0;
#pragma unroll
                for (int uj = 0; uj < kStreamU * V; uj++) {
                    const int u = uj / V, j = uj % V;
                    if (!okk[u][j]) continue;
                    if constexpr (sizeof(T) == 8) {
                        const double t = L1 ? __longlong_as_double((long long)(bits_of(vv[u][j]) & 0x7FFFFFFFFFFFFFFFull))
                                            : (double)vv[u][j];
                        const bool inr = df_in_range(t, false);
                        const df st = split_f64_finite(t);
                        lazy_add(lz, df{inr ? st.hi : 0.0f, inr ? st.lo : 0.0f});
                        widem |= (inr ? 0u : 1u) << uj;
                        bad |= f64_is_nan(t);
                        const long long kk = order_key(t);
                        mxk = kk > mxk ? kk : mxk;
                    } else {
                        const float t = L1 ? fabsf((float)vv[u][j]) : (float)vv[u][j];
                        acc = df_add_f(acc, t);
                        bad |= (t != t);
                        mxf = fmaxf(mxf, t);
                    }
                }
                if constexpr (sizeof(T) == 8) {
                    // values outside the df operating range: exact FP64, one trip per element
                    for (unsigned m = widem; m; m &= m - 1) {
                        const T tv = pick2(vv, __ffs(m) - 1);
                        acc_wide += L1 ? fabs((double)tv) : (double)tv;
                    }
                    // fold the lazy pair (at most 64 terms) into FP64: one FP64 add per 4 sweeps
                    if ((it & 3) == 3) {
                        acc64 += df_to_f64_int(df{lz.hi, lz.lo});
                        lz = LazyDf{0.0f, 0.0f};
                    }
                }
            }
            if constexpr (sizeof(T) == 8) acc64 += df_to_f64_int(df{lz.hi, lz.lo});
            q[0] = df_to_f64(acc) + acc64 + acc_wide;
            if constexpr (sizeof(T) == 8) q[3] = from_order_key(mxk);
            else q[3] = (double)mxf;
            passes++;
        }
        // chunks of at least condat_chunk elements (the J updates are scalar FP64 work, which
        // a partition into many small chunks multiplies), at most one per warp
        const int64_t nchunk = min(nwarps, max((int64_t)1, (n + A.condat_chunk - 1) / A.condat_chunk));
        if (condat) {
            double Sw = 0.0;
            long long nJw = 0;
            if (gwarp < nchunk)
                condat_chunk<T, L1>(y, warm ? static_cast<const T*>(A.xbar) : nullptr, sp, aligned, r, gwarp, nchunk,
                                    Sw, nJw);
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
            if (badw && A.validate) atomicOr(&gp.hdr->flags, kFlagBadInput);
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
            write_partials<4>(gp.part, gp.member, G, 0, pv);
        }
        __syncthreads();
        if (!group_barrier(gp, bar_target, A.limit_ns, A.fault_inject != 0)) {
            if (threadIdx.x == 0) A.info->status = CQK_TIMEOUT;
            return;
        }
        bar_target += (unsigned)G;
        double red[4];
        grid_reduce<4>(gp.part, G, 0, 3, red, sh, bc);
        abs_sum = red[0];
        if (condat && red[2] > 0.0) {
            lam0 = (r - red[1]) / red[2];  // eq. (lambdaJ) on the union of the chunks' J
            nchunks = (int)nchunk;
            tile = 32 * condat_k<T>() * V;
        } else if (condat) {
            // warm start with an empty J_+ (no element of the estimate's support): Sec. 3.3
            const double y1 = (double)y[sp.lo];
            lam0 = fmax(r / (double)n, L1 ? -fabs(y1) : -y1);
            nchunks = (int)nchunk;
            tile = 32 * condat_k<T>() * V;
        } else if (A.init == CQK_INIT_GIVEN) {
            lam0 = fmax(A.lambda0, -red[3]);  // Alg. 4, line 1
        } else {
            lam0 = fmax((r - red[0]) / (double)n, -red[3]);  // eq. (CQKlambda0) with b = d = 1; Alg. 4 line 1
        }
    }
    bool bad_input = A.validate && (__ldcg(&gp.hdr->flags) & kFlagBadInput);

    // ------------------------------------------------------------------ Newton loop (Alg. 4)
    // thread 0 keeps the bracket and the stopping logic; every thread keeps lambda
    double lam = lam0, final_lam = lam0;
    double lower = -INFINITY, upper = INFINITY, slope = 0.0;  // thread 0
    int status = CQK_OK, stop = CQK_STOP_NONE, k = 0;         // thread 0 (status also all)
    bool copy = false;                                       // l1 ball, y inside
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
            PassAcc pa;
            pa.acc64 = 0.0;
            pa.acc32 = df_make(0.0f);
            pa.cm = pa.ct = 0u;
            pa.nan = false;
            const bool rev = (k & 1) == 0;
            const bool first = (k == 0);
            if constexpr (sizeof(T) == 8) {
                const GtThreshold g = make_gt(-lam);
                const df Lm = df_make(0.0f);
                if (g.neg) {
                    if (first) newton_sweep<T, L1, true, true>(y, sp, gp, aligned, rev, g.bits, 0.f, 0.f, lam, Lm, pa);
                    else newton_sweep<T, L1, true, false>(y, sp, gp, aligned, rev, g.bits, 0.f, 0.f, lam, Lm, pa);
                } else {
                    if (first) newton_sweep<T, L1, false, true>(y, sp, gp, aligned, rev, g.bits, 0.f, 0.f, lam, Lm, pa);
                    else newton_sweep<T, L1, false, false>(y, sp, gp, aligned, rev, g.bits, 0.f, 0.f, lam, Lm, pa);
                }
            } else {
                const float rd = f32_rd(-lam), ru = f32_ru(-lam);
                const df Lm = df_from_f64(lam);
                if (first) newton_sweep<T, L1, false, true>(y, sp, gp, aligned, rev, 0ull, rd, ru, lam, Lm, pa);
                else newton_sweep<T, L1, false, false>(y, sp, gp, aligned, rev, 0ull, rd, ru, lam, Lm, pa);
                pa.acc64 = df_to_f64(pa.acc32);
            }
            passes++;
            if (A.validate && first && __any_sync(0xffffffffu, pa.nan) && lane == 0)
                atomicOr(&gp.hdr->flags, kFlagBadInput);
            write_pass_partials(gp, par, pa.acc64, pa.cm, pa.ct, sh_d, sh_u);
            if (!group_barrier(gp, bar_target, A.limit_ns, A.fault_inject != 0)) {
                if (threadIdx.x == 0) A.info->status = CQK_TIMEOUT;
                return;
            }
            bar_target += (unsigned)G;
            if (threadIdx.x < 32) {
                double red[3];
                warp0_grid_sums(gp.part, G, par, red);
                if (threadIdx.x == 0) {
                    int done = 0, bad = 0;
                    double next = lam;
                    if (A.validate && first && (__ldcg(&gp.hdr->flags) & kFlagBadInput)) {
                        bad = 1;
                        done = 1;
                    } else {
                        const double phi = red[0], dminus = red[1], dplus = red[2];
                        const double gk = phi - r;
                        double step = 0.0;
                        if (k == 0) {
                            if (gk == 0.0) {
                                stop = CQK_STOP_EXACT;
                                done = 1;
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
                            done = 1;
                        } else {
                            upper = lam;
                            slope = dminus;
                            step = -gk / dminus;
                        }
                        double fin = lam;
                        if (!done && upper - lower < A.eps34 * fmax(fabs(upper), fabs(lower))) {
                            stop = CQK_STOP_BRACKET;
                            done = 1;
                        }
                        if (!done && fabs(step) < A.eps34) {
                            stop = CQK_STOP_STEP;
                            done = 1;
                            if (A.final_step) fin = lam + step;  // the Newton step already computed
                        }
                        if (!done) {
                            next = lam + step;
                            if (next == lam) {
                                stop = CQK_STOP_SAME;
                                done = 1;
                            }
                        }
                        s_final = fin;
                    }
                    s_lam = next;
                    s_done = done;
                    s_bad = bad;
                }
            }
            __syncthreads();
            par ^= 1;
            if (s_bad) {
                bad_input = true;
                status = CQK_BAD_INPUT;
                k++;
                break;
            }
            if (s_done) {
                final_lam = s_final;
                k++;
                break;
            }
            lam = s_lam;
            final_lam = lam;
            __syncthreads();  // s_lam is rewritten only after every thread has read it
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
        const WarpSweep sw(qlo, qhi, kStreamU, gp.member, gp.g);
        const bool rev = (k & 1) == 0;  // opposite direction to the last Newton pass
        for (int64_t it = 0; it < sw.count; it++) {
            const int64_t base = sw.base(it, rev);
            T vv[kStreamU][V];
            bool okk[kStreamU][V];
#pragma unroll
            for (int u = 0; u < kStreamU; u++) load_vec<T>(y, sp, base + u * 32 + lane, aligned, vv[u], okk[u]);
#pragma unroll
            for (int u = 0; u < kStreamU; u++) {
                const int64_t qw = base + u * 32;
                const int64_t q = qw + lane;
                const T(&v)[V] = vv[u];
                const bool(&ok)[V] = okk[u];
                T o[V];
                bool sel[V];
                unsigned selv = 0;
#pragma unroll
                for (int j = 0; j < V; j++) {
                    if constexpr (sizeof(T) == 8) {
                        const unsigned long long b = bits_of((double)v[j]);
                        const unsigned long long ab = b & 0x7FFFFFFFFFFFFFFFull;
                        sel[j] = ok[j] && (copy ? ab != 0ull : gt_bits(L1 ? ab : b, g));
                    } else {
                        const float f = (float)v[j];
                        sel[j] = ok[j] && (copy ? f != 0.0f : (L1 ? fabsf(f) : f) > rd);
                    }
                    o[j] = copy ? v[j] : T(0);
                    nz += sel[j];
                    selv |= (sel[j] && !copy ? 1u : 0u) << j;
                }
                // x_i = y_i + lambda (l1: sgn(y_i)(|y_i| + lambda)), one trip per selected element
                for (unsigned m = selv; m; m &= m - 1) {
                    const int j = __ffs(m) - 1;
                    const T vj = pick(v, j);
                    if constexpr (sizeof(T) == 8) {
                        // |x_i| = |y_i| + lambda > 0; the l1 ball copies the sign of y_i (bit operations)
                        const unsigned long long yb = bits_of((double)vj);
                        const double xm =
                            (L1 ? __longlong_as_double((long long)(yb & 0x7FFFFFFFFFFFFFFFull)) : (double)vj) + lamf;
                        const double xv =
                            L1 ? __longlong_as_double((long long)(bits_of(xm) | (yb & 0x8000000000000000ull))) : xm;
                        put(o, j, (T)xv);
                        sx += xm;
                    } else {
                        const float f = (float)vj;
                        const df t = df_add_f(Lm, L1 ? fabsf(f) : f);
                        float xv = __fadd_rn(t.hi, t.lo);
                        if (L1 && f < 0.0f) xv = -xv;
                        put(o, j, (T)xv);
                        sx32 = df_add_f(sx32, fabsf(xv));
                    }
                }
                store_vec<T>(x, sp, q, aligned, o);
                if (A.mask) store_mask<V>(A.mask, sp, qw, sel);
            }
        }
    }
    if constexpr (sizeof(T) == 4) sx = df_to_f64(sx32);
    double pv[2] = {sx, (double)nz}, tot[2];
    if (last_block_sums<2>(gp.part, gp.member, G, &gp.hdr->ticket, pv, tot, sh) && threadIdx.x == 0) {
        cqk_info inf;
        const double sumx = copy ? abs_sum : tot[0];  // inside the l1 ball x = y
        inf.lambda = final_lam;
        inf.residual = sumx - r;
        inf.abs_bx = sumx;
        inf.slope = slope;
        inf.lambda0 = lam0;
        inf.nfree = (int64_t)tot[1];
        inf.iters = k;
        const int e = *(volatile int*)&gp.hdr->error;
        inf.status = e ? e : status;
        inf.passes = passes + (bad_input ? 0 : 1);
        inf.stop = stop;
        inf.nchunks = nchunks;
        inf.tile = tile;
        *A.info = inf;
    }
}

template <typename T, bool L1>
__global__ void __launch_bounds__(NT, 2) simplex_kernel(SimplexArgs A) {
    Grp gp;
    gp.member = blockIdx.x;
    gp.g = gridDim.x;
    gp.sp = Span{0, A.n};
    gp.hdr = A.hdr;
    gp.part = A.part;
    simplex_solve<T, L1>(A, gp);
}

// A batch: blocks take (instance, member) slots from the queue until it is empty; every
// instance is the span [offsets[i], offsets[i+1]) of y and x, with its own r, info, header
// and partial sums.
struct SimplexBatchArgs {
    SimplexArgs base;
    const int64_t* offsets;
    const double* r;
    cqk_info* info;
    int64_t B;
    BatchRefs R;
};

template <typename T, bool L1>
__global__ void __launch_bounds__(NT, 2) simplex_batched_kernel(SimplexBatchArgs P) {
    while (true) {
        const Slot sl = next_slot(P.R, P.B);
        if (sl.inst < 0) break;
        const Grp gp = slot_group(P.R, P.offsets, sl);
        SimplexArgs A = P.base;
        A.r = P.r[sl.inst];
        A.info = P.info + sl.inst;
        const int64_t len = gp.sp.hi - gp.sp.lo;
        const bool r_ok = A.r > 0.0 && A.r < INFINITY;
        if (len <= 0 || !r_ok) {
            // no element: the simplex {sum x = r > 0} is empty, the l1 ball holds the empty x
            if (sl.member == 0 && threadIdx.x == 0) {
                if (len < 0 || !r_ok) write_plain_info(A.info, CQK_BAD_ARG, CQK_STOP_NONE, A.r);
                else if (L1) write_plain_info(A.info, CQK_OK, CQK_STOP_INSIDE, A.r);
                else write_plain_info(A.info, CQK_INFEASIBLE, CQK_STOP_NONE, A.r);
            }
            continue;
        }
        simplex_solve<T, L1>(A, gp);
    }
}

}  // namespace

int launch_simplex_batched(int64_t B, const int64_t* offsets, int dtype, const void* y, const double* r, int l1,
                           void* x, uint32_t* mask, cqk_info* info, const Opts& o, void* ws, cudaStream_t s) {
    SimplexBatchArgs P;
    memset(&P, 0, sizeof(P));
    SimplexArgs& A = P.base;
    A.y = y;
    A.x = x;
    A.mask = mask;
    A.init = o.init;
    A.lambda0 = o.lambda0;
    A.max_iter = o.max_iter;
    A.eps34 = kEps34F64;
    A.validate = o.validate;
    A.final_step = o.final_step;
    A.limit_ns = o.limit_ns;
    A.fault_inject = o.fault_inject;
    A.condat_chunk = o.condat_chunk;
    A.xbar = o.xbar;
    const bool xbar_misaligned = o.init == CQK_INIT_WARM && ((uintptr_t)o.xbar % 16) != 0;
    A.aligned = ((((uintptr_t)y) | ((uintptr_t)x)) % 16 == 0 && !xbar_misaligned) ? 1 : 0;
    P.offsets = offsets;
    P.r = r;
    P.info = info;
    P.B = B;
    P.R = BatchRefs::at(ws, B);
    const void* kern;
    if (dtype == CQK_F64)
        kern = l1 ? (const void*)simplex_batched_kernel<double, true> : (const void*)simplex_batched_kernel<double, false>;
    else
        kern = l1 ? (const void*)simplex_batched_kernel<float, true> : (const void*)simplex_batched_kernel<float, false>;
    int grid = persistent_grid(kern, NT, 0, INT64_MAX / 2, o.max_blocks);
    if (grid <= 0) return CQK_CUDA_ERROR;
    if ((int64_t)grid > B * kMaxGroup) grid = (int)(B * kMaxGroup);
    const int64_t per_block = o.group_elems > 0 ? o.group_elems : kSimplexGroupElems;
    int rc = plan_batch(offsets, B, per_block, grid, ws, s);
    if (rc != CQK_OK) return rc;
    void* args[] = {&P};
    cudaError_t e = cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(NT), args, 0, s);
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return CQK_CUDA_ERROR;
    }
    return CQK_OK;
}

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
    A.condat_chunk = o.condat_chunk;
    A.xbar = o.xbar;
    const bool xbar_misaligned = o.init == CQK_INIT_WARM && ((uintptr_t)o.xbar % 16) != 0;
    A.hdr = static_cast<WsHeader*>(ws);
    A.part = reinterpret_cast<double*>(static_cast<char*>(ws) + sizeof(WsHeader));
    A.aligned = ((((uintptr_t)y) | ((uintptr_t)x)) % 16 == 0 && !xbar_misaligned) ? 1 : 0;
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
