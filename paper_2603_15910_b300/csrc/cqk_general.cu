// cqk_general.cu -- the general CQK solve (Alg. 1) and the stand-alone phi evaluation.
//
// One cooperative launch per solve:
//   pass 0   s = sum b_i a_i/d_i, q = sum b_i^2/d_i -> lambda_0 = (r - s)/q  (eq. (CQKlambda0))
//   pass k   at lambda_k, for every i, v_i = a_i + lambda_k b_i and, with no division
//            (b_i, d_i > 0), the status of x_i(lambda_k) of eq. (xopt):
//              v_i <  d_i l_i  -> x_i = l_i;   v_i > d_i u_i -> x_i = u_i;   else x_i = v_i/d_i
//            and the sums
//              phi    = sum b_i x_i                                 (eq. (opt))
//              phi'_+ = sum over lower_i <= lambda < upper_i of b_i^2/d_i   (eq. (phideriv))
//              phi'_- = sum over lower_i <  lambda <= upper_i of b_i^2/d_i
//              sum |b_i x_i|                                        (criterion 1, Sec. 4)
//            then the Alg. 1 update, computed identically by every block.
//   pass bp  (only when the needed lateral derivative is 0) the closest breakpoint
//            (d_i l_i - a_i)/b_i or (d_i u_i - a_i)/b_i strictly right / left of lambda (Alg. 1),
//            in FP64 exactly as defined.
//   final    x = x(lambda*) (bounds copied exactly), free mask, b'x - r of the stored x.
//
// lambda_k "on" a breakpoint: v_i = d_i l_i holds when lambda equals the breakpoint
// lower_i; after a breakpoint step lambda is the FP64-rounded breakpoint, so v_i - d_i l_i
// is a rounding residue.  |v_i - d_i l_i| <= 2^-42 (|a_i| + |lambda b_i| + |d_i l_i|) is
// therefore read as v_i = d_i l_i (the element sits at its breakpoint), and likewise for u.
//
// Per-element arithmetic: double-float (cqk_device.cuh) for FP64 data in the df operating
// range, exact FP64 per lane otherwise, and FP32 with a df multiplier for FP32 data.
#include <string.h>

#include "cqk_block.cuh"

namespace cqk {
namespace {

constexpr float kTieRel = 2.2737367544323206e-13f;  // 2^-42

struct GeneralArgs {
    int64_t n;
    const void *a, *b, *d, *l, *u;
    void* x;
    uint32_t* mask;
    cqk_info* info;
    double* phi_out;  // phi-only mode: 4 doubles
    double r;
    int init;
    double lambda0;
    int max_iter;
    double eps34_stop1;  // criterion 1 (storage precision)
    double eps34;        // criteria 2 and 3 (lambda is FP64)
    int validate;
    int final_step;
    int aligned;
    int phi_only;
    unsigned long long limit_ns;
    int fault_inject;
    WsHeader* hdr;
    double* part;
};

// Per-thread accumulators of one pass.  The df sums are flushed into the FP64 ones every
// kFlushEvery sweep iterations (16 vectors), bounding the df summation error by ~16*V*2^-47 of
// the flushed partial sums.
constexpr int kFlushEvery = 8;   // sweep iterations (kGenU vectors each) between flushes
constexpr int kGenU = 2;         // 16-byte vectors per array in flight per lane
struct EvalAcc {
    df phi, absbx, sfree;
    double phi64, absbx64, sfree64, satl, satu;
    long long nfree;
    bool bad;
    __device__ void init() {
        phi = absbx = sfree = df_make(0.0f);
        phi64 = absbx64 = sfree64 = satl = satu = 0.0;
        nfree = 0;
        bad = false;
    }
    __device__ void flush() {
        phi64 += df_to_f64(phi);
        absbx64 += df_to_f64(absbx);
        sfree64 += df_to_f64(sfree);
        phi = absbx = sfree = df_make(0.0f);
    }
};

// status of one element: 0 free, 1 x = l, 2 x = u
struct Cls {
    int c;
    bool tieL, tieU;
};

// ---- FP64 data, exact FP64 (values outside the df range) -------------------------------
__device__ __noinline__ double elem_f64_exact(double a, double b, double d, double l, double u, double lam,
                                                 EvalAcc& acc, bool want_acc, Cls& cl) {
    const double lb = lam * b;
    const double v = a + lb;
    const double dl = isinf(l) ? l : d * l;
    const double du = isinf(u) ? u : d * u;
    const double sc = fabs(a) + fabs(lb);
    const bool tieL = !isinf(l) && fabs(v - dl) <= 2.2737367544323206e-13 * (sc + fabs(dl));
    const bool tieU = !isinf(u) && fabs(v - du) <= 2.2737367544323206e-13 * (sc + fabs(du));
    cl.tieL = tieL;
    cl.tieU = tieU;
    double x;
    if (tieL || v < dl) { x = l; cl.c = 1; }
    else if (tieU || v > du) { x = u; cl.c = 2; }
    else { x = v / d; cl.c = 0; }
    if (want_acc) {
        const double bx = b * x;
        acc.phi64 += bx;
        acc.absbx64 += fabs(bx);
        const double w = b * b / d;
        if (cl.c == 0) acc.sfree64 += w;
        if (tieL && !tieU) acc.satl += w;
        if (tieU && !tieL) acc.satu += w;
    }
    return x;
}

// ---- FP64 data in the df range ----------------------------------------------------------
__device__ __forceinline__ df elem_df(double a, double b, double d, double l, double u, df Lm, EvalAcc& acc,
                                      bool want_acc, Cls& cl, df& beta_out) {
    const df A = split_f64(a), B = split_f64(b), D = split_f64(d), Lo = split_f64(l), Up = split_f64(u);
    const df lb = df_mul(Lm, B);
    const df v = df_add(A, lb);
    const bool linf = isinf(Lo.hi), uinf = isinf(Up.hi);
    const df dl = linf ? Lo : df_mul(D, Lo);
    const df du = uinf ? Up : df_mul(D, Up);
    const float sc = fabsf(A.hi) + fabsf(lb.hi);
    const df eL = df_add(v, df_neg(dl)), eU = df_add(v, df_neg(du));
    const bool tieL = !linf && fabsf(eL.hi) <= kTieRel * (sc + fabsf(dl.hi));
    const bool tieU = !uinf && fabsf(eU.hi) <= kTieRel * (sc + fabsf(du.hi));
    cl.tieL = tieL;
    cl.tieU = tieU;
    const bool below = tieL || (!linf && eL.hi < 0.0f);
    const bool above = !below && (tieU || (!uinf && eU.hi > 0.0f));
    cl.c = below ? 1 : (above ? 2 : 0);
    const float rd = rcp_approx(D.hi);
    const df invd = df_div(df_make(1.0f), D, rd);
    df x = df_mul(v, invd);
    if (below) x = Lo;
    if (above) x = Up;
    if (want_acc) {
        const df bx = df_mul(B, x);
        acc.phi = df_add(acc.phi, bx);
        acc.absbx = df_add(acc.absbx, bx.hi < 0.0f ? df_neg(bx) : bx);
        const df beta = df_mul(df_mul(B, B), invd);
        acc.sfree = df_add(acc.sfree, cl.c == 0 ? beta : df_make(0.0f));
        beta_out = beta;
    }
    return x;
}

// sanity checks of Sec. 5.1.1 on the bit patterns: d > 0, b > 0 finite; a finite; l <= u;
// no NaN (integer pipe only)
__device__ __forceinline__ bool bad_elem(double a, double b, double d, double l, double u) {
    return !f64_pos_finite(d) || !f64_pos_finite(b) || !f64_is_finite(a) || f64_is_nan(l) || f64_is_nan(u) ||
           order_key(l) > order_key(u);
}

// ---- FP32 data -----------------------------------------------------------------------------
// v = a + lambda b with lambda a float pair: TwoProd + TwoSum; the tests compare the df v
// with the exact products d*l, d*u (TwoProd); x = v/d rounded to float; b*x, |b x| and
// b^2/d are accumulated in df.
__device__ __forceinline__ float elem_f32(float a, float b, float d, float l, float u, df Lm, EvalAcc& acc,
                                          bool want_acc, Cls& cl, df& beta_out) {
    const df lb = df_mul_f(Lm, b);
    const df v = df_add_f(lb, a);
    const bool linf = isinf(l), uinf = isinf(u);
    const df dl = linf ? df_make(l) : two_prod(d, l);
    const df du = uinf ? df_make(u) : two_prod(d, u);
    const float sc = fabsf(a) + fabsf(lb.hi);
    const df eL = df_add(v, df_neg(dl)), eU = df_add(v, df_neg(du));
    const bool tieL = !linf && fabsf(eL.hi) <= kTieRel * (sc + fabsf(dl.hi));
    const bool tieU = !uinf && fabsf(eU.hi) <= kTieRel * (sc + fabsf(du.hi));
    cl.tieL = tieL;
    cl.tieU = tieU;
    const bool below = tieL || (!linf && eL.hi < 0.0f);
    const bool above = !below && (tieU || (!uinf && eU.hi > 0.0f));
    cl.c = below ? 1 : (above ? 2 : 0);
    const float rd = rcp_approx(d);
    const float vh = __fadd_rn(v.hi, v.lo);
    float x = __fmul_rn(vh, rd);
    x = fmaf(fmaf(-x, d, vh), rd, x);  // one correction: ~1 ulp
    if (below) x = l;
    if (above) x = u;
    if (want_acc) {
        const df bx = two_prod(b, x);
        acc.phi = df_add(acc.phi, bx);
        acc.absbx = df_add(acc.absbx, bx.hi < 0.0f ? df_neg(bx) : bx);
        const float bb = __fmul_rn(b, b);
        float beta = __fmul_rn(bb, rd);
        beta = fmaf(fmaf(-beta, d, bb), rd, beta);
        acc.sfree = df_add_f(acc.sfree, cl.c == 0 ? beta : 0.0f);
        beta_out = df_make(beta);
    }
    return x;
}

// ---- one pass over all elements: accumulate (write_x = false) or write x / mask / residual
template <typename T>
__device__ __forceinline__ void eval_pass(const GeneralArgs& A, double lam, bool write_x, bool check, bool rev,
                                          EvalAcc& acc) {
    constexpr int V = VecOf<T>::V;
    constexpr int U = kGenU;
    const T* __restrict__ pa = static_cast<const T*>(A.a);
    const T* __restrict__ pb = static_cast<const T*>(A.b);
    const T* __restrict__ pd = static_cast<const T*>(A.d);
    const T* __restrict__ pl = static_cast<const T*>(A.l);
    const T* __restrict__ pu = static_cast<const T*>(A.u);
    T* __restrict__ px = static_cast<T*>(A.x);
    const int64_t n = A.n;
    const int64_t nv = (n + V - 1) / V;
    const int lane = threadIdx.x & 31;
    const bool aligned = A.aligned != 0;
    const df Lm = df_from_f64(lam);
    const bool lam_ok = fabs(lam) <= 1.152921504606847e18;  // 2^60
    const WarpSweep sw(nv, U);
    int steps = 0;
    for (int64_t it = 0; it < sw.count; it++) {
        if (++steps == kFlushEvery) {
            acc.flush();
            steps = 0;
        }
        const int64_t base = sw.base(it, rev);
        T va[U][V], vb[U][V], vd[U][V], vl[U][V], vu[U][V];
        bool ok[U][V];
#pragma unroll
        for (int w = 0; w < U; w++) {
            const int64_t q = base + w * 32 + lane;
            load_vec<T>(pa, n, q, aligned, va[w], ok[w]);
            load_vec<T>(pb, n, q, aligned, vb[w], ok[w]);
            load_vec<T>(pd, n, q, aligned, vd[w], ok[w]);
            load_vec<T>(pl, n, q, aligned, vl[w], ok[w]);
            load_vec<T>(pu, n, q, aligned, vu[w], ok[w]);
        }
#pragma unroll
        for (int w = 0; w < U; w++) {
            const int64_t qw = base + w * 32;
            const int64_t q = qw + lane;
            T xo[V];
            bool fr[V];
            df beta[V];
            unsigned tiem = 0, widem = 0;
#pragma unroll
            for (int j = 0; j < V; j++) {
                fr[j] = false;
                xo[j] = T(0);
                beta[j] = df_make(0.0f);
                if (!ok[w][j]) continue;
                const T a = va[w][j], b = vb[w][j], d = vd[w][j], l = vl[w][j], u = vu[w][j];
                Cls cl;
                if constexpr (sizeof(T) == 8) {
                    if (check) acc.bad |= bad_elem(a, b, d, l, u);
                    const bool inr = lam_ok && df_in_range(a, false) && df_in_range(b, false) &&
                                     df_in_range(d, false) && df_in_range(l, true) && df_in_range(u, true);
                    if (!inr) {
                        widem |= 1u << j;
                        continue;
                    }
                    const df xv = elem_df(a, b, d, l, u, Lm, acc, !write_x, cl, beta[j]);
                    if (write_x) xo[j] = cl.c == 1 ? l : (cl.c == 2 ? u : df_to_f64(xv));
                } else {
                    if (check) acc.bad |= bad_elem(a, b, d, l, u);
                    xo[j] = elem_f32(a, b, d, l, u, Lm, acc, !write_x, cl, beta[j]);
                }
                fr[j] = cl.c == 0;
                tiem |= ((cl.tieL && !cl.tieU) ? 1u : 0u) << (2 * j);
                tiem |= ((cl.tieU && !cl.tieL) ? 2u : 0u) << (2 * j);
            }
            // rare cases, one loop trip per element concerned (a data-dependent loop keeps FP64
            // instructions off the common path): elements on a breakpoint (lateral-slope ties)
            // and FP64 values outside the df operating range (exact FP64)
            if (!write_x) {
                for (unsigned m = tiem; m; m &= m - 1) {
                    const int bit = __ffs(m) - 1;
                    const double bj = df_to_f64(pick(beta, bit >> 1));
                    if (bit & 1) acc.satu += bj;
                    else acc.satl += bj;
                }
            }
            if constexpr (sizeof(T) == 8) {
                for (unsigned m = widem; m; m &= m - 1) {
                    const int j = __ffs(m) - 1;
                    Cls cl;
                    const T xj = elem_f64_exact(pick(va[w], j), pick(vb[w], j), pick(vd[w], j), pick(vl[w], j),
                                                pick(vu[w], j), lam, acc, !write_x, cl);
                    put(xo, j, xj);
                    put(fr, j, cl.c == 0);
                }
            }
            if (write_x) {
                // sums of the stored x: b'x, sum |b x|, number of free variables
                unsigned wide2 = 0;
#pragma unroll
                for (int j = 0; j < V; j++) {
                    if (!ok[w][j]) continue;
                    const T b = vb[w][j];
                    if constexpr (sizeof(T) == 8) {
                        const bool inr = df_in_range(b, false) && df_in_range(xo[j], false);
                        const df p = inr ? df_mul(split_f64(b), split_f64(xo[j])) : df_make(0.0f);
                        acc.phi = df_add(acc.phi, p);
                        acc.absbx = df_add(acc.absbx, p.hi < 0.0f ? df_neg(p) : p);
                        wide2 |= (inr ? 0u : 1u) << j;
                    } else {
                        const df p = two_prod((float)b, (float)xo[j]);
                        acc.phi = df_add(acc.phi, p);
                        acc.absbx = df_add(acc.absbx, p.hi < 0.0f ? df_neg(p) : p);
                    }
                    acc.nfree += fr[j];
                }
                for (unsigned m = wide2; m; m &= m - 1) {
                    const int j = __ffs(m) - 1;
                    const double bx = (double)pick(vb[w], j) * (double)pick(xo, j);
                    acc.phi64 += bx;
                    acc.absbx64 += fabs(bx);
                }
                if (px) store_vec<T>(px, n, q, aligned, xo);
                if (A.mask) store_mask<V>(A.mask, n, qw, fr);
            }
        }
    }
}

// closest breakpoint strictly right (dir > 0) / left (dir < 0) of lam, FP64 as defined
template <typename T>
__device__ __forceinline__ double breakpoint_pass(const GeneralArgs& A, double lam, int dir) {
    const T* pa = static_cast<const T*>(A.a);
    const T* pb = static_cast<const T*>(A.b);
    const T* pd = static_cast<const T*>(A.d);
    const T* pl = static_cast<const T*>(A.l);
    const T* pu = static_cast<const T*>(A.u);
    double best = dir > 0 ? INFINITY : -INFINITY;
    const int64_t stride = (int64_t)gridDim.x * NT;
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < A.n; i += stride) {
        const double a = pa[i], b = pb[i], d = pd[i], l = pl[i], u = pu[i];
        const double c0 = (d * l - a) / b, c1 = (d * u - a) / b;
        if (dir > 0) {
            if (isfinite(c0) && c0 > lam) best = fmin(best, c0);
            if (isfinite(c1) && c1 > lam) best = fmin(best, c1);
        } else {
            if (isfinite(c0) && c0 < lam) best = fmax(best, c0);
            if (isfinite(c1) && c1 < lam) best = fmax(best, c1);
        }
    }
    return best;
}

template <typename T>
__device__ __forceinline__ void lambda0_pass(const GeneralArgs& A, double& s_out, double& q_out) {
    constexpr int V = VecOf<T>::V;
    const T* __restrict__ pa = static_cast<const T*>(A.a);
    const T* __restrict__ pb = static_cast<const T*>(A.b);
    const T* __restrict__ pd = static_cast<const T*>(A.d);
    const int64_t n = A.n;
    const int64_t nv = (n + V - 1) / V;
    const int lane = threadIdx.x & 31;
    const bool aligned = A.aligned != 0;
    df s = df_make(0.0f), q = df_make(0.0f);
    double s64 = 0.0, q64 = 0.0;
    int steps = 0;
    constexpr int U = kGenU;
    const WarpSweep sw(nv, U);
    for (int64_t it = 0; it < sw.count; it++) {
        if (++steps == kFlushEvery) {
            s64 += df_to_f64(s);
            q64 += df_to_f64(q);
            s = q = df_make(0.0f);
            steps = 0;
        }
        const int64_t base = sw.base(it, false);
        T va[U][V], vb[U][V], vd[U][V];
        bool ok[U][V];
#pragma unroll
        for (int w = 0; w < U; w++) {
            load_vec<T>(pa, n, base + w * 32 + lane, aligned, va[w], ok[w]);
            load_vec<T>(pb, n, base + w * 32 + lane, aligned, vb[w], ok[w]);
            load_vec<T>(pd, n, base + w * 32 + lane, aligned, vd[w], ok[w]);
        }
        unsigned wide = 0;
#pragma unroll
        for (int wj = 0; wj < U * V; wj++) {
            const int w = wj / V, j = wj % V;
            if (!ok[w][j]) continue;
            const T a = va[w][j], b = vb[w][j], d = vd[w][j];
            if constexpr (sizeof(T) == 8) {
                const bool inr = df_in_range(a, false) && df_in_range(b, false) && df_in_range(d, false) &&
                                 f64_pos_finite(d);
                const df B = split_f64(inr ? b : 1.0), D = split_f64(inr ? d : 1.0);
                const df wgt = df_mul(B, df_div(df_make(1.0f), D, rcp_approx(D.hi)));
                s = df_add(s, inr ? df_mul(wgt, split_f64(a)) : df_make(0.0f));
                q = df_add(q, inr ? df_mul(wgt, B) : df_make(0.0f));
                wide |= (inr ? 0u : 1u) << wj;
            } else {
                const float rd = rcp_approx(d);
                float wgt = __fmul_rn(b, rd);
                wgt = fmaf(fmaf(-wgt, d, b), rd, wgt);
                s = df_add(s, two_prod(wgt, a));
                q = df_add(q, two_prod(wgt, b));
            }
        }
        for (unsigned m = wide; m; m &= m - 1) {  // exact FP64 outside the df range (rare)
            const int wj = __ffs(m) - 1;
            const double a = pick(va[wj / V], wj % V), b = pick(vb[wj / V], wj % V), d = pick(vd[wj / V], wj % V);
            s64 += b * a / d;
            q64 += b * b / d;
        }
    }
    s_out = df_to_f64(s) + s64;
    q_out = df_to_f64(q) + q64;
}

#define CQK_BARRIER_OR_LEAVE()                                                  \
    do {                                                                        \
        if (!grid_barrier(bar, bar_target, err, A.limit_ns, CQK_TIMEOUT)) {     \
            if (threadIdx.x == 0) A.info->status = CQK_TIMEOUT;                 \
            return;                                                             \
        }                                                                       \
        bar_target += (unsigned)G;                                              \
    } while (0)

template <typename T>
__global__ void __launch_bounds__(NT, 2) general_kernel(GeneralArgs A) {
    __shared__ double sh[kPartialQ][NWARP];
    __shared__ double bc[kPartialQ];
    const int G = gridDim.x;
    unsigned bar_target = (unsigned)G + (A.fault_inject ? 1u : 0u);
    unsigned* bar = &A.hdr->bar_count;
    int* err = &A.hdr->error;
    const double r = A.r;
    int passes = 0, par = 0;

    if (A.phi_only) {  // cqk_phi: one evaluation at A.lambda0 (and x when requested)
        EvalAcc acc;
        acc.init();
        eval_pass<T>(A, A.lambda0, false, false, false, acc);
        acc.flush();
        double pv[3] = {acc.phi64, acc.sfree64, acc.absbx64};
        double pt[2] = {acc.satl, acc.satu};
        block_sum<3>(pv, sh);
        block_sum<2>(pt, sh);
        if (threadIdx.x == 0) {
            const double w5[5] = {pv[0], pv[1], pv[2], pt[0], pt[1]};
            write_partials<5>(A.part, 0, w5);
        }
        if (A.x) {
            EvalAcc acc2;
            acc2.init();
            eval_pass<T>(A, A.lambda0, true, false, true, acc2);
        }
        double dummy[1] = {0.0}, tot[1];
        if (last_block_sums<1>(A.part, &A.hdr->ticket, dummy, tot, sh)) {
            double red[5];
            grid_reduce<5>(A.part, 0, -1, red, sh, bc);
            if (threadIdx.x == 0) {
                A.phi_out[0] = red[0];
                A.phi_out[1] = red[1] + red[3];
                A.phi_out[2] = red[1] + red[4];
                A.phi_out[3] = red[2];
            }
        }
        return;
    }

    // ---- pass 0: lambda_0
    double lam0 = A.lambda0;
    if (A.init == CQK_INIT_FORMULA) {
        double s, q;
        lambda0_pass<T>(A, s, q);
        double pv[2] = {s, q};
        block_sum<2>(pv, sh);
        write_partials<2>(A.part, par, pv);
        CQK_BARRIER_OR_LEAVE();
        double red[2];
        grid_reduce<2>(A.part, par, -1, red, sh, bc);
        par ^= 1;
        lam0 = (r - red[0]) / red[1];  // eq. (CQKlambda0), J = all variables
        passes++;
    }

    // ---- Alg. 1
    double lam = lam0, lower = -INFINITY, upper = INFINITY, phi_lower = NAN, phi_upper = NAN, slope = 0.0;
    double final_lam = lam;
    int status = CQK_OK, stop = CQK_STOP_NONE, k = 0;
    bool bad_input = false;
    for (k = 0;; k++) {
        if (k >= A.max_iter) {
            status = CQK_MAXITER;
            break;
        }
        EvalAcc acc;
        acc.init();
        eval_pass<T>(A, lam, false, k == 0 && A.validate, (k & 1) == 1, acc);
        acc.flush();
        passes++;
        if (__any_sync(0xffffffffu, acc.bad) && (threadIdx.x & 31) == 0) atomicOr(&A.hdr->flags, kFlagBadInput);
        double pv[5] = {acc.phi64, acc.sfree64, acc.satl, acc.satu, acc.absbx64};
        block_sum<5>(pv, sh);
        write_partials<5>(A.part, par, pv);
        CQK_BARRIER_OR_LEAVE();
        double red[5];
        grid_reduce<5>(A.part, par, -1, red, sh, bc);
        par ^= 1;
        if (k == 0 && A.validate && (__ldcg(&A.hdr->flags) & kFlagBadInput)) {
            bad_input = true;
            status = CQK_BAD_INPUT;
            k++;
            break;
        }
        const double phi = red[0], dplus = red[1] + red[2], dminus = red[1] + red[3], absbx = red[4];
        const double g = phi - r;
        final_lam = lam;
        if (g == 0.0) {
            stop = CQK_STOP_EXACT;
            k++;
            break;
        }
        if (fabs(g) < A.eps34_stop1 * (absbx + fabs(r))) {
            stop = CQK_STOP_RESIDUAL;
            if (A.final_step) {
                double s = g < 0 ? (dplus > 0 ? -g / dplus : 0.0) : (dminus > 0 ? -g / dminus : 0.0);
                const double t = lam + s;
                if (g < 0 && !(t < upper)) s = 0.0;
                if (g > 0 && !(t > lower)) s = 0.0;
                final_lam = lam + s;
            }
            k++;
            break;
        }
        double next = lam;
        int need_bp = 0;
        bool done = false;
        if (g < 0) {
            lower = lam;
            phi_lower = phi;
            if (dplus > 0) {
                slope = dplus;
                const double step = -g / dplus;
                const double t = lam + step;
                if (fabs(step) < A.eps34) {
                    stop = CQK_STOP_STEP;
                    if (A.final_step && t < upper) final_lam = t;
                    done = true;
                } else if (t < upper) {
                    next = t;
                } else {
                    next = lower - (phi_lower - r) * (upper - lower) / (phi_upper - phi_lower);
                }
            } else {
                need_bp = +1;
            }
        } else {
            upper = lam;
            phi_upper = phi;
            if (dminus > 0) {
                slope = dminus;
                const double step = -g / dminus;
                const double t = lam + step;
                if (fabs(step) < A.eps34) {
                    stop = CQK_STOP_STEP;
                    if (A.final_step && t > lower) final_lam = t;
                    done = true;
                } else if (t > lower) {
                    next = t;
                } else {
                    next = lower - (phi_lower - r) * (upper - lower) / (phi_upper - phi_lower);
                }
            } else {
                need_bp = -1;
            }
        }
        if (done) {
            k++;
            break;
        }
        if (need_bp) {
            // closest breakpoint right of the lower end / left of the upper end (Alg. 1); the
            // block maximum of (-bp) or (bp) keeps one reduction code path
            double bp = breakpoint_pass<T>(A, need_bp > 0 ? lower : upper, need_bp);
            bp = need_bp > 0 ? -bp : bp;
            bp = warp_max(bp);
            if ((threadIdx.x & 31) == 0) sh[0][threadIdx.x >> 5] = bp;
            __syncthreads();
            if (threadIdx.x == 0) {
                double m = -INFINITY;
                for (int w = 0; w < NWARP; w++) m = fmax(m, sh[0][w]);
                const double pvb[1] = {m};
                write_partials<1>(A.part, par, pvb);
            }
            __syncthreads();
            passes++;
            CQK_BARRIER_OR_LEAVE();
            double redb[1];
            grid_reduce<1>(A.part, par, 0, redb, sh, bc);
            par ^= 1;
            const double m = need_bp > 0 ? -redb[0] : redb[0];
            if (!isfinite(m)) {
                status = CQK_INFEASIBLE;
                k++;
                break;
            }
            next = m;
        }
        if (upper - lower < A.eps34 * fmax(fabs(upper), fabs(lower))) {
            stop = CQK_STOP_BRACKET;
            k++;
            break;
        }
        if (next == lam) {
            stop = CQK_STOP_SAME;
            k++;
            break;
        }
        lam = next;
        final_lam = lam;
    }

    // ---- final pass: x = x(lambda*), mask, sums of the stored x
    EvalAcc acc;
    acc.init();
    if (!bad_input && status != CQK_INFEASIBLE) {
        eval_pass<T>(A, final_lam, true, false, (k & 1) == 1, acc);
        passes++;
    }
    acc.flush();
    double pv[3] = {acc.phi64, acc.absbx64, (double)acc.nfree}, tot[3];
    if (last_block_sums<3>(A.part, &A.hdr->ticket, pv, tot, sh) && threadIdx.x == 0) {
        cqk_info inf;
        inf.lambda = final_lam;
        inf.residual = tot[0] - r;
        inf.abs_bx = tot[1];
        inf.slope = slope;
        inf.lambda0 = lam0;
        inf.nfree = (int64_t)tot[2];
        inf.iters = k;
        const int e = *(volatile int*)&A.hdr->error;
        inf.status = e ? e : status;
        inf.passes = passes;
        inf.stop = stop;
        inf.nchunks = 0;
        inf.tile = 0;
        *A.info = inf;
    }
}

GeneralArgs make_args(int64_t n, const void* a, const void* b, const void* d, const void* l, const void* u, void* x,
                      void* ws, int dtype) {
    GeneralArgs A;
    memset(&A, 0, sizeof(A));
    A.n = n;
    A.a = a;
    A.b = b;
    A.d = d;
    A.l = l;
    A.u = u;
    A.x = x;
    A.hdr = static_cast<WsHeader*>(ws);
    A.part = reinterpret_cast<double*>(static_cast<char*>(ws) + sizeof(WsHeader));
    const uintptr_t all = (uintptr_t)a | (uintptr_t)b | (uintptr_t)d | (uintptr_t)l | (uintptr_t)u | (uintptr_t)x;
    A.aligned = (all % 16 == 0) ? 1 : 0;
    A.eps34 = kEps34F64;
    A.eps34_stop1 = dtype == CQK_F64 ? kEps34F64 : kEps34F32;
    return A;
}

int launch(GeneralArgs A, int dtype, int max_blocks, cudaStream_t s, void* ws) {
    const void* kern = dtype == CQK_F64 ? (const void*)general_kernel<double> : (const void*)general_kernel<float>;
    const int64_t vec = dtype == CQK_F64 ? 2 : 4;
    const int grid = persistent_grid(kern, NT, 0, (A.n + vec - 1) / vec, max_blocks);
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

}  // namespace

int launch_general(int64_t n, int dtype, const void* a, const void* b, const void* d, const void* l, const void* u,
                   double r, void* x, uint32_t* mask, cqk_info* info, const Opts& o, void* ws, cudaStream_t s) {
    GeneralArgs A = make_args(n, a, b, d, l, u, x, ws, dtype);
    A.mask = mask;
    A.info = info;
    A.r = r;
    A.init = o.init;
    A.lambda0 = o.lambda0;
    A.max_iter = o.max_iter;
    A.validate = o.validate;
    A.final_step = o.final_step;
    A.limit_ns = o.limit_ns;
    A.fault_inject = o.fault_inject;
    return launch(A, dtype, o.max_blocks, s, ws);
}

int launch_phi(int64_t n, int dtype, const void* a, const void* b, const void* d, const void* l, const void* u,
               double lambda, void* x, double* out, void* ws, cudaStream_t s) {
    GeneralArgs A = make_args(n, a, b, d, l, u, x, ws, dtype);
    A.phi_only = 1;
    A.lambda0 = lambda;
    A.phi_out = out;
    A.limit_ns = 2000000000ull;
    return launch(A, dtype, 0, s, ws);
}

}  // namespace cqk
