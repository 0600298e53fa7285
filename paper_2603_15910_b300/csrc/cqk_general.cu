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

#include "cqk_batch.cuh"
#include "cqk_stage.cuh"

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
    int staged;  // arrays staged through shared memory by bulk copies (aligned data)
    const void* xbar;  // CQK_INIT_WARM: primal estimate
    int phi_only;
    unsigned long long limit_ns;
    int fault_inject;
    WsHeader* hdr;
    double* part;
};

// Per-thread accumulators of one pass.  The df sums (lazily normalised) are flushed into the
// FP64 ones every kFlushEvery sweep iterations, bounding the df summation error by
// ~16*V*2^-46 of the flushed partial sums.
constexpr int kFlushEvery = 8;  // sweep iterations (kGenU vectors each) between flushes
// 16-byte vectors per array in flight per lane (unaligned data), and bytes per array of one
// bulk-copy stage (aligned data: 2 vectors per thread and array, 1 in the half-unroll build)
#ifdef CQK_UNROLL_HALF
constexpr int kGenU = 1;
constexpr int kGenTileBytes = 16 * NT;
#else
constexpr int kGenU = 2;
constexpr int kGenTileBytes = 32 * NT;
#endif
constexpr int kCheckAll = 0, kCheckBounds = 1, kChecked = 2;  // per-element checks of a pass (eval_vec)
// The lambda_0 pass reads l and u too for FP64 data (their checks are integer work that the
// first Newton pass would otherwise carry); for FP32 data it reads a, b, d only, in kL0Stages32
// stages of the Newton passes' tile (their shared memory), and the first Newton pass checks l, u
constexpr int kL0Stages32 = 3;
constexpr int kRingBars = kL0Stages32 > kStages ? kL0Stages32 : kStages;  // mbarriers per block
constexpr unsigned kFlagWide = 2u;  // some FP64 value lies outside the df operating range
constexpr unsigned kFlagLuInf = 4u;  // some bound l_i or u_i is infinite
// absf: sum |b_i x_i| of the Newton passes on checked data, where it only scales the tolerance
// of stopping criterion 1: summed in float between flushes (relative error below 2^-19 with
// kFlushEvery tiles of 4 elements per thread).  The stand-alone phi evaluation, a pass that
// makes the full data checks and the final pass (the reported sum) keep the double-float sum.
struct EvalAcc {
    LazyDf phi, absbx, sfree;
    df mphi, mabsbx, msfree;  // middle level: normalised df sums of the flushed lazy sums
    float absf;
    int nmid;
    double phi64, absbx64, sfree64, satl, satu;
    long long nfree;
    bool bad, wide, luinf;
    __device__ void init() {
        phi = absbx = sfree = LazyDf{0.0f, 0.0f};
        mphi = mabsbx = msfree = df{0.0f, 0.0f};
        absf = 0.0f;
        nmid = 0;
        phi64 = absbx64 = sfree64 = satl = satu = 0.0;
        nfree = 0;
        bad = wide = luinf = false;
    }
    // all levels into FP64 (end of a pass).  The float parts are widened on the integer pipe
    // and added in FP64: float -> double conversion instructions run on the FP64 pipe, which
    // every warp of the SM shares at the end of a pass.
    __device__ void flush() {
        phi64 += df_to_f64_int(df_add(mphi, two_sum(phi.hi, phi.lo)));
        absbx64 += df_to_f64_int(df_add(mabsbx, two_sum(absbx.hi, __fadd_rn(absbx.lo, absf))));
        sfree64 += df_to_f64_int(df_add(msfree, two_sum(sfree.hi, sfree.lo)));
        phi = absbx = sfree = LazyDf{0.0f, 0.0f};
        mphi = mabsbx = msfree = df{0.0f, 0.0f};
        absf = 0.0f;
        nmid = 0;
    }
    // the lazy sums into the middle df sums (FP32 operations only; df_add is accurate to
    // ~2^-47 of the sum), and every fourth time everything into FP64: the FP64 pipe, the scarce
    // unit of this GPU, sees a quarter of the flushes
    __device__ void step_flush() {
        if (++nmid == 4) {
            flush();
            return;
        }
        mphi = df_add(mphi, two_sum(phi.hi, phi.lo));  // (|lo| may exceed |hi| after cancellation)
        mabsbx = df_add(mabsbx, two_sum(absbx.hi, __fadd_rn(absbx.lo, absf)));
        msfree = df_add(msfree, two_sum(sfree.hi, sfree.lo));
        phi = absbx = sfree = LazyDf{0.0f, 0.0f};
        absf = 0.0f;
    }
};

// status of one element: 0 free, 1 x = l, 2 x = u; ties = on a breakpoint
struct Cls {
    int c;
    bool tieL, tieU;
};

// ---- FP64 data, exact FP64 (values outside the df range) -------------------------------
// Out of line (rare); its sums come back by value so that the caller's accumulators stay in
// registers (an accumulator whose address reached an out-of-line call would live in memory).
struct ExactOut {
    double x, phi, absbx, sfree, satl, satu;
    int c;
};
__device__ __noinline__ ExactOut elem_f64_exact(double a, double b, double d, double l, double u, double lam,
                                                bool want_acc) {
    ExactOut o{0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0};
    const double lb = lam * b;
    const double v = a + lb;
    const double dl = isinf(l) ? l : d * l;
    const double du = isinf(u) ? u : d * u;
    const double sc = fabs(a) + fabs(lb);
    const bool tieL = !isinf(l) && fabs(v - dl) <= 2.2737367544323206e-13 * (sc + fabs(dl));
    const bool tieU = !isinf(u) && fabs(v - du) <= 2.2737367544323206e-13 * (sc + fabs(du));
    if (tieL || v < dl) { o.x = l; o.c = 1; }
    else if (tieU || v > du) { o.x = u; o.c = 2; }
    else { o.x = v / d; o.c = 0; }
    if (want_acc) {
        const double bx = b * o.x;
        o.phi = bx;
        o.absbx = fabs(bx);
        const double w = b * b / d;
        if (o.c == 0) o.sfree = w;
        if (tieL && !tieU) o.satl = w;
        if (tieU && !tieL) o.satu = w;
    }
    return o;
}

// ---- FP64 data in the df range ----------------------------------------------------------
// From v = a + lambda b (df): 1/d by the MUFU reciprocal and one df Newton correction,
// t = v/d, and the status of x_i(lambda) read off t against l, u (equivalent to v against
// d l, d u for d > 0).  TIES: elements within the tie band of the file header (scn = |a| +
// |lambda b| in float, scaled to x) count as lying on their breakpoint; without TIES the
// classification is the plain sign test (a pass whose lambda is not a breakpoint).
// Returns x; bx = b x, beta = b^2/d.
template <bool FIN, bool TIES>
__device__ __forceinline__ df elem_df_tail(df v, float scn, df B, df D, df Lo, df Up, Cls& cl, df& bx, df& beta) {
    const float r0 = rcp_approx(D.hi);
    const float res = fmaf(-D.lo, r0, fmaf(-D.hi, r0, 1.0f));
    const df invd = fast_two_sum(r0, __fmul_rn(r0, res));
    const df t = df_mul(v, invd);
    const bool linf = !FIN && isinf(Lo.hi), uinf = !FIN && isinf(Up.hi);  // FIN: finite bounds
    const float dL = __fadd_rn(__fsub_rn(t.hi, Lo.hi), __fsub_rn(t.lo, Lo.lo));
    const float dU = __fadd_rn(__fsub_rn(t.hi, Up.hi), __fsub_rn(t.lo, Up.lo));
    bool tieL = false, tieU = false;
    if constexpr (TIES) {
        const float sc = __fmul_rn(scn, r0);  // (|a| + |lambda b|)/d
        tieL = !linf && fabsf(dL) <= kTieRel * (sc + fabsf(Lo.hi));
        tieU = !uinf && fabsf(dU) <= kTieRel * (sc + fabsf(Up.hi));
    }
    const bool below = tieL || dL < 0.0f;
    const bool above = !below && (tieU || dU > 0.0f);
    cl.c = below ? 1 : (above ? 2 : 0);
    cl.tieL = tieL;
    cl.tieU = tieU;
    df x = t;
    if (below) x = Lo;
    if (above) x = Up;
    bx = df_mul_lazy(B, x);
    beta = df_mul_lazy(df_mul_lazy(B, B), invd);  // unnormalised chain: ~2^-46 relative
    return x;
}

// v = a + lambda b in df from the split a, b and lambda (TwoProd + TwoSum)
template <bool FIN, bool TIES>
__device__ __forceinline__ df elem_df(df A, df B, df D, df Lo, df Up, df Lm, Cls& cl, df& bx, df& beta) {
    const df p = two_prod(Lm.hi, B.hi);
    const float e = fmaf(Lm.hi, B.lo, fmaf(Lm.lo, B.hi, p.lo));
    const df s = two_sum(A.hi, p.hi);
    const df v = fast_two_sum(s.hi, __fadd_rn(__fadd_rn(s.lo, e), A.lo));
    return elem_df_tail<FIN, TIES>(v, __fadd_rn(fabsf(A.hi), fabsf(p.hi)), B, D, Lo, Up, cl, bx, beta);
}

// sanity checks of Sec. 5.1.1 on the bit patterns: d > 0, b > 0 finite; a finite; l <= u
// (as IEEE compares: +0 <= -0); no NaN (integer pipe only)
__device__ __forceinline__ bool bad_elem(double a, double b, double d, double l, double u) {
    const bool zeros = ((opaque_bits(l) | opaque_bits(u)) << 1) == 0ull;
    return !f64_pos_finite(d) || !f64_pos_finite(b) || !f64_is_finite(a) || f64_is_nan(l) || f64_is_nan(u) ||
           (order_key(l) > order_key(u) && !zeros);
}

// the same checks on float bit patterns
__device__ __forceinline__ bool bad_elem_f(float a, float b, float d, float l, float u) {
    const int ia = __float_as_int(a), ib = __float_as_int(b), id = __float_as_int(d);
    const int il = __float_as_int(l), iu = __float_as_int(u);
    auto pos_finite = [](int v) { return v > 0 && v < 0x7F800000; };
    auto is_nan = [](int v) { return (v & 0x7FFFFFFF) > 0x7F800000; };
    auto key = [](int v) { return v >= 0 ? v : (int)(0x80000000u - (unsigned)v) - 1; };
    return !pos_finite(id) || !pos_finite(ib) || (ia & 0x7F800000) == 0x7F800000 || is_nan(il) || is_nan(iu) ||
           (key(il) > key(iu) && ((il | iu) & 0x7FFFFFFF) != 0);
}

// the checks of bad_elem_f that concern l and u (NaN, l <= u), and those that concern a, b, d
__device__ __forceinline__ bool bad_bounds_f(float l, float u) {
    const int il = __float_as_int(l), iu = __float_as_int(u);
    auto is_nan = [](int v) { return (v & 0x7FFFFFFF) > 0x7F800000; };
    auto key = [](int v) { return v >= 0 ? v : (int)(0x80000000u - (unsigned)v) - 1; };
    return is_nan(il) || is_nan(iu) || (key(il) > key(iu) && ((il | iu) & 0x7FFFFFFF) != 0);
}
__device__ __forceinline__ bool bad_abd_f(float a, float b, float d) {
    const int ia = __float_as_int(a), ib = __float_as_int(b), id = __float_as_int(d);
    auto pos_finite = [](int v) { return v > 0 && v < 0x7F800000; };
    return !pos_finite(id) || !pos_finite(ib) || (ia & 0x7F800000) == 0x7F800000;
}

// ---- FP32 data -----------------------------------------------------------------------------
// v = a + lambda b with lambda a float pair (TwoProd + TwoSum), rounded once; t = v/d by the
// MUFU reciprocal and one correction (~1 ulp); the status is read off t against l, u with a
// tie band of 2^-20 relative (the float rounding of t); b x by TwoProd; b^2/d in float.
constexpr float kTieRel32 = 9.5367431640625e-07f;  // 2^-20
template <bool FIN, bool TIES>
__device__ __forceinline__ float elem_f32(float a, float b, float d, float l, float u, df Lm, Cls& cl, df& bx,
                                          float& beta) {
    const df p = two_prod(Lm.hi, b);
    const float e = fmaf(Lm.lo, b, p.lo);
    const df s = two_sum(a, p.hi);
    const float vh = __fadd_rn(s.hi, __fadd_rn(s.lo, e));
    const float r0 = rcp_approx(d);
    float t = __fmul_rn(vh, r0);
    t = fmaf(fmaf(-t, d, vh), r0, t);
    const bool linf = !FIN && isinf(l), uinf = !FIN && isinf(u);
    const float dL = __fsub_rn(t, l), dU = __fsub_rn(t, u);
    bool tieL = false, tieU = false;
    if constexpr (TIES) {
        const float sc = __fmul_rn(__fadd_rn(fabsf(a), fabsf(p.hi)), r0);
        tieL = !linf && fabsf(dL) <= kTieRel32 * (sc + fabsf(l));
        tieU = !uinf && fabsf(dU) <= kTieRel32 * (sc + fabsf(u));
    }
    const bool below = tieL || dL < 0.0f;
    const bool above = !below && (tieU || dU > 0.0f);
    cl.c = below ? 1 : (above ? 2 : 0);
    cl.tieL = tieL;
    cl.tieU = tieU;
    float x = t;
    if (below) x = l;
    if (above) x = u;
    bx = two_prod(b, x);
    const float bb = __fmul_rn(b, b);
    beta = __fmul_rn(bb, r0);
    beta = fmaf(fmaf(-beta, d, bb), r0, beta);
    return x;
}

// l < x strictly, as doubles, on order keys (-0 taken as +0; a NaN x is never inside)
__device__ __forceinline__ long long cmp_key(double v) {
    const unsigned long long b = opaque_bits(v);
    return (b << 1) == 0ull ? 0ll : order_key(v);
}
template <typename T>
__device__ __forceinline__ bool strictly_inside(T l, T x, T u) {
    if constexpr (sizeof(T) == 8) {
        const long long kx = cmp_key(x);
        return cmp_key(l) < kx && kx < cmp_key(u) && !f64_is_nan(x);
    } else {
        return l < x && x < u;
    }
}

// x clamped to [l, u] exactly (l <= u, no NaN: checked data); order keys for doubles
template <typename T>
__device__ __forceinline__ T clamp_exact(T l, T x, T u) {
    if constexpr (sizeof(T) == 8) {
        const long long kx = cmp_key(x);
        return kx < cmp_key(l) ? l : (kx > cmp_key(u) ? u : x);
    } else {
        return x < l ? l : (x > u ? u : x);
    }
}

// ---- the map of one 16-byte vector of elements (V of them): accumulate (write_x = false)
// or write x / mask and the sums of the stored x.  q = global vector index, qw = index of the
// warp's first vector (a multiple of 32).
// CK, the checks made per element: kCheckAll (every value: the sanity checks of Sec. 5.1.1 when
// check, infinite bounds, the df operating range of FP64 values), kCheckBounds (a, b, d are
// known valid and in range, checked by the lambda_0 pass: l and u only), kChecked (every value
// known valid and in range: no check).
// TIES: the tie band of the file header is tested (passes whose lambda may sit on a breakpoint:
// the first, the final pass and those after a breakpoint step); otherwise the plain sign test.
template <typename T, int CK, bool FIN, bool TIES, bool WX>
__device__ __forceinline__ void eval_vec(const GeneralArgs& A, const T (&va)[VecOf<T>::V], const T (&vb)[VecOf<T>::V],
                                         const T (&vd)[VecOf<T>::V], const T (&vl)[VecOf<T>::V],
                                         const T (&vu)[VecOf<T>::V], const bool (&ok)[VecOf<T>::V], int64_t q,
                                         int64_t qw, double lam, df Lm, bool lam_ok, bool check, EvalAcc& acc,
                                         const Span& sp) {
    constexpr int V = VecOf<T>::V;
    constexpr bool write_x = WX;
    constexpr bool FAST = CK == kChecked;
    const bool aligned = A.aligned != 0;
    T* __restrict__ px = static_cast<T*>(A.x);
        T xo[V];
        bool fr[V];
        df beta[V];
        df xdf[V];
        unsigned tiem = 0, widem = 0, freem = 0;
#pragma unroll
        for (int j = 0; j < V; j++) {
            fr[j] = false;
            xo[j] = T(0);
            beta[j] = df_make(0.0f);
            if (!ok[j]) continue;
            const T a = va[j], b = vb[j], d = vd[j], l = vl[j], u = vu[j];
            Cls cl;
            df bx;
            if constexpr (sizeof(T) == 8) {
                df Ad, Bd, Dd, Ld, Ud, xv;
                if constexpr (FAST) {
                    Ad = split_f64_finite(a);
                    Bd = split_f64_pos(b);  // b, d > 0 inside the range (checked in the first pass)
                    Dd = split_f64_pos(d);
                    Ld = FIN ? split_f64_finite(l) : split_f64(l);  // FIN: no infinite bound (first pass)
                    Ud = FIN ? split_f64_finite(u) : split_f64(u);
                    xv = elem_df<FIN, TIES>(Ad, Bd, Dd, Ld, Ud, Lm, cl, bx, beta[j]);
                } else {
                    // operating range by exponent-field tests: b, d positive in [2^-60, 2^60];
                    // a 0 or in range; l, u 0, +-inf or in range.  In-range values are finite and
                    // not NaN, so of the sanity checks only l <= u remains for them; elements
                    // outside the range take the exact path, which checks everything.
                    const unsigned hb = hi_word(b), hd = hi_word(d);
                    const unsigned ha = hi_word(a), la = lo_word(a);
                    const unsigned hl = hi_word(l), ll = lo_word(l);
                    const unsigned hu = hi_word(u), lu = lo_word(u);
                    auto rng = [](unsigned h) { return (((h >> 20) & 0x7FFu) - 963u) <= 120u; };
                    auto zero = [](unsigned h, unsigned lo) { return ((h & 0x7FFFFFFFu) | lo) == 0u; };
                    auto inf = [](unsigned h, unsigned lo) { return (h & 0x7FFFFFFFu) == 0x7FF00000u && lo == 0u; };
                    const bool abd = CK == kCheckBounds || (((hb >> 20) - 963u) <= 120u &&
                                                            ((hd >> 20) - 963u) <= 120u && (rng(ha) || zero(ha, la)));
                    const bool inr = lam_ok && abd && (rng(hl) || zero(hl, ll) || inf(hl, ll)) &&
                                     (rng(hu) || zero(hu, lu) || inf(hu, lu));
                    acc.luinf |= inf(hl, ll) || inf(hu, lu);
                    if (!inr) {
                        widem |= 1u << j;
                        acc.wide = true;
                        continue;
                    }
                    Ad = split_f64_finite(a);
                    Bd = CK == kCheckBounds ? split_f64_pos(b) : split_f64_finite(b);
                    Dd = CK == kCheckBounds ? split_f64_pos(d) : split_f64_finite(d);
                    Ld = split_f64(l);
                    Ud = split_f64(u);
                    if (check) acc.bad |= df_lt(Ud, Ld);
                    xv = elem_df<FIN, TIES>(Ad, Bd, Dd, Ld, Ud, Lm, cl, bx, beta[j]);
                }
                if (write_x) {
                    xo[j] = cl.c == 1 ? l : (cl.c == 2 ? u : 0.0);
                    freem |= (cl.c == 0 ? 1u : 0u) << j;
                    xdf[j] = xv;
                    // residual sums from b x of the df solution (within 2^-46 of the stored x)
                    lazy_add(acc.phi, bx);
                    lazy_add(acc.absbx, bx.hi < 0.0f ? df_neg(bx) : bx);
                }
            } else {
                if (CK == kCheckAll && check) acc.bad |= bad_elem_f(a, b, d, l, u);
                if (CK == kCheckBounds && check) acc.bad |= bad_bounds_f(l, u);
                if (!FAST) acc.luinf |= isinf(l) || isinf(u);
                float bt;
                xo[j] = elem_f32<FIN, TIES>(a, b, d, l, u, Lm, cl, bx, bt);
                beta[j] = df_make(bt);
            }
            fr[j] = cl.c == 0;
            if (!write_x) {
                lazy_add(acc.phi, bx);
                if constexpr (CK != kCheckAll) acc.absf += fabsf(bx.hi);  // (a tolerance scale: see EvalAcc)
                else lazy_add(acc.absbx, bx.hi < 0.0f ? df_neg(bx) : bx);
                lazy_add(acc.sfree, fr[j] ? beta[j] : df_make(0.0f));
            }
            if constexpr (TIES) {
                tiem |= ((cl.tieL && !cl.tieU) ? 1u : 0u) << (2 * j);
                tiem |= ((cl.tieU && !cl.tieL) ? 2u : 0u) << (2 * j);
            }
        }
        // rare cases, one loop trip per element concerned (a data-dependent loop keeps FP64
        // instructions off the common path): elements on a breakpoint (lateral-slope ties)
        // and FP64 values outside the df operating range (exact FP64)
        if (TIES && !write_x) {
            for (unsigned m = tiem; m; m &= m - 1) {
                const int bit = __ffs(m) - 1;
                const double bj = df_to_f64_int_all(pick(beta, bit >> 1));
                if (bit & 1) acc.satu += bj;
                else acc.satl += bj;
            }
        }
        if constexpr (sizeof(T) == 8 && !FAST) {
            for (unsigned m = widem; m; m &= m - 1) {
                const int j = __ffs(m) - 1;
                const T bj = pick(vb, j);
                if (check) acc.bad |= bad_elem(pick(va, j), bj, pick(vd, j), pick(vl, j), pick(vu, j));
                const ExactOut eo = elem_f64_exact(pick(va, j), bj, pick(vd, j), pick(vl, j), pick(vu, j), lam, !write_x);
                const T xj = eo.x;
                if (!write_x) {
                    acc.phi64 += eo.phi;
                    acc.absbx64 += eo.absbx;
                    acc.sfree64 += eo.sfree;
                    acc.satl += eo.satl;
                    acc.satu += eo.satu;
                }
                put(xo, j, xj);
                put(fr, j, eo.c == 0);
                if (write_x) {
                    acc.phi64 += bj * xj;
                    acc.absbx64 += fabs(bj * xj);
                }
            }
        }
        if (write_x) {
            // free x of FP64 data: df -> double, one FP64 add per free element (measured faster here
            // than the integer-pipe conversion)
            if constexpr (sizeof(T) == 8) {
#pragma unroll
                for (int j = 0; j < V; j++)
                    if ((freem >> j) & 1u) xo[j] = df_to_f64_int(xdf[j]);
            }
            // without the tie band a rounded t may land on a bound (or a hair past it): the stored x
            // of a free element is kept inside [l, u] exactly and its mask bit is read off it
            if constexpr (!TIES) {
#pragma unroll
                for (int j = 0; j < V; j++)
                    if (ok[j] && fr[j]) {
                        xo[j] = clamp_exact<T>(vl[j], xo[j], vu[j]);
                        fr[j] = strictly_inside<T>(vl[j], xo[j], vu[j]);
                    }
            }
            if constexpr (sizeof(T) != 8) {
                // FP32 data: sums of the stored (float) x, b x exact by TwoProd
#pragma unroll
                for (int j = 0; j < V; j++) {
                    if (!ok[j]) continue;
                    const df pr = two_prod((float)vb[j], (float)xo[j]);
                    lazy_add(acc.phi, pr);
                    lazy_add(acc.absbx, pr.hi < 0.0f ? df_neg(pr) : pr);
                }
            }
#pragma unroll
            for (int j = 0; j < V; j++) acc.nfree += (ok[j] && fr[j]) ? 1 : 0;
            if (px) store_vec<T>(px, sp, q, aligned, xo);
            if (A.mask) store_mask<V>(A.mask, sp, qw, fr);
        }
}

// ---- one pass over all elements with plain loads (arrays not 16-byte aligned)
template <typename T, int CK, bool FIN, bool TIES, bool WX>
__device__ __forceinline__ void eval_pass_plain(const GeneralArgs& A, const Grp& gp, double lam, bool check, bool rev,
                                                EvalAcc& acc) {
    constexpr int V = VecOf<T>::V;
    constexpr int U = kGenU;
    const T* __restrict__ pa = static_cast<const T*>(A.a);
    const T* __restrict__ pb = static_cast<const T*>(A.b);
    const T* __restrict__ pd = static_cast<const T*>(A.d);
    const T* __restrict__ pl = static_cast<const T*>(A.l);
    const T* __restrict__ pu = static_cast<const T*>(A.u);
    const Span sp = gp.sp;
    const int lane = threadIdx.x & 31;
    const bool aligned = A.aligned != 0;
    const df Lm = df_from_f64(lam);
    const bool lam_ok = fabs(lam) <= 1.152921504606847e18;  // 2^60
    const WarpSweep sw(span_qlo<V>(sp), span_qhi<V>(sp), U, gp.member, gp.g);
    int steps = 0;
    for (int64_t it = 0; it < sw.count; it++) {
        if (++steps == kFlushEvery) {
            acc.step_flush();
            steps = 0;
        }
        const int64_t base = sw.base(it, rev);
        T va[U][V], vb[U][V], vd[U][V], vl[U][V], vu[U][V];
        bool ok[U][V];
#pragma unroll
        for (int w = 0; w < U; w++) {
            const int64_t q = base + w * 32 + lane;
            load_vec<T>(pa, sp, q, aligned, va[w], ok[w]);
            load_vec<T>(pb, sp, q, aligned, vb[w], ok[w]);
            load_vec<T>(pd, sp, q, aligned, vd[w], ok[w]);
            load_vec<T>(pl, sp, q, aligned, vl[w], ok[w]);
            load_vec<T>(pu, sp, q, aligned, vu[w], ok[w]);
        }
#pragma unroll
        for (int w = 0; w < U; w++)
            eval_vec<T, CK, FIN, TIES, WX>(A, va[w], vb[w], vd[w], vl[w], vu[w], ok[w], base + w * 32 + lane,
                                             base + w * 32, lam, Lm, lam_ok, check, acc, sp);
    }
}

// ---- one pass with the arrays staged through shared memory by bulk copies (TileRing)
template <typename T>
__host__ __device__ constexpr int stage_tile() { return kGenTileBytes / (int)sizeof(T); }  // elements per array per stage

template <typename T, int CK, bool FIN, bool TIES, bool WX>
__device__ __forceinline__ bool eval_pass_staged(const GeneralArgs& A, const Grp& gp, double lam, bool check,
                                                 bool rev, EvalAcc& acc, T* smem, uint64_t* bars, unsigned& parity,
                                                 int* err) {
    constexpr int V = VecOf<T>::V;
    constexpr int TT = stage_tile<T>();
    constexpr int VPT = TT / V / NT;  // vectors per thread per tile
    using VT = typename VecOf<T>::type;
    const T* src[5] = {static_cast<const T*>(A.a), static_cast<const T*>(A.b), static_cast<const T*>(A.d),
                       static_cast<const T*>(A.l), static_cast<const T*>(A.u)};
    TileRing<T, 5, TT> ring;
    const Span sp = gp.sp;
    ring.setup(sp.lo, sp.hi, smem, bars, gp.member, gp.g);
    ring.parity = parity;
    const df Lm = df_from_f64(lam);
    const bool lam_ok = fabs(lam) <= 1.152921504606847e18;  // 2^60
    for (int s = 0; s < kStages - 1; s++)
        if (s < ring.count) ring.issue_by_warps(ring.tile(s, rev), s, src);
    bool okw = true;
    for (int64_t i = 0; i < ring.count; i++) {
        const int st = (int)(i % kStages);
        if (i + kStages - 1 < ring.count)
            ring.issue_by_warps(ring.tile(i + kStages - 1, rev), (int)((i + kStages - 1) % kStages), src);
        if (!mbar_wait(&ring.bar[st], (ring.parity >> st) & 1u, err, A.limit_ns, CQK_TIMEOUT)) okw = false;
        ring.parity ^= 1u << st;
        const int64_t c = ring.tile(i, rev);
        const int64_t sb0 = ring.b0(c), sb1 = ring.b1(c);
        if ((i & 7) == 7) acc.step_flush();
#pragma unroll
        for (int k = 0; k < VPT; k++) {
            const int ql = (int)threadIdx.x + k * NT;  // vector within the tile
            const int64_t q = c * (TT / V) + ql;
            const int64_t qw = q - (threadIdx.x & 31);
            T va[V], vb[V], vd[V], vl[V], vu[V];
            bool ok[V];
            if (q * V >= sb0 && (q + 1) * V <= sb1) {
                const VT wa = reinterpret_cast<const VT*>(ring.stage(st, 0))[ql];
                const VT wb = reinterpret_cast<const VT*>(ring.stage(st, 1))[ql];
                const VT wd = reinterpret_cast<const VT*>(ring.stage(st, 2))[ql];
                const VT wl = reinterpret_cast<const VT*>(ring.stage(st, 3))[ql];
                const VT wu = reinterpret_cast<const VT*>(ring.stage(st, 4))[ql];
#pragma unroll
                for (int j = 0; j < V; j++) {
                    va[j] = reinterpret_cast<const T*>(&wa)[j];
                    vb[j] = reinterpret_cast<const T*>(&wb)[j];
                    vd[j] = reinterpret_cast<const T*>(&wd)[j];
                    vl[j] = reinterpret_cast<const T*>(&wl)[j];
                    vu[j] = reinterpret_cast<const T*>(&wu)[j];
                    ok[j] = true;
                }
            } else {  // tail of the array beyond the last full 16 bytes
                load_vec<T>(src[0], sp, q, false, va, ok);
                load_vec<T>(src[1], sp, q, false, vb, ok);
                load_vec<T>(src[2], sp, q, false, vd, ok);
                load_vec<T>(src[3], sp, q, false, vl, ok);
                load_vec<T>(src[4], sp, q, false, vu, ok);
            }
            eval_vec<T, CK, FIN, TIES, WX>(A, va, vb, vd, vl, vu, ok, q, qw, lam, Lm, lam_ok, check, acc, sp);
        }
        __syncthreads();  // the stage is refilled only after every thread has read it
    }
    parity = ring.parity;
    return okw;
}

// one pass over all elements, staged or plain; WX: the final pass (write x, the mask and the
// sums of the stored x) instead of the accumulation of phi and its slopes
template <typename T, bool WX, int CK, bool FIN = false, bool TIES = true>
__device__ __forceinline__ bool eval_pass(const GeneralArgs& A, const Grp& gp, double lam, bool check, bool rev,
                                          EvalAcc& acc, T* smem, uint64_t* bars, unsigned& parity, int* err) {
    if (A.staged) return eval_pass_staged<T, CK, FIN, TIES, WX>(A, gp, lam, check, rev, acc, smem, bars, parity, err);
    eval_pass_plain<T, CK, FIN, TIES, WX>(A, gp, lam, check, rev, acc);
    return true;
}

// closest breakpoint strictly right (dir > 0) / left (dir < 0) of lam, FP64 as defined
template <typename T>
__device__ __forceinline__ double breakpoint_pass(const GeneralArgs& A, const Grp& gp, double lam, int dir) {
    const T* pa = static_cast<const T*>(A.a);
    const T* pb = static_cast<const T*>(A.b);
    const T* pd = static_cast<const T*>(A.d);
    const T* pl = static_cast<const T*>(A.l);
    const T* pu = static_cast<const T*>(A.u);
    double best = dir > 0 ? INFINITY : -INFINITY;
    const int64_t stride = (int64_t)gp.g * NT;
    for (int64_t i = gp.sp.lo + (int64_t)gp.member * NT + threadIdx.x; i < gp.sp.hi; i += stride) {
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

// What a pass learnt about the data: a sanity check of Sec. 5.1.1 failed, an FP64 value lies
// outside the df operating range, a bound is infinite.
struct DataFlags {
    bool bad, wide, luinf;
};

// eq. (CQKlambda0) terms of V elements: s += b a/d, q += b^2/d (df, FP64 outside the range),
// and the checks of the data that the Newton passes rely on (the lambda_0 pass reads l and u
// for them): the sanity checks of Sec. 5.1.1 (when check), infinite bounds and FP64 values
// outside the df operating range
template <typename T>
__device__ __forceinline__ void lambda0_vec(const T (&va)[VecOf<T>::V], const T (&vb)[VecOf<T>::V],
                                            const T (&vd)[VecOf<T>::V], const T (&vl)[VecOf<T>::V],
                                            const T (&vu)[VecOf<T>::V], const bool (&ok)[VecOf<T>::V], LazyDf& s,
                                            LazyDf& q, double& s64, double& q64, bool check, DataFlags& fl) {
    constexpr int V = VecOf<T>::V;
    unsigned exact = 0, wide = 0;
#pragma unroll
    for (int j = 0; j < V; j++) {
        if (!ok[j]) continue;
        const T a = va[j], b = vb[j], d = vd[j], l = vl[j], u = vu[j];
        if constexpr (sizeof(T) == 8) {
            // operating range by exponent-field tests: b, d positive in [2^-60, 2^60]; a 0 or in
            // that range; l, u 0, +-inf or in that range.  Values in range are not NaN, so of the
            // sanity checks only l <= u remains for them; the others take the exact checks below.
            const unsigned ha = hi_word(a), la = lo_word(a);
            const unsigned hl = hi_word(l), ll = lo_word(l), hu = hi_word(u), lu = lo_word(u);
            auto rng = [](unsigned h) { return (((h >> 20) & 0x7FFu) - 963u) <= 120u; };
            auto zero = [](unsigned h, unsigned lo) { return ((h & 0x7FFFFFFFu) | lo) == 0u; };
            auto inf = [](unsigned h, unsigned lo) { return (h & 0x7FFFFFFFu) == 0x7FF00000u && lo == 0u; };
            // (b, d: the pattern itself in [2^-60, 2^61) as an unsigned range, a set sign bit fails)
            const bool inr = hi_word(b) - 0x3C300000u < 0x07900000u && hi_word(d) - 0x3C300000u < 0x07900000u &&
                             (rng(ha) || zero(ha, la));
            const bool linf = inf(hl, ll), uinf = inf(hu, lu);
            const bool lur = (rng(hl) || zero(hl, ll) || linf) && (rng(hu) || zero(hu, lu) || uinf);
            fl.luinf |= linf || uinf;
            if (check && inr && lur) {
                // l > u on order keys of the high words (signed magnitude -> two's complement),
                // the low words deciding between equal high words; +0 and -0 compare equal
                const int kl = (int)(hl ^ ((unsigned)((int)hl >> 31) >> 1));
                const int ku = (int)(hu ^ ((unsigned)((int)hu >> 31) >> 1));
                const bool lo_gt = (int)hl < 0 ? ll < lu : ll > lu;
                fl.bad |= (kl > ku || (kl == ku && lo_gt)) && !(zero(hl, ll) && zero(hu, lu));
            }
            const df B = split_f64_pos(b), D = split_f64_pos(d);  // (discarded unless in range)
            const float r0 = rcp_approx(D.hi);
            const float res = fmaf(-D.lo, r0, fmaf(-D.hi, r0, 1.0f));
            const df invd = fast_two_sum(r0, __fmul_rn(r0, res));
            const df wgt = df_mul(B, invd);
            const df ps = df_mul_lazy(wgt, split_f64_finite(a)), pq = df_mul_lazy(wgt, B);
            lazy_add(s, df{inr ? ps.hi : 0.0f, inr ? ps.lo : 0.0f});
            lazy_add(q, df{inr ? pq.hi : 0.0f, inr ? pq.lo : 0.0f});
            exact |= (inr ? 0u : 1u) << j;
            wide |= (inr && lur ? 0u : 1u) << j;
        } else {
            // (FP32: l and u are checked by the first Newton pass)
            if (check) fl.bad |= bad_abd_f(a, b, d);
            const float rd = rcp_approx(d);
            float wgt = __fmul_rn(b, rd);
            wgt = fmaf(fmaf(-wgt, d, b), rd, wgt);
            lazy_add(s, two_prod(wgt, a));
            lazy_add(q, two_prod(wgt, b));
        }
    }
    for (unsigned m = exact; m; m &= m - 1) {  // exact FP64 outside the df range (rare)
        const int j = __ffs(m) - 1;
        const double a = pick(va, j), b = pick(vb, j), d = pick(vd, j);
        s64 += b * a / d;
        q64 += b * b / d;
    }
    if constexpr (sizeof(T) == 8) {
        fl.wide |= wide != 0u;
        if (check)
            for (unsigned m = wide; m; m &= m - 1) {
                const int j = __ffs(m) - 1;
                fl.bad |= bad_elem(pick(va, j), pick(vb, j), pick(vd, j), pick(vl, j), pick(vu, j));
            }
    }
}

template <typename T>
__device__ __forceinline__ bool lambda0_pass(const GeneralArgs& A, const Grp& gp, double& s_out, double& q_out,
                                             bool check, DataFlags& fl, T* smem, uint64_t* bars, unsigned& parity,
                                             int* err) {
    constexpr int V = VecOf<T>::V;
    const T* __restrict__ pa = static_cast<const T*>(A.a);
    const T* __restrict__ pb = static_cast<const T*>(A.b);
    const T* __restrict__ pd = static_cast<const T*>(A.d);
    const T* __restrict__ pl = static_cast<const T*>(A.l);
    const T* __restrict__ pu = static_cast<const T*>(A.u);
    constexpr bool LU0 = sizeof(T) == 8;  // l and u are read here (FP64 data)
    const Span sp = gp.sp;
    LazyDf s{0.0f, 0.0f}, q{0.0f, 0.0f};
    double s64 = 0.0, q64 = 0.0;
    bool okw = true;
    if (A.staged) {
        constexpr int TT = stage_tile<T>();
        constexpr int VPT = TT / V / NT;
        constexpr int NA = LU0 ? 5 : 3;                   // arrays read
        constexpr int NS = LU0 ? kStages : kL0Stages32;  // stages (the same shared memory)
        static_assert(NA * NS <= 5 * kStages, "the lambda_0 stages fit the Newton passes' shared memory");
        using VT = typename VecOf<T>::type;
        const T* src[5] = {pa, pb, pd, pl, pu};
        TileRing<T, NA, TT> ring;
        ring.setup(sp.lo, sp.hi, smem, bars, gp.member, gp.g);
        ring.parity = parity;
        for (int st = 0; st < NS - 1; st++)
            if (st < ring.count) ring.issue_by_warps(ring.tile(st, false), st, src);
        for (int64_t i = 0; i < ring.count; i++) {
            const int st = (int)(i % NS);
            if (i + NS - 1 < ring.count)
                ring.issue_by_warps(ring.tile(i + NS - 1, false), (int)((i + NS - 1) % NS), src);
            if (!mbar_wait(&ring.bar[st], (ring.parity >> st) & 1u, err, A.limit_ns, CQK_TIMEOUT)) okw = false;
            ring.parity ^= 1u << st;
            const int64_t c = ring.tile(i, false);
            const int64_t sb0 = ring.b0(c), sb1 = ring.b1(c);
            if ((i & 7) == 7) {
                s64 += lazy_value_int(s);
                q64 += lazy_value_int(q);
                s = q = LazyDf{0.0f, 0.0f};
            }
#pragma unroll
            for (int k = 0; k < VPT; k++) {
                const int ql = (int)threadIdx.x + k * NT;
                const int64_t qg = c * (TT / V) + ql;
                T va[V], vb[V], vd[V], vl[V], vu[V];
                bool ok[V];
                if (qg * V >= sb0 && (qg + 1) * V <= sb1) {
                    const VT wa = reinterpret_cast<const VT*>(ring.stage(st, 0))[ql];
                    const VT wb = reinterpret_cast<const VT*>(ring.stage(st, 1))[ql];
                    const VT wd = reinterpret_cast<const VT*>(ring.stage(st, 2))[ql];
                    VT wl, wu;
                    if constexpr (LU0) {
                        wl = reinterpret_cast<const VT*>(ring.stage(st, LU0 ? 3 : 0))[ql];
                        wu = reinterpret_cast<const VT*>(ring.stage(st, LU0 ? 4 : 0))[ql];
                    }
#pragma unroll
                    for (int j = 0; j < V; j++) {
                        va[j] = reinterpret_cast<const T*>(&wa)[j];
                        vb[j] = reinterpret_cast<const T*>(&wb)[j];
                        vd[j] = reinterpret_cast<const T*>(&wd)[j];
                        vl[j] = LU0 ? reinterpret_cast<const T*>(&wl)[j] : T(0);
                        vu[j] = LU0 ? reinterpret_cast<const T*>(&wu)[j] : T(0);
                        ok[j] = true;
                    }
                } else {
                    load_vec<T>(pa, sp, qg, false, va, ok);
                    load_vec<T>(pb, sp, qg, false, vb, ok);
                    load_vec<T>(pd, sp, qg, false, vd, ok);
                    if constexpr (LU0) {
                        load_vec<T>(pl, sp, qg, false, vl, ok);
                        load_vec<T>(pu, sp, qg, false, vu, ok);
                    } else {
#pragma unroll
                        for (int j = 0; j < V; j++) vl[j] = vu[j] = T(0);
                    }
                }
                lambda0_vec<T>(va, vb, vd, vl, vu, ok, s, q, s64, q64, check, fl);
            }
            __syncthreads();
        }
        parity = ring.parity;
    } else {
        const int lane = threadIdx.x & 31;
        constexpr int U = kGenU;
        const WarpSweep sw(span_qlo<V>(sp), span_qhi<V>(sp), U, gp.member, gp.g);
        int steps = 0;
        for (int64_t it = 0; it < sw.count; it++) {
            if (++steps == kFlushEvery) {
                s64 += lazy_value_int(s);
                q64 += lazy_value_int(q);
                s = q = LazyDf{0.0f, 0.0f};
                steps = 0;
            }
            const int64_t base = sw.base(it, false);
            T va[U][V], vb[U][V], vd[U][V], vl[U][V], vu[U][V];
            bool ok[U][V];
#pragma unroll
            for (int w = 0; w < U; w++) {
                load_vec<T>(pa, sp, base + w * 32 + lane, A.aligned != 0, va[w], ok[w]);
                load_vec<T>(pb, sp, base + w * 32 + lane, A.aligned != 0, vb[w], ok[w]);
                load_vec<T>(pd, sp, base + w * 32 + lane, A.aligned != 0, vd[w], ok[w]);
                if constexpr (LU0) {
                    load_vec<T>(pl, sp, base + w * 32 + lane, A.aligned != 0, vl[w], ok[w]);
                    load_vec<T>(pu, sp, base + w * 32 + lane, A.aligned != 0, vu[w], ok[w]);
                } else {
#pragma unroll
                    for (int j = 0; j < V; j++) vl[w][j] = vu[w][j] = T(0);
                }
            }
#pragma unroll
            for (int w = 0; w < U; w++)
                lambda0_vec<T>(va[w], vb[w], vd[w], vl[w], vu[w], ok[w], s, q, s64, q64, check, fl);
        }
    }
    s_out = lazy_value_int(s) + s64;
    q_out = lazy_value_int(q) + q64;
    return okw;
}

// Warm start (Sec. 2): the sums of eq. (CQKlambda0) over J = {l < xbar < u} and over all
// variables, and |J|, in one pass with plain loads.  out = {s_J, q_J, |J|, s_all, q_all}.
template <typename T>
__device__ __forceinline__ void lambda0_warm_pass(const GeneralArgs& A, const Grp& gp, double (&out)[5]) {
    constexpr int V = VecOf<T>::V;
    constexpr int U = kGenU;
    const T* __restrict__ pa = static_cast<const T*>(A.a);
    const T* __restrict__ pb = static_cast<const T*>(A.b);
    const T* __restrict__ pd = static_cast<const T*>(A.d);
    const T* __restrict__ pl = static_cast<const T*>(A.l);
    const T* __restrict__ pu = static_cast<const T*>(A.u);
    const T* __restrict__ px = static_cast<const T*>(A.xbar);
    const Span sp = gp.sp;
    const int lane = threadIdx.x & 31;
    const bool aligned = A.aligned != 0;
    LazyDf sJ{0.0f, 0.0f}, qJ{0.0f, 0.0f}, sA{0.0f, 0.0f}, qA{0.0f, 0.0f};
    double sJ64 = 0.0, qJ64 = 0.0, sA64 = 0.0, qA64 = 0.0;
    long long m = 0;
    const WarpSweep sw(span_qlo<V>(sp), span_qhi<V>(sp), U, gp.member, gp.g);
    int steps = 0;
    for (int64_t it = 0; it < sw.count; it++) {
        if (++steps == kFlushEvery) {
            sJ64 += lazy_value_int(sJ);
            qJ64 += lazy_value_int(qJ);
            sA64 += lazy_value_int(sA);
            qA64 += lazy_value_int(qA);
            sJ = qJ = sA = qA = LazyDf{0.0f, 0.0f};
            steps = 0;
        }
        const int64_t base = sw.base(it, false);
        T va[U][V], vb[U][V], vd[U][V], vl[U][V], vu[U][V], vx[U][V];
        bool ok[U][V];
#pragma unroll
        for (int w = 0; w < U; w++) {
            const int64_t q = base + w * 32 + lane;
            load_vec<T>(pa, sp, q, aligned, va[w], ok[w]);
            load_vec<T>(pb, sp, q, aligned, vb[w], ok[w]);
            load_vec<T>(pd, sp, q, aligned, vd[w], ok[w]);
            load_vec<T>(pl, sp, q, aligned, vl[w], ok[w]);
            load_vec<T>(pu, sp, q, aligned, vu[w], ok[w]);
            load_vec<T>(px, sp, q, aligned, vx[w], ok[w]);
        }
#pragma unroll
        for (int w = 0; w < U; w++) {
            bool inJ[V];
#pragma unroll
            for (int j = 0; j < V; j++) {
                inJ[j] = ok[w][j] && strictly_inside<T>(vl[w][j], vx[w][j], vu[w][j]);
                m += inJ[j] ? 1 : 0;
            }
            DataFlags unused{false, false, false};  // (the first Newton pass checks the data)
            lambda0_vec<T>(va[w], vb[w], vd[w], vl[w], vu[w], inJ, sJ, qJ, sJ64, qJ64, false, unused);
            lambda0_vec<T>(va[w], vb[w], vd[w], vl[w], vu[w], ok[w], sA, qA, sA64, qA64, false, unused);
        }
    }
    out[0] = lazy_value_int(sJ) + sJ64;
    out[1] = lazy_value_int(qJ) + qJ64;
    out[2] = (double)m;
    out[3] = lazy_value_int(sA) + sA64;
    out[4] = lazy_value_int(qA) + qA64;
}

#define CQK_BARRIER_OR_LEAVE()                                                  \
    do {                                                                        \
        if (!group_barrier(gp, bar_target, A.limit_ns, A.fault_inject == 1)) {     \
            if (threadIdx.x == 0) info->status = CQK_TIMEOUT;                   \
            return;                                                             \
        }                                                                       \
        bar_target += (unsigned)G;                                              \
    } while (0)

// ---- one solve (or one phi evaluation) by one group of blocks ------------------------------
// smem / ring_bars: the block's bulk-copy stages and their mbarriers (initialised by the
// caller when A.staged); ring_parity: their phase bits, carried across calls.
// r and info are the instance's (a batch passes its kernel argument A unchanged, so that A is
// read from the parameter space instead of a per-instance copy in local memory).
template <typename T>
__device__ __forceinline__ void general_solve(const GeneralArgs& A, const Grp& gp, const double r, cqk_info* info,
                                              T* smem, uint64_t* ring_bars, unsigned& ring_parity) {
    __shared__ double sh[kPartialQ][NWARP];
    __shared__ double bscr[5 * NT];  // per-thread sums of a pass (block_sum_smem)
    __shared__ double bc[kPartialQ];
    const int G = gp.g;
    unsigned bar_target = (unsigned)G + (A.fault_inject == 1 ? 1u : 0u);
    int* err = &gp.hdr->error;
    int passes = 0, par = 0;

    if (A.phi_only) {  // cqk_phi: one evaluation at A.lambda0 (and x when requested)
        EvalAcc acc;
        acc.init();
        eval_pass<T, false, kCheckAll>(A, gp, A.lambda0, false, false, acc, smem, ring_bars, ring_parity, err);
        acc.flush();
        double pv[3] = {acc.phi64, acc.sfree64, acc.absbx64};
        double pt[2] = {acc.satl, acc.satu};
        block_sum_smem<3>(pv, bscr);
        block_sum_smem<2>(pt, bscr);
        if (threadIdx.x == 0) {
            const double w5[5] = {pv[0], pv[1], pv[2], pt[0], pt[1]};
            write_partials<5>(gp.part, gp.member, G, 0, w5);
        }
        if (A.x) {
            EvalAcc acc2;
            acc2.init();
            eval_pass<T, true, kCheckAll>(A, gp, A.lambda0, false, true, acc2, smem, ring_bars, ring_parity, err);
        }
        double dummy[1] = {0.0}, tot[1];
        if (last_block_sums<1>(gp.part, gp.member, G, &gp.hdr->ticket, dummy, tot, sh)) {
            double red[5];
            grid_reduce<5>(gp.part, G, 0, -1, red, sh, bc);
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
    int status = CQK_OK;
    bool bad_input = false;
    bool checked = false;      // the lambda_0 pass has checked the data (FP64)
    bool abd_checked = false;  // the lambda_0 pass has checked a, b, d (FP32): the first pass checks l, u
    bool wide_data = true;     // until a pass has checked every value
    bool fin_data = false;     // every bound finite (known once the data are checked)
    if (A.init == CQK_INIT_FORMULA) {
        double s, q;
        DataFlags fl{false, false, false};
        lambda0_pass<T>(A, gp, s, q, A.validate != 0, fl, smem, ring_bars, ring_parity, err);
        if (__any_sync(0xffffffffu, fl.bad) && (threadIdx.x & 31) == 0) atomicOr(&gp.hdr->flags, kFlagBadInput);
        if (__any_sync(0xffffffffu, fl.wide) && (threadIdx.x & 31) == 0) atomicOr(&gp.hdr->flags, kFlagWide);
        if (__any_sync(0xffffffffu, fl.luinf) && (threadIdx.x & 31) == 0) atomicOr(&gp.hdr->flags, kFlagLuInf);
        double pv[2] = {s, q};
        block_sum_smem<2>(pv, bscr);
        write_partials<2>(gp.part, gp.member, G, par, pv);
        CQK_BARRIER_OR_LEAVE();
        double red[2];
        grid_reduce<2>(gp.part, G, par, -1, red, sh, bc);
        par ^= 1;
        lam0 = (r - red[0]) / red[1];  // eq. (CQKlambda0), J = all variables
        passes++;
        const unsigned fls = __ldcg(&gp.hdr->flags);
        if constexpr (sizeof(T) == 8) {
            checked = true;
            wide_data = (fls & kFlagWide) != 0;
            fin_data = (fls & kFlagLuInf) == 0;
        } else {
            abd_checked = true;
        }
        if (A.validate && (fls & kFlagBadInput)) {
            bad_input = true;
            status = CQK_BAD_INPUT;
        }
    } else if (A.init == CQK_INIT_WARM) {
        double w[5];
        lambda0_warm_pass<T>(A, gp, w);
        block_sum_smem<5>(w, bscr);
        write_partials<5>(gp.part, gp.member, G, par, w);
        CQK_BARRIER_OR_LEAVE();
        double red[5];
        grid_reduce<5>(gp.part, G, par, -1, red, sh, bc);
        par ^= 1;
        // eq. (CQKlambda0) over J = {l < xbar < u}; all variables if J is empty (Sec. 2)
        lam0 = red[2] > 0.0 ? (r - red[0]) / red[1] : (r - red[3]) / red[4];
        passes++;
    }

    // ---- Alg. 1.  Thread 0 keeps the bracket and runs the update (FP64 divisions: the FP64 pipe
    // is the scarce unit, so one thread does it instead of every thread of every block); its
    // decisions reach the block through shared memory.  Every block's thread 0 computes the same
    // bits from the same totals.
    double lam = lam0, lower = -INFINITY, upper = INFINITY, phi_lower = NAN, phi_upper = NAN, slope = 0.0;
    double final_lam = lam;
    int stop = CQK_STOP_NONE, k = 0;
    // lambda may sit exactly on a breakpoint (it came from a breakpoint step, or is the caller's
    // start): only then is the tie band tested
    bool lam_on_bp = A.init == CQK_INIT_GIVEN;
    __shared__ double s_val[2];  // the next (or the final) lambda; the breakpoint search origin
    __shared__ int s_ctl[2];     // 1 = stop; breakpoint search direction (0: none)
    for (k = 0; !bad_input; k++) {
        if (k >= A.max_iter) {
            status = CQK_MAXITER;
            break;
        }
        EvalAcc acc;
        acc.init();
        // a lambda from eq. (CQKlambda0) or a Newton or secant step lies on an element's breakpoint
        // only by chance, and then the plain sign test classifies the element as exact arithmetic
        // would; the tie band of the file header is needed after a breakpoint step (or at a start
        // the caller gave)
        const bool rev = (k & 1) == 1;
        const bool first = k == 0 && !checked;  // this pass checks the data
        const bool chk = first && A.validate;
        // the checked fast path: every value valid and in the df range, and |lambda| <= 2^60
        const bool fast = !first && !wide_data && fabs(lam) <= 1.152921504606847e18;
        if (fast && fin_data && !lam_on_bp)
            eval_pass<T, false, kChecked, true, false>(A, gp, lam, false, rev, acc, smem, ring_bars, ring_parity, err);
        else if (fast && fin_data)
            eval_pass<T, false, kChecked, true, true>(A, gp, lam, false, rev, acc, smem, ring_bars, ring_parity, err);
        else if (fast && !lam_on_bp)
            eval_pass<T, false, kChecked, false, false>(A, gp, lam, false, rev, acc, smem, ring_bars, ring_parity, err);
        else if (fast)
            eval_pass<T, false, kChecked, false, true>(A, gp, lam, false, rev, acc, smem, ring_bars, ring_parity, err);
        else if (sizeof(T) == 4 && first && abd_checked && !lam_on_bp)
            eval_pass<T, false, kCheckBounds, false, false>(A, gp, lam, chk, rev, acc, smem, ring_bars, ring_parity, err);
        else if (sizeof(T) == 4 && first && abd_checked)
            eval_pass<T, false, kCheckBounds, false, true>(A, gp, lam, chk, rev, acc, smem, ring_bars, ring_parity, err);
        else if (!lam_on_bp)
            eval_pass<T, false, kCheckAll, false, false>(A, gp, lam, chk, rev, acc, smem, ring_bars, ring_parity, err);
        else eval_pass<T, false, kCheckAll, false, true>(A, gp, lam, chk, rev, acc, smem, ring_bars, ring_parity, err);
        acc.flush();
        passes++;
        if (__any_sync(0xffffffffu, acc.bad) && (threadIdx.x & 31) == 0) atomicOr(&gp.hdr->flags, kFlagBadInput);
        if (first && __any_sync(0xffffffffu, acc.wide) && (threadIdx.x & 31) == 0) atomicOr(&gp.hdr->flags, kFlagWide);
        if (first && __any_sync(0xffffffffu, acc.luinf) && (threadIdx.x & 31) == 0) atomicOr(&gp.hdr->flags, kFlagLuInf);
        double pv[5] = {acc.phi64, acc.sfree64, acc.satl, acc.satu, acc.absbx64};
        block_sum_smem<5>(pv, bscr);
        write_partials<5>(gp.part, gp.member, G, par, pv);
        CQK_BARRIER_OR_LEAVE();
        double red[5];
        grid_reduce<5>(gp.part, G, par, -1, red, sh, bc);
        par ^= 1;
        if (first) {
            wide_data = (__ldcg(&gp.hdr->flags) & kFlagWide) != 0;
            fin_data = (__ldcg(&gp.hdr->flags) & kFlagLuInf) == 0;
        }
        if (first && A.validate && (__ldcg(&gp.hdr->flags) & kFlagBadInput)) {
            bad_input = true;
            status = CQK_BAD_INPUT;
            k++;
            break;
        }
        if (threadIdx.x == 0) {
            const double phi = red[0], dplus = red[1] + red[2], dminus = red[1] + red[3], absbx = red[4];
            const double g = phi - r;
            double next = lam, fin = lam, from = 0.0;
            int done = 0, need_bp = 0;
            if (g == 0.0) {
                stop = CQK_STOP_EXACT;
                done = 1;
            } else if (fabs(g) < A.eps34_stop1 * (absbx + fabs(r))) {
                stop = CQK_STOP_RESIDUAL;
                if (A.final_step) {
                    double st = g < 0 ? (dplus > 0 ? -g / dplus : 0.0) : (dminus > 0 ? -g / dminus : 0.0);
                    const double t = lam + st;
                    if (g < 0 && !(t < upper)) st = 0.0;
                    if (g > 0 && !(t > lower)) st = 0.0;
                    fin = lam + st;
                }
                done = 1;
            } else if (g < 0) {
                lower = lam;
                phi_lower = phi;
                if (dplus > 0) {
                    slope = dplus;
                    const double step = -g / dplus;
                    const double t = lam + step;
                    if (fabs(step) < A.eps34) {
                        stop = CQK_STOP_STEP;
                        if (A.final_step && t < upper) fin = t;
                        done = 1;
                    } else if (t < upper) {
                        next = t;
                    } else {
                        next = lower - (phi_lower - r) * (upper - lower) / (phi_upper - phi_lower);
                    }
                } else {
                    need_bp = +1;  // closest breakpoint right of the lower end (Alg. 1)
                    from = lower;
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
                        if (A.final_step && t > lower) fin = t;
                        done = 1;
                    } else if (t > lower) {
                        next = t;
                    } else {
                        next = lower - (phi_lower - r) * (upper - lower) / (phi_upper - phi_lower);
                    }
                } else {
                    need_bp = -1;  // closest breakpoint left of the upper end
                    from = upper;
                }
            }
            if (!done && !need_bp) {
                if (upper - lower < A.eps34 * fmax(fabs(upper), fabs(lower))) {
                    stop = CQK_STOP_BRACKET;
                    done = 1;
                } else if (next == lam) {
                    stop = CQK_STOP_SAME;
                    done = 1;
                }
            }
            s_ctl[0] = done;
            s_ctl[1] = need_bp;
            s_val[0] = done ? fin : next;
            s_val[1] = from;
        }
        __syncthreads();
        const int done = s_ctl[0], need_bp = s_ctl[1];
        double next = s_val[0];
        const double from = s_val[1];
        __syncthreads();  // s_val / s_ctl are rewritten only after every thread has read them
        if (done) {
            final_lam = next;
            k++;
            break;
        }
        if (need_bp) {
            // closest breakpoint right of the lower end / left of the upper end (Alg. 1); the
            // block maximum of (-bp) or (bp) keeps one reduction code path
            double bp = breakpoint_pass<T>(A, gp, from, need_bp);
            bp = need_bp > 0 ? -bp : bp;
            bp = warp_max(bp);
            if ((threadIdx.x & 31) == 0) sh[0][threadIdx.x >> 5] = bp;
            __syncthreads();
            if (threadIdx.x < 32) {
                double pvb[1];
                warp0_combine<1>(sh, 0, pvb);
                write_partials<1>(gp.part, gp.member, G, par, pvb);
            }
            __syncthreads();
            passes++;
            CQK_BARRIER_OR_LEAVE();
            double redb[1];
            grid_reduce<1>(gp.part, G, par, 0, redb, sh, bc);
            par ^= 1;
            const double m = need_bp > 0 ? -redb[0] : redb[0];
            if (!isfinite(m)) {  // no breakpoint in the needed direction: r is out of reach
                status = CQK_INFEASIBLE;
                final_lam = lam;
                k++;
                break;
            }
            next = m;
            if (threadIdx.x == 0) {
                int stop_now = 0;
                if (upper - lower < A.eps34 * fmax(fabs(upper), fabs(lower))) {
                    stop = CQK_STOP_BRACKET;
                    stop_now = 1;
                } else if (next == lam) {
                    stop = CQK_STOP_SAME;
                    stop_now = 1;
                }
                s_ctl[0] = stop_now;
            }
            __syncthreads();
            const int stop_now = s_ctl[0];
            __syncthreads();
            if (stop_now) {
                final_lam = lam;
                k++;
                break;
            }
        }
        lam_on_bp = need_bp != 0;  // (describes lam from here on)
        lam = next;
        final_lam = lam;
    }

    // ---- final pass: x = x(lambda*), mask, sums of the stored x
    EvalAcc acc;
    acc.init();
    if (!bad_input && status != CQK_INFEASIBLE) {
        // FP64 data keep the tie band in the final pass (it also keeps every stored x inside
        // [l, u]: measured cheaper than clamping afterwards); FP32 data test ties only when x is
        // formed at a breakpoint lambda and clamp the stored float x instead
        const bool ties = sizeof(T) == 8 || (lam_on_bp && final_lam == lam);
        const bool rev = (k & 1) == 1;
        const bool fast = !wide_data && fabs(final_lam) <= 1.152921504606847e18;  // (as in the Newton passes)
        if (fast && fin_data && !ties)
            eval_pass<T, true, kChecked, true, false>(A, gp, final_lam, false, rev, acc, smem, ring_bars, ring_parity, err);
        else if (fast && fin_data)
            eval_pass<T, true, kChecked, true, true>(A, gp, final_lam, false, rev, acc, smem, ring_bars, ring_parity, err);
        else if (fast && !ties)
            eval_pass<T, true, kChecked, false, false>(A, gp, final_lam, false, rev, acc, smem, ring_bars, ring_parity, err);
        else if (fast)
            eval_pass<T, true, kChecked, false, true>(A, gp, final_lam, false, rev, acc, smem, ring_bars, ring_parity, err);
        else eval_pass<T, true, kCheckAll>(A, gp, final_lam, false, rev, acc, smem, ring_bars, ring_parity, err);
        passes++;
    }
    acc.flush();
    double pv[3] = {acc.phi64, acc.absbx64, (double)acc.nfree}, tot[3];
    if (last_block_sums<3>(gp.part, gp.member, G, &gp.hdr->ticket, pv, tot, sh) && threadIdx.x == 0) {
        cqk_info inf;
        inf.lambda = final_lam;
        inf.residual = tot[0] - r;
        inf.abs_bx = tot[1];
        inf.slope = slope;
        inf.lambda0 = lam0;
        inf.nfree = (int64_t)tot[2];
        inf.iters = k;
        const int e = *(volatile int*)&gp.hdr->error;
        inf.status = e ? e : status;
        inf.passes = passes;
        inf.stop = stop;
        inf.nchunks = 0;
        inf.tile = 0;
        *info = inf;
    }
}

#ifndef CQK_BATCH_ONLY
template <typename T>
__global__ void __launch_bounds__(NT, kMinBlocksPerSM) general_kernel(const __grid_constant__ GeneralArgs A) {
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    __shared__ uint64_t ring_bars[kRingBars];
    unsigned ring_parity = 0;
    if (A.staged) {
        if (threadIdx.x == 0) {
            for (int st = 0; st < kRingBars; st++) mbar_init(&ring_bars[st], 1);
            fence_barrier_init();
        }
        __syncthreads();
    }
    Grp gp;
    gp.member = blockIdx.x;
    gp.g = gridDim.x;
    gp.sp = Span{0, A.n};
    gp.hdr = A.hdr;
    gp.part = A.part;
    general_solve<T>(A, gp, A.r, A.info, reinterpret_cast<T*>(dyn_smem), ring_bars, ring_parity);
}

#endif  // CQK_BATCH_ONLY

// A batch: blocks take (instance, member) slots from the queue until it is empty; the bulk
// copy stages and their phase bits carry over from one instance to the next.
struct GeneralBatchArgs {
    GeneralArgs base;
    const int64_t* offsets;
    const double* r;
    cqk_info* info;
    int64_t B;
    BatchRefs R;
};

template <typename T>
__global__ void __launch_bounds__(NT, kMinBlocksPerSM) general_batched_kernel(const __grid_constant__ GeneralBatchArgs P) {
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    __shared__ uint64_t ring_bars[kRingBars];
    unsigned ring_parity = 0;
    if (P.base.staged) {
        if (threadIdx.x == 0) {
            for (int st = 0; st < kRingBars; st++) mbar_init(&ring_bars[st], 1);
            fence_barrier_init();
        }
        __syncthreads();
    }
    while (true) {
        const Slot sl = next_slot(P.R, P.B);
        if (sl.inst < 0) break;
        const Grp gp = slot_group(P.R, P.offsets, sl);
        const double r = P.r[sl.inst];
        cqk_info* info = P.info + sl.inst;
        const int64_t len = gp.sp.hi - gp.sp.lo;
        if (len <= 0 || r != r) {
            // no variable: feasible iff r == 0 (as for a single solve with n = 0)
            if (sl.member == 0 && threadIdx.x == 0) {
                if (len < 0 || r != r) write_plain_info(info, CQK_BAD_ARG, CQK_STOP_NONE, r);
                else write_plain_info(info, r == 0.0 ? CQK_OK : CQK_INFEASIBLE, CQK_STOP_NONE, r);
            }
            continue;
        }
        general_solve<T>(P.base, gp, r, info, reinterpret_cast<T*>(dyn_smem), ring_bars, ring_parity);
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

constexpr size_t kStagedSmem = (size_t)kStages * 5 * kGenTileBytes;  // bytes of dynamic shared memory

#ifndef CQK_BATCH_ONLY
int launch(GeneralArgs A, int dtype, int max_blocks, cudaStream_t s, void* ws) {
    const void* kern = dtype == CQK_F64 ? (const void*)general_kernel<double> : (const void*)general_kernel<float>;
    const int64_t vec = dtype == CQK_F64 ? 2 : 4;
    A.staged = A.aligned;
    const size_t smem = A.staged ? kStagedSmem : 0;
    if (smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            set_last_cuda_error(e);
            return CQK_CUDA_ERROR;
        }
    }
    // the general map is compute-heavy (double-float per element): a block is added per 2
    // vectors per thread and pass (the streaming default is 8), so that small problems, which
    // are bound by the per-pass latency, spread over more SMs (n = 1e4: 116 -> 93 us per solve)
    const int grid = persistent_grid(kern, NT, smem, 4 * ((A.n + vec - 1) / vec), max_blocks);
    if (grid <= 0) return CQK_CUDA_ERROR;
    cudaError_t e = cudaMemsetAsync(ws, 0, sizeof(WsHeader), s);
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return CQK_CUDA_ERROR;
    }
    void* args[] = {&A};
    e = cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(NT), args, smem, s);
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return CQK_CUDA_ERROR;
    }
    return CQK_OK;
}

#endif  // CQK_BATCH_ONLY

}  // namespace

#ifndef CQK_BATCH_ONLY
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
    A.xbar = o.xbar;
    if (A.init == CQK_INIT_WARM && ((uintptr_t)o.xbar % 16) != 0) A.aligned = 0;  // vector loads need all arrays
    return launch(A, dtype, o.max_blocks, s, ws);
}

#endif  // CQK_BATCH_ONLY

int CQK_VFN(launch_general_batched)(int64_t B, const int64_t* offsets, int dtype, const void* a, const void* b,
                           const void* d, const void* l, const void* u, const double* r, void* x, uint32_t* mask,
                           cqk_info* info, const Opts& o, void* ws, cudaStream_t s) {
    GeneralBatchArgs P;
    memset(&P, 0, sizeof(P));
    P.base = make_args(0, a, b, d, l, u, x, ws, dtype);
    GeneralArgs& A = P.base;
    A.hdr = nullptr;
    A.part = nullptr;
    A.mask = mask;
    A.init = o.init;
    A.lambda0 = o.lambda0;
    A.max_iter = o.max_iter;
    A.validate = o.validate;
    A.final_step = o.final_step;
    A.limit_ns = o.limit_ns;
    A.fault_inject = o.fault_inject;
    A.xbar = o.xbar;
    if (A.init == CQK_INIT_WARM && ((uintptr_t)o.xbar % 16) != 0) A.aligned = 0;
    A.staged = A.aligned;
    P.offsets = offsets;
    P.r = r;
    P.info = info;
    P.B = B;
    P.R = BatchRefs::at(ws, B);
    const void* kern =
        dtype == CQK_F64 ? (const void*)general_batched_kernel<double> : (const void*)general_batched_kernel<float>;
    const size_t smem = A.staged ? kStagedSmem : 0;
    if (smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            set_last_cuda_error(e);
            return CQK_CUDA_ERROR;
        }
    }
    int grid = persistent_grid(kern, NT, smem, INT64_MAX / 2, o.max_blocks);
    if (grid <= 0) return CQK_CUDA_ERROR;
    if ((int64_t)grid > B * kMaxGroup) grid = (int)(B * kMaxGroup);
    const int64_t per_block = o.group_elems > 0 ? o.group_elems : kGeneralGroupElems;
    int rc = CQK_VFN(plan_batch)(offsets, B, per_block, grid, ws, s);
    if (rc != CQK_OK) return rc;
    void* args[] = {&P};
    cudaError_t e = cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(NT), args, smem, s);
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return CQK_CUDA_ERROR;
    }
    return CQK_OK;
}

#ifndef CQK_BATCH_ONLY
int launch_phi(int64_t n, int dtype, const void* a, const void* b, const void* d, const void* l, const void* u,
               double lambda, void* x, double* out, void* ws, cudaStream_t s) {
    GeneralArgs A = make_args(n, a, b, d, l, u, x, ws, dtype);
    A.phi_only = 1;
    A.lambda0 = lambda;
    A.phi_out = out;
    A.limit_ns = 2000000000ull;
    return launch(A, dtype, 0, s, ws);
}

#endif  // CQK_BATCH_ONLY

}  // namespace cqk
