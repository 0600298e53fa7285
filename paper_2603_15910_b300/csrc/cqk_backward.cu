// cqk_backward.cu -- the adjoint of the solution map x*(a, b, d, l, u, r) (the paper has no
// backward pass; the formulas follow from differentiating its optimality conditions).
//
// At the solution, with F = {i : l_i < x_i < u_i} (the free set of the forward mask),
// x_i = (a_i + lambda b_i)/d_i on F, x_i is a bound off F, and sum_i b_i x_i = r (eq. (xopt),
// eq. (opt)).  Differentiating and eliminating d lambda, for an upstream gradient g:
//     Q = sum_F b_i^2/d_i,   mu = (sum_F b_i g_i/d_i) / Q
//     da_i = (g_i - mu b_i)/d_i on F, 0 off F;   dd_i = -x_i da_i;   db_i = lambda da_i - mu x_i
//     dl_i = g_i - mu b_i at a lower bound, du_i = g_i - mu b_i at an upper bound (else 0)
//     dr   = mu
// The simplex (b = d = 1, l = 0, u = +inf) gives dy_i = g_i - mean_F(g) on F, dr = mean_F(g);
// the l1 ball (Lemma 3.2) gives, with s = sgn(x), dy_i = g_i - s_i mean_F(s g) on F = {x != 0}
// and dr = mean_F(s g), or dy = g, dr = 0 when y lies inside the ball.  F empty (Q = 0): the
// map is not differentiable in r; mu = 0 and the status is CQK_NONDIFF.
//
// Two passes per instance: a map-reduce for (sum_F b g/d, Q), a group barrier, and a map
// that writes the requested gradients.  Arithmetic: double-float (~2^-44 relative) with an
// exact FP64 path for values outside its range, for both storage types.  The simplex adjoint
// with the forward mask streams g through shared-memory stages (bwd_simplex_staged).
#include <string.h>

#include "cqk_batch.cuh"
#include "cqk_stage.cuh"

namespace cqk {
namespace {

// 16-byte vectors per array in flight per lane (projections: g and x; the simplex with the
// forward mask: g alone); the half-unroll build keeps half as many
#ifdef CQK_UNROLL_HALF
constexpr int kBwdU = 2;
constexpr int kBwdUNoX = 3;
#else
constexpr int kBwdU = 4;
constexpr int kBwdUNoX = 6;
#endif
// general: a single instance keeps two vectors per array in flight (n = 2e7 FP64: 0.62 ->
// 0.58 ms); the batched kernel, whose per-slot state takes registers too, keeps one (two
// spilled and measured slower on the 256-instance batch)
constexpr int kBwdUGen = 2;
constexpr int kBwdUGenBatched = 1;

enum BwdKind { kBwdGeneral = 0, kBwdSimplex = 1, kBwdL1 = 2 };

struct BwdArgs {
    const void *g, *x, *a, *b, *d, *l, *u;
    const uint32_t* mask;
    const cqk_info* info;
    void *ga, *gb, *gd, *gl, *gu;
    double* gr;
    int32_t* status;
    int aligned;
    unsigned long long limit_ns;
    int fault_inject;
    int64_t n;  // single instance
    WsHeader* hdr;
    double* part;
    const int64_t* offsets;  // batch
    int64_t B;
    BatchRefs R;
};

// order comparisons of stored values on the integer pipe (an FP64 compare per element would
// take the FP64 unit): keys with -0 taken as +0; NaN never compares
template <typename T>
__device__ __forceinline__ long long cmpkey(T v) {
    if constexpr (sizeof(T) == 8) {
        const unsigned long long b = opaque_bits((double)v);
        return (b << 1) == 0ull ? 0ll : order_key((double)v);
    } else {
        return (long long)__float_as_int((float)v);  // unused for floats
    }
}
template <typename T>
__device__ __forceinline__ bool lt_val(T a, T b) {
    if constexpr (sizeof(T) == 8) return !f64_is_nan((double)a) && !f64_is_nan((double)b) && cmpkey(a) < cmpkey(b);
    else return a < b;
}
template <typename T>
__device__ __forceinline__ bool eq_val(T a, T b) {
    if constexpr (sizeof(T) == 8) return !f64_is_nan((double)a) && cmpkey(a) == cmpkey(b);
    else return a == b;
}

// the forward mask word holding vector q (0 when the vector has no element of the span), loaded
// with the vector's data so that both share one memory round trip
template <typename T>
__device__ __forceinline__ uint32_t mask_word(const BwdArgs& A, const Span& sp, int64_t q) {
    constexpr int V = VecOf<T>::V;
    const int64_t e0 = q * V;
    if (!A.mask || e0 >= sp.hi || e0 + V <= sp.lo) return 0u;
    return __ldg(A.mask + (e0 >> 5));
}

// free bits of the V elements of vector q (from the forward mask word, else from l < x < u)
template <typename T, int KIND>
__device__ __forceinline__ unsigned free_bits(const BwdArgs& A, int64_t q, uint32_t mw, const T (&x)[VecOf<T>::V],
                                              const T (&l)[VecOf<T>::V], const T (&u)[VecOf<T>::V]) {
    constexpr int V = VecOf<T>::V;
    if (A.mask) return (mw >> ((q * V) & 31)) & ((1u << V) - 1u);
    unsigned f = 0;
#pragma unroll
    for (int j = 0; j < V; j++) {
        bool fr;
        if (KIND == kBwdGeneral) fr = lt_val<T>(l[j], x[j]) && lt_val<T>(x[j], u[j]);
        else if (KIND == kBwdSimplex) fr = x[j] > T(0);
        else fr = x[j] != T(0);
        f |= (fr ? 1u : 0u) << j;
    }
    return f;
}

template <typename T>
__device__ __forceinline__ void load_or(const void* p, const Span& sp, int64_t q, bool aligned, T (&v)[VecOf<T>::V],
                                        bool (&ok)[VecOf<T>::V], T fill) {
    if (p) {
        load_vec<T>(static_cast<const T*>(p), sp, q, aligned, v, ok);
    } else {
#pragma unroll
        for (int j = 0; j < VecOf<T>::V; j++) v[j] = fill;
    }
}

template <typename T>
__device__ __forceinline__ void store_or(void* p, const Span& sp, int64_t q, bool aligned, const T (&v)[VecOf<T>::V]) {
    if (p) store_vec<T>(static_cast<T*>(p), sp, q, aligned, v);
}

// ---- per-element arithmetic -----------------------------------------------------------------
// Double-float (FP32 pipe, ~2^-44 relative) for FP64 data in the df operating range and for
// FP32 data; FP64 values outside the range take an exact FP64 path per element (out of line,
// so that it costs nothing when unused).  FP64 results are formed from the double-float ones by
// one FP64 add each (the parts widened on the integer pipe): measured faster than assembling
// the double on the integer pipe alone (the 256-instance general adjoint: 1.17 against 1.31 ms
// with half of the outputs so formed, 1.5 ms with all).

template <typename T>
__device__ __forceinline__ df to_df(T v) {
    if constexpr (sizeof(T) == 8) return split_f64_finite((double)v);
    else return df_make((float)v);
}
template <typename T>
__device__ __forceinline__ T from_df(df v) {
    if constexpr (sizeof(T) == 8) return df_to_f64_int(v);
    else return __fadd_rn(v.hi, v.lo);
}
// 1/d as a float pair (d > 0)
__device__ __forceinline__ df inv_df(df D) {
    const float r0 = rcp_approx(D.hi);
    const float res = fmaf(-D.lo, r0, fmaf(-D.hi, r0, 1.0f));
    return fast_two_sum(r0, __fmul_rn(r0, res));
}
template <typename T>
__device__ __forceinline__ bool in_df_range(T v) {
    if constexpr (sizeof(T) == 8) return df_in_range((double)v, false);
    else return true;
}

// exact FP64 fallbacks (values outside the df range)
__device__ __noinline__ void bwd_sum_exact(double g, double x, double b, double d, int kind, double& S, double& Q) {
    if (kind == kBwdGeneral) {
        const double w = b / d;
        S += w * g;
        Q += w * b;
    } else {
        S += (kind == kBwdL1 && x < 0.0) ? -g : g;
        Q += 1.0;
    }
}
__device__ __noinline__ void bwd_map_exact(double g, double x, double b, double d, bool fr, bool lower, double mu,
                                           double lam, int kind, double* out) {
    // out: ga (or gy), gb, gd, gl, gu
    if (kind == kBwdGeneral) {
        const double res = g - mu * b;
        const double daj = fr ? res / d : 0.0;
        out[0] = daj;
        out[1] = lam * daj - mu * x;
        out[2] = -x * daj;
        out[3] = !fr && lower ? res : 0.0;
        out[4] = !fr && !lower ? res : 0.0;
    } else {
        out[0] = fr ? g - ((kind == kBwdL1 && x < 0.0) ? -mu : mu) : 0.0;
    }
}

// ---- the general adjoint per vector, shared by the register and the staged sweeps ---------

// x_i at its lower bound (else at its upper one): x = l, and for a fixed variable (l = u) the
// side of the bound on which (a + lambda b)/d lies
template <typename T>
__device__ __forceinline__ bool at_lower(const BwdArgs& A, int64_t e, T x, T l, T u, T b, T d, double lam) {
    bool lower = eq_val<T>(x, l);
    if (lower && eq_val<T>(l, u) && A.a) {
        const double aj = (double)static_cast<const T*>(A.a)[e];
        lower = (aj + lam * (double)b) / (double)d <= (double)l;
    }
    return lower;
}

// pass 1: sum_F b g/d and sum_F b^2/d over the free elements (fb) of one vector (double-float,
// FP64 outside the df range)
template <typename T>
__device__ __forceinline__ void bwd_general_sums(unsigned fb, const T (&vg)[VecOf<T>::V], const T (&vb)[VecOf<T>::V],
                                                 const T (&vd)[VecOf<T>::V], const bool (&ok)[VecOf<T>::V], LazyDf& Sl,
                                                 LazyDf& Ql, double& S64, double& Q64) {
    constexpr int V = VecOf<T>::V;
    unsigned widem = 0;
#pragma unroll
    for (int j = 0; j < V; j++) {
        if (!ok[j] || !((fb >> j) & 1u)) continue;
        if (!(in_df_range<T>(vg[j]) && in_df_range<T>(vb[j]) && in_df_range<T>(vd[j]))) {
            widem |= 1u << j;
            continue;
        }
        const df G = to_df<T>(vg[j]), B = to_df<T>(vb[j]);
        const df W = df_mul(B, inv_df(to_df<T>(vd[j])));
        lazy_add(Sl, df_mul_lazy(W, G));
        lazy_add(Ql, df_mul_lazy(W, B));
    }
    for (unsigned m = widem; m; m &= m - 1) {
        const int j = __ffs(m) - 1;
        bwd_sum_exact((double)pick(vg, j), 0.0, (double)pick(vb, j), (double)pick(vd, j), kBwdGeneral, S64, Q64);
    }
}

// pass 2: the gradients of one vector (q: its global index), stored to every requested output
template <typename T>
__device__ __forceinline__ void bwd_general_grads(const BwdArgs& A, const Span& sp, int64_t q, bool aligned, unsigned fb,
                                                  const T (&vg)[VecOf<T>::V], const T (&vx)[VecOf<T>::V],
                                                  const T (&vb)[VecOf<T>::V], const T (&vd)[VecOf<T>::V],
                                                  const T (&vl)[VecOf<T>::V], const T (&vu)[VecOf<T>::V],
                                                  const bool (&ok)[VecOf<T>::V], bool need_lu, bool par_ok, df M, df Lm,
                                                  double mu, double lam) {
    constexpr int V = VecOf<T>::V;
    T oa[V], ob[V], od[V], ol[V], ou[V];
    unsigned widem = 0;
#pragma unroll
    for (int j = 0; j < V; j++) {
        const bool fr = (fb >> j) & 1u;
        oa[j] = ob[j] = od[j] = ol[j] = ou[j] = T(0);
        if (!ok[j]) continue;
        if (!(par_ok && in_df_range<T>(vg[j]) && in_df_range<T>(vx[j]) && in_df_range<T>(vb[j]) &&
              in_df_range<T>(vd[j]))) {
            widem |= 1u << j;
            continue;
        }
        const df G = to_df<T>(vg[j]), B = to_df<T>(vb[j]), X = to_df<T>(vx[j]);
        const df res = df_add(G, df_neg(df_mul(M, B)));
        const df mx = df_mul(M, X);
        if (fr) {
            const df ga = df_mul(res, inv_df(to_df<T>(vd[j])));
            oa[j] = from_df<T>(ga);
            od[j] = from_df<T>(df_neg(df_mul(X, ga)));
            ob[j] = from_df<T>(df_add(df_mul(Lm, ga), df_neg(mx)));
        } else {
            ob[j] = from_df<T>(df_neg(mx));
            const bool lower = need_lu && at_lower<T>(A, q * V + j, vx[j], vl[j], vu[j], vb[j], vd[j], lam);
            const T rv = from_df<T>(res);
            ol[j] = lower ? rv : T(0);
            ou[j] = lower ? T(0) : rv;
        }
    }
    for (unsigned m = widem; m; m &= m - 1) {
        const int j = __ffs(m) - 1;
        const bool fr = (fb >> j) & 1u;
        const bool lower = !fr && need_lu &&
                           at_lower<T>(A, q * V + j, pick(vx, j), pick(vl, j), pick(vu, j), pick(vb, j), pick(vd, j), lam);
        double o5[5];
        bwd_map_exact((double)pick(vg, j), (double)pick(vx, j), (double)pick(vb, j), (double)pick(vd, j), fr, lower, mu,
                      lam, kBwdGeneral, o5);
        put(oa, j, (T)o5[0]);
        put(ob, j, (T)o5[1]);
        put(od, j, (T)o5[2]);
        put(ol, j, (T)o5[3]);
        put(ou, j, (T)o5[4]);
    }
    store_or<T>(A.ga, sp, q, aligned, oa);
    store_or<T>(A.gb, sp, q, aligned, ob);
    store_or<T>(A.gd, sp, q, aligned, od);
    store_or<T>(A.gl, sp, q, aligned, ol);
    store_or<T>(A.gu, sp, q, aligned, ou);
}

// one instance by one group (WARP: by one warp alone; gp.sp is the only field used).  NOX: the
// simplex with the forward mask, where F comes from the mask and x is not read.
template <typename T, int KIND, bool NOX, bool WARP = false, int UG = kBwdUGen>
__device__ __forceinline__ void bwd_instance(const BwdArgs& A, const Grp& gp, int64_t inst) {
    constexpr int V = VecOf<T>::V;
    constexpr int U = KIND == kBwdGeneral ? UG : (NOX ? kBwdUNoX : kBwdU);
    __shared__ double sh[kPartialQ][NWARP];
    __shared__ double bc[kPartialQ];
    const Span sp = gp.sp;
    const bool aligned = A.aligned != 0;
    const int lane = threadIdx.x & 31;
    const cqk_info* inf = A.info + inst;
    const double lam = KIND == kBwdGeneral ? inf->lambda : 0.0;
    const bool inside = KIND == kBwdL1 && inf->stop == CQK_STOP_INSIDE;
    const bool need_lu = KIND == kBwdGeneral && (!A.mask || A.gl || A.gu);
    const void* xp = NOX ? nullptr : A.x;
    const WarpSweep sw = WARP ? WarpSweep::solo(span_qlo<V>(sp), span_qhi<V>(sp), U)
                              : WarpSweep(span_qlo<V>(sp), span_qhi<V>(sp), U, gp.member, gp.g);

    // ---- pass 1: sum_F b g/d and Q = sum_F b^2/d (simplex / l1: sum_F (s) g and |F|); the
    // general kind with the forward mask needs neither x nor l, u here
    const void* xp1 = (KIND == kBwdGeneral && A.mask) ? nullptr : xp;
    LazyDf Sl{0.0f, 0.0f}, Ql{0.0f, 0.0f};
    double S64 = 0.0, Q64 = 0.0;
    long long nF = 0;
    if (!inside) {
        for (int64_t it = 0; it < sw.count; it++) {
            if ((it & 7) == 7) {
                S64 += lazy_value_int(Sl);
                Q64 += lazy_value_int(Ql);
                Sl = Ql = LazyDf{0.0f, 0.0f};
            }
            const int64_t base = sw.base(it, false);
            T vg[U][V], vx[U][V], vb[U][V], vd[U][V], vl[U][V], vu[U][V];
            bool ok[U][V];
            uint32_t mw[U];
#pragma unroll
            for (int w = 0; w < U; w++) {
                const int64_t q = base + w * 32 + lane;
                load_vec<T>(static_cast<const T*>(A.g), sp, q, aligned, vg[w], ok[w]);
                mw[w] = mask_word<T>(A, sp, q);
                load_or<T>(xp1, sp, q, aligned, vx[w], ok[w], T(0));
                if (KIND == kBwdGeneral) {
                    load_or<T>(A.b, sp, q, aligned, vb[w], ok[w], T(1));
                    load_or<T>(A.d, sp, q, aligned, vd[w], ok[w], T(1));
                }
                if (KIND == kBwdGeneral && !A.mask) {
                    load_or<T>(A.l, sp, q, aligned, vl[w], ok[w], T(0));
                    load_or<T>(A.u, sp, q, aligned, vu[w], ok[w], T(0));
                }
            }
#pragma unroll
            for (int w = 0; w < U; w++) {
                const int64_t q = base + w * 32 + lane;
                const unsigned fb = free_bits<T, KIND>(A, q, mw[w], vx[w], vl[w], vu[w]);
                if constexpr (KIND == kBwdGeneral) {
                    bwd_general_sums<T>(fb, vg[w], vb[w], vd[w], ok[w], Sl, Ql, S64, Q64);
                    continue;
                }
                unsigned widem = 0;
#pragma unroll
                for (int j = 0; j < V; j++) {
                    if (!ok[w][j] || !((fb >> j) & 1u)) continue;
                    if (!in_df_range<T>(vg[w][j])) {
                        widem |= 1u << j;
                        continue;
                    }
                    const df G = to_df<T>(vg[w][j]);
                    if (KIND == kBwdSimplex) lazy_add(Sl, G);
                    else lazy_add(Sl, vx[w][j] > T(0) ? G : df_neg(G));
                    nF++;
                }
                for (unsigned m = widem; m; m &= m - 1) {
                    const int j = __ffs(m) - 1;
                    bwd_sum_exact((double)pick(vg[w], j), (double)pick(vx[w], j), 1.0, 1.0, KIND, S64, Q64);
                }
            }
        }
    }
    double pv[2] = {lazy_value_int(Sl) + S64, KIND == kBwdGeneral ? lazy_value_int(Ql) + Q64 : (double)nF + Q64};
    double red[2];
    if constexpr (WARP) {
        red[0] = warp_sum(pv[0]);
        red[1] = warp_sum(pv[1]);
    } else {
        block_sum<2>(pv, sh);
        write_partials<2>(gp.part, gp.member, gp.g, 0, pv);
        const unsigned target = (unsigned)gp.g + (A.fault_inject == 1 ? 1u : 0u);
        if (!group_barrier(gp, target, A.limit_ns, A.fault_inject == 1)) {
            if (threadIdx.x == 0 && A.status) A.status[inst] = CQK_TIMEOUT;
            return;
        }
        grid_reduce<2>(gp.part, gp.g, 0, -1, red, sh, bc);
    }
    const bool nondiff = !inside && !(red[1] > 0.0);
    const double mu = (inside || nondiff) ? 0.0 : red[0] / red[1];
    const df M = df_from_f64(mu), Lm = df_from_f64(lam);
    const bool par_ok = fabs(mu) <= 1.152921504606847e18 && fabs(lam) <= 1.152921504606847e18;  // 2^60

    // ---- pass 2: the gradients
    for (int64_t it = 0; it < sw.count; it++) {
        const int64_t base = sw.base(it, true);
        T vg[U][V], vx[U][V], vb[U][V], vd[U][V], vl[U][V], vu[U][V];
        bool ok[U][V];
        uint32_t mw[U];
#pragma unroll
        for (int w = 0; w < U; w++) {
            const int64_t q = base + w * 32 + lane;
            load_vec<T>(static_cast<const T*>(A.g), sp, q, aligned, vg[w], ok[w]);
            mw[w] = inside ? 0u : mask_word<T>(A, sp, q);
            load_or<T>(xp, sp, q, aligned, vx[w], ok[w], T(0));
            if (KIND == kBwdGeneral) {
                load_or<T>(A.b, sp, q, aligned, vb[w], ok[w], T(1));
                load_or<T>(A.d, sp, q, aligned, vd[w], ok[w], T(1));
            }
            if (need_lu) {
                load_or<T>(A.l, sp, q, aligned, vl[w], ok[w], T(0));
                load_or<T>(A.u, sp, q, aligned, vu[w], ok[w], T(0));
            }
        }
#pragma unroll
        for (int w = 0; w < U; w++) {
            const int64_t q = base + w * 32 + lane;
            const unsigned fb = inside ? ((1u << V) - 1u) : free_bits<T, KIND>(A, q, mw[w], vx[w], vl[w], vu[w]);
            if constexpr (KIND == kBwdGeneral) {
                bwd_general_grads<T>(A, sp, q, aligned, fb, vg[w], vx[w], vb[w], vd[w], vl[w], vu[w], ok[w], need_lu,
                                     par_ok, M, Lm, mu, lam);
                continue;
            }
            T oa[V];
            unsigned widem = 0;
#pragma unroll
            for (int j = 0; j < V; j++) {
                const bool fr = (fb >> j) & 1u;
                oa[j] = T(0);
                if (!ok[w][j]) continue;
                if (KIND == kBwdL1 && inside) {
                    oa[j] = vg[w][j];
                    continue;
                }
                if (!(par_ok && in_df_range<T>(vg[w][j]) && in_df_range<T>(vx[w][j]))) {
                    widem |= 1u << j;
                    continue;
                }
                if (fr) {
                    const df G = to_df<T>(vg[w][j]);
                    const bool neg = KIND == kBwdL1 && vx[w][j] < T(0);
                    oa[j] = from_df<T>(df_add(G, neg ? M : df_neg(M)));
                }
            }
            for (unsigned m = widem; m; m &= m - 1) {
                const int j = __ffs(m) - 1;
                double o5[5];
                bwd_map_exact((double)pick(vg[w], j), (double)pick(vx[w], j), 1.0, 1.0, (fb >> j) & 1u, false, mu, lam,
                              KIND, o5);
                put(oa, j, (T)o5[0]);
            }
            store_or<T>(A.ga, sp, q, aligned, oa);
        }
    }
    if constexpr (WARP) {
        if (lane == 0) {
            if (A.gr) A.gr[inst] = mu;
            if (A.status) A.status[inst] = nondiff ? CQK_NONDIFF : CQK_OK;
        }
    } else if (gp.member == 0 && threadIdx.x == 0) {
        if (A.gr) A.gr[inst] = mu;
        if (A.status) {
            const int e = *(volatile int*)&gp.hdr->error;
            A.status[inst] = e ? e : (nondiff ? CQK_NONDIFF : CQK_OK);
        }
    }
}

// The simplex adjoint with the forward mask on 16-byte aligned data: g streams through
// kBwdStages shared-memory stages of 16 KB by bulk copies (tiles of the span dealt round robin
// to the group's blocks), so that each block keeps 48 KB in flight instead of the few vectors
// its registers hold.  Pass 1 sums g over F, pass 2 (tiles in reverse order, the last ones
// still in L2) writes gy = g - mean_F(g) on F and 0 off F.  The arithmetic per element is the
// one of bwd_instance.
constexpr int kBwdStages = 4;
constexpr size_t kBwdSmem = (size_t)kBwdStages * 16384;

template <typename T>
__device__ void bwd_simplex_staged(const BwdArgs& A, const Grp& gp, int64_t inst, T* smem, uint64_t* bars,
                                   unsigned& parity) {
    constexpr int V = VecOf<T>::V;
    constexpr int TT = 16384 / (int)sizeof(T);
    constexpr int VPT = TT / V / NT;  // vectors per thread and tile
    constexpr int S = kBwdStages;
    using VT = typename VecOf<T>::type;
    static_assert(VPT * V * NT == TT, "tile layout");
    __shared__ double sh[kPartialQ][NWARP];
    __shared__ double bc[kPartialQ];
    const Span sp = gp.sp;
    const T* __restrict__ g = static_cast<const T*>(A.g);
    const T* src[1] = {g};
    TileRing<T, 1, TT> ring;
    ring.setup(sp.lo, sp.hi, smem, bars, gp.member, gp.g);
    ring.parity = parity;
    int* err = gp.hdr ? &gp.hdr->error : nullptr;
    int dummy_err = 0;
    if (!err) err = &dummy_err;

    // the V values of vector ql of tile c (stage when the bulk copy delivered it, else global)
    auto vec_of = [&](const T* stage, int64_t c, int ql, int64_t sb0, int64_t sb1, T (&v)[V], bool (&ok)[V]) {
        const int64_t q = c * (TT / V) + ql;
        if (q * V >= sb0 && (q + 1) * V <= sb1) {
            const VT w = reinterpret_cast<const VT*>(stage)[ql];
#pragma unroll
            for (int j = 0; j < V; j++) {
                v[j] = reinterpret_cast<const T*>(&w)[j];
                ok[j] = true;
            }
        } else {
            load_vec<T>(g, sp, q, false, v, ok);
        }
    };
    // one sweep over the block's tiles: f(stage, c, sb0, sb1, i, mask words) per tile, all
    // threads; the mask words of a tile are loaded before its stage is waited for
    auto sweep = [&](bool rev, auto&& f) {
        if (threadIdx.x == 0)
            for (int k = 0; k < S - 1; k++)
                if (k < ring.count) ring.issue(ring.tile(k, rev), k, src);
        int stg = 0;
        for (int64_t i = 0; i < ring.count; i++, stg = stg + 1 == S ? 0 : stg + 1) {
            if (threadIdx.x == 0 && i + S - 1 < ring.count) {
                const int s2 = stg == 0 ? S - 1 : stg - 1;  // (i + S - 1) mod S
                ring.issue(ring.tile(i + S - 1, rev), s2, src);
            }
            const int64_t c = ring.tile(i, rev);
            uint32_t mw[VPT];
#pragma unroll
            for (int k = 0; k < VPT; k++) mw[k] = mask_word<T>(A, sp, c * (TT / V) + k * NT + (int)threadIdx.x);
            mbar_wait(&ring.bar[stg], (ring.parity >> stg) & 1u, err, A.limit_ns, CQK_TIMEOUT);
            ring.parity ^= 1u << stg;
            f(ring.stage(stg, 0), c, ring.b0(c), ring.b1(c), i, mw);
            __syncthreads();  // the stage is refilled only after every thread has read it
        }
    };

    // ---- pass 1: sum_F g and |F|
    LazyDf Sl{0.0f, 0.0f};
    double S64 = 0.0, Q64 = 0.0;
    long long nF = 0;
    sweep(false, [&](const T* stage, int64_t c, int64_t sb0, int64_t sb1, int64_t i, const uint32_t (&mw)[VPT]) {
        if ((i & 7) == 7) {
            S64 += lazy_value_int(Sl);
            Sl = LazyDf{0.0f, 0.0f};
        }
#pragma unroll
        for (int k = 0; k < VPT; k++) {
            const int ql = k * NT + (int)threadIdx.x;
            const int64_t q = c * (TT / V) + ql;
            T v[V];
            bool ok[V];
            vec_of(stage, c, ql, sb0, sb1, v, ok);
            const unsigned fb = (mw[k] >> ((q * V) & 31)) & ((1u << V) - 1u);
#pragma unroll
            for (int j = 0; j < V; j++) {
                if (!ok[j] || !((fb >> j) & 1u)) continue;
                if (!in_df_range<T>(v[j])) {
                    bwd_sum_exact((double)v[j], 0.0, 1.0, 1.0, kBwdSimplex, S64, Q64);
                    continue;
                }
                lazy_add(Sl, to_df<T>(v[j]));
                nF++;
            }
        }
    });
    double pv[2] = {lazy_value_int(Sl) + S64, (double)nF + Q64};
    double red[2];
    block_sum<2>(pv, sh);
    write_partials<2>(gp.part, gp.member, gp.g, 0, pv);
    const unsigned target = (unsigned)gp.g + (A.fault_inject == 1 ? 1u : 0u);
    if (!group_barrier(gp, target, A.limit_ns, A.fault_inject == 1)) {
        if (threadIdx.x == 0 && A.status) A.status[inst] = CQK_TIMEOUT;
        parity = ring.parity;
        return;
    }
    grid_reduce<2>(gp.part, gp.g, 0, -1, red, sh, bc);
    const bool nondiff = !(red[1] > 0.0);
    const double mu = nondiff ? 0.0 : red[0] / red[1];
    const df M = df_from_f64(mu);
    const bool par_ok = fabs(mu) <= 1.152921504606847e18;  // 2^60

    // ---- pass 2: gy
    T* __restrict__ gy = static_cast<T*>(A.ga);
    sweep(true, [&](const T* stage, int64_t c, int64_t sb0, int64_t sb1, int64_t, const uint32_t (&mw)[VPT]) {
#pragma unroll
        for (int k = 0; k < VPT; k++) {
            const int ql = k * NT + (int)threadIdx.x;
            const int64_t q = c * (TT / V) + ql;
            T v[V];
            bool ok[V];
            vec_of(stage, c, ql, sb0, sb1, v, ok);
            const unsigned fb = (mw[k] >> ((q * V) & 31)) & ((1u << V) - 1u);
            T oa[V];
#pragma unroll
            for (int j = 0; j < V; j++) {
                const bool fr = (fb >> j) & 1u;
                oa[j] = T(0);
                if (!ok[j] || !fr) continue;
                if (par_ok && in_df_range<T>(v[j])) {
                    oa[j] = from_df<T>(df_add(to_df<T>(v[j]), df_neg(M)));
                } else {
                    double o5[5];
                    bwd_map_exact((double)v[j], 0.0, 1.0, 1.0, true, false, mu, 0.0, kBwdSimplex, o5);
                    oa[j] = (T)o5[0];
                }
            }
            if (gy) store_vec<T>(gy, sp, q, A.aligned != 0, oa);
        }
    });
    parity = ring.parity;
    if (gp.member == 0 && threadIdx.x == 0) {
        if (A.gr) A.gr[inst] = mu;
        if (A.status) {
            const int e = gp.hdr ? *(volatile int*)&gp.hdr->error : 0;
            A.status[inst] = e ? e : (nondiff ? CQK_NONDIFF : CQK_OK);
        }
    }
}

template <typename T, int KIND, bool BATCHED, bool NOX>
__global__ void __launch_bounds__(NT, kMinBlocksPerSM) backward_kernel(const __grid_constant__ BwdArgs A) {
    // the staged simplex adjoint (NOX on aligned data): stages and their mbarriers
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    __shared__ uint64_t bars[NOX ? kBwdStages : 1];
    unsigned parity = 0;
    const bool staged = NOX && A.aligned != 0;
    if (NOX) {
        if (threadIdx.x == 0) {
            for (int k = 0; k < kBwdStages; k++) mbar_init(&bars[k], 1);
            fence_barrier_init();
        }
        __syncthreads();
    }
    if constexpr (!BATCHED) {
        Grp gp;
        gp.member = blockIdx.x;
        gp.g = gridDim.x;
        gp.sp = Span{0, A.n};
        gp.hdr = A.hdr;
        gp.part = A.part;
        if (staged) bwd_simplex_staged<T>(A, gp, 0, reinterpret_cast<T*>(dyn_smem), bars, parity);
        else bwd_instance<T, KIND, NOX>(A, gp, 0);
        return;
    } else {
        while (true) {
            const Slot sl = next_slot(A.R, A.B);
            if (KIND != kBwdGeneral && sl.pack_first >= 0) {  // small instances, one per warp
                const long long p = sl.pack_first + (threadIdx.x >> 5);
                if (p < A.B) {
                    const int inst = A.R.order[p];
                    Grp gw;
                    gw.member = 0;
                    gw.g = 1;
                    gw.sp = Span{A.offsets[inst], A.offsets[inst + 1]};
                    gw.hdr = nullptr;
                    gw.part = nullptr;
                    if (gw.sp.hi < gw.sp.lo) {
                        if ((threadIdx.x & 31) == 0) {
                            if (A.gr) A.gr[inst] = 0.0;
                            if (A.status) A.status[inst] = CQK_BAD_ARG;
                        }
                    } else {
                        bwd_instance<T, KIND, NOX, true, kBwdUGenBatched>(A, gw, inst);
                    }
                }
                continue;
            }
            if (sl.inst < 0) break;
            const Grp gp = slot_group(A.R, A.offsets, sl);
            if (gp.sp.hi < gp.sp.lo) {
                if (sl.member == 0 && threadIdx.x == 0) {
                    if (A.gr) A.gr[sl.inst] = 0.0;
                    if (A.status) A.status[sl.inst] = CQK_BAD_ARG;
                }
                continue;
            }
            if (staged) bwd_simplex_staged<T>(A, gp, sl.inst, reinterpret_cast<T*>(dyn_smem), bars, parity);
            else bwd_instance<T, KIND, NOX, false, kBwdUGenBatched>(A, gp, sl.inst);
        }
    }
}

template <typename T, int KIND, bool NOX = false>
const void* pick_kernel(bool batched) {
#ifdef CQK_BATCH_ONLY
    return batched ? (const void*)backward_kernel<T, KIND, true, NOX> : nullptr;  // variant builds: batches only
#else
    return batched ? (const void*)backward_kernel<T, KIND, true, NOX> : (const void*)backward_kernel<T, KIND, false, NOX>;
#endif
}

}  // namespace

int CQK_VFN(launch_backward)(int kind, int64_t B, const int64_t* offsets, int64_t n, int dtype, const void* g, const void* x,
                    const void* a, const void* b, const void* d, const void* l, const void* u, const uint32_t* mask,
                    const cqk_info* info, void* ga, void* gb, void* gd, void* gl, void* gu, double* gr,
                    int32_t* status, const Opts& o, void* ws, cudaStream_t s) {
    BwdArgs A;
    memset(&A, 0, sizeof(A));
    A.g = g;
    A.x = x;
    A.a = a;
    A.b = b;
    A.d = d;
    A.l = l;
    A.u = u;
    A.mask = mask;
    A.info = info;
    A.ga = ga;
    A.gb = gb;
    A.gd = gd;
    A.gl = gl;
    A.gu = gu;
    A.gr = gr;
    A.status = status;
    A.limit_ns = o.limit_ns;
    A.fault_inject = o.fault_inject;
    const uintptr_t all = (uintptr_t)g | (uintptr_t)x | (uintptr_t)b | (uintptr_t)d | (uintptr_t)l | (uintptr_t)u |
                          (uintptr_t)ga | (uintptr_t)gb | (uintptr_t)gd | (uintptr_t)gl | (uintptr_t)gu;
    A.aligned = (all % 16 == 0) ? 1 : 0;
    const bool batched = offsets != nullptr;
    const void* kern;
    const bool nox = kind == kBwdSimplex && mask;  // F from the mask: x is not read
    if (dtype == CQK_F64) {
        kern = kind == kBwdGeneral ? pick_kernel<double, kBwdGeneral>(batched)
               : kind == kBwdSimplex ? (nox ? pick_kernel<double, kBwdSimplex, true>(batched)
                                            : pick_kernel<double, kBwdSimplex>(batched))
                                     : pick_kernel<double, kBwdL1>(batched);
    } else {
        kern = kind == kBwdGeneral ? pick_kernel<float, kBwdGeneral>(batched)
               : kind == kBwdSimplex ? (nox ? pick_kernel<float, kBwdSimplex, true>(batched)
                                            : pick_kernel<float, kBwdSimplex>(batched))
                                     : pick_kernel<float, kBwdL1>(batched);
    }
    if (!kern) return CQK_BAD_ARG;
    const int64_t vec = dtype == CQK_F64 ? 2 : 4;
    // the staged simplex adjoint takes kBwdSmem of dynamic shared memory (requested for every
    // NOX launch: the kernel decides on alignment at run time)
    const size_t smem = nox ? kBwdSmem : 0;
    int grid;
    cudaError_t e;
    if (smem) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            set_last_cuda_error(e);
            return CQK_CUDA_ERROR;
        }
    }
    if (batched) {
        A.offsets = offsets;
        A.B = B;
        A.R = BatchRefs::at(ws, B);
        grid = persistent_grid(kern, NT, smem, INT64_MAX / 2, o.max_blocks);
        if (grid <= 0) return CQK_CUDA_ERROR;
        if ((int64_t)grid > B * kMaxGroup) grid = (int)(B * kMaxGroup);
        const int64_t per_block =
            o.group_elems > 0 ? o.group_elems : (kind == kBwdGeneral ? kBackwardGroupElems : kSimplexGroupElems);
        const int rc = CQK_VFN(plan_batch)(offsets, B, per_block, grid, ws, s, kind == kBwdGeneral ? 0 : o.warp_log2);
        if (rc != CQK_OK) return rc;
    } else {
        A.n = n;
        A.hdr = static_cast<WsHeader*>(ws);
        A.part = reinterpret_cast<double*>(static_cast<char*>(ws) + sizeof(WsHeader));
        grid = persistent_grid(kern, NT, smem, (n + vec - 1) / vec, o.max_blocks);
        if (grid <= 0) return CQK_CUDA_ERROR;
        e = cudaMemsetAsync(ws, 0, sizeof(WsHeader), s);
        if (e != cudaSuccess) {
            set_last_cuda_error(e);
            return CQK_CUDA_ERROR;
        }
    }
    void* args[] = {&A};
    e = cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(NT), args, smem, s);
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return CQK_CUDA_ERROR;
    }
    return CQK_OK;
}

}  // namespace cqk
