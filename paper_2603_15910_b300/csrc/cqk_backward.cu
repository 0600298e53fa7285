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
// that writes the requested gradients.  Arithmetic is FP64 for both storage types.
#include <string.h>

#include "cqk_batch.cuh"

namespace cqk {
namespace {

constexpr int kBwdU = 2;  // 16-byte vectors per array in flight per lane

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

// free bits of the V elements of vector q (from the forward mask, else from l < x < u)
template <typename T, int KIND>
__device__ __forceinline__ unsigned free_bits(const BwdArgs& A, const Span& sp, int64_t q, const T (&x)[VecOf<T>::V],
                                              const T (&l)[VecOf<T>::V], const T (&u)[VecOf<T>::V]) {
    constexpr int V = VecOf<T>::V;
    if (A.mask) {
        const int64_t e0 = q * V;
        if (e0 >= sp.hi || e0 + V <= sp.lo) return 0u;  // no element of the span: no mask word
        const uint32_t w = __ldg(A.mask + (e0 >> 5));
        return (w >> (e0 & 31)) & ((1u << V) - 1u);
    }
    unsigned f = 0;
#pragma unroll
    for (int j = 0; j < V; j++) {
        bool fr;
        if (KIND == kBwdGeneral) fr = l[j] < x[j] && x[j] < u[j];
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

// one instance by one group
template <typename T, int KIND>
__device__ __forceinline__ void bwd_instance(const BwdArgs& A, const Grp& gp, int64_t inst) {
    constexpr int V = VecOf<T>::V;
    constexpr int U = kBwdU;
    __shared__ double sh[kPartialQ][NWARP];
    __shared__ double bc[kPartialQ];
    const Span sp = gp.sp;
    const bool aligned = A.aligned != 0;
    const int lane = threadIdx.x & 31;
    const cqk_info* inf = A.info + inst;
    const double lam = KIND == kBwdGeneral ? inf->lambda : 0.0;
    const bool inside = KIND == kBwdL1 && inf->stop == CQK_STOP_INSIDE;
    const bool need_lu = KIND == kBwdGeneral && (!A.mask || A.gl || A.gu);
    const WarpSweep sw(span_qlo<V>(sp), span_qhi<V>(sp), U, gp.member, gp.g);

    // ---- pass 1: sum_F b g/d and Q = sum_F b^2/d (simplex / l1: sum_F (s) g and |F|)
    double S = 0.0, Q = 0.0;
    if (!inside) {
        for (int64_t it = 0; it < sw.count; it++) {
            const int64_t base = sw.base(it, false);
            T vg[U][V], vx[U][V], vb[U][V], vd[U][V], vl[U][V], vu[U][V];
            bool ok[U][V];
#pragma unroll
            for (int w = 0; w < U; w++) {
                const int64_t q = base + w * 32 + lane;
                load_vec<T>(static_cast<const T*>(A.g), sp, q, aligned, vg[w], ok[w]);
                load_or<T>(A.x, sp, q, aligned, vx[w], ok[w], T(0));
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
                const unsigned fb = free_bits<T, KIND>(A, sp, q, vx[w], vl[w], vu[w]);
#pragma unroll
                for (int j = 0; j < V; j++) {
                    if (!ok[w][j] || !((fb >> j) & 1u)) continue;
                    const double gj = (double)vg[w][j];
                    if (KIND == kBwdGeneral) {
                        const double wj = (double)vb[w][j] / (double)vd[w][j];
                        S += wj * gj;
                        Q += wj * (double)vb[w][j];
                    } else if (KIND == kBwdSimplex) {
                        S += gj;
                        Q += 1.0;
                    } else {
                        S += vx[w][j] > T(0) ? gj : -gj;
                        Q += 1.0;
                    }
                }
            }
        }
    }
    double pv[2] = {S, Q};
    block_sum<2>(pv, sh);
    write_partials<2>(gp.part, gp.member, gp.g, 0, pv);
    const unsigned target = (unsigned)gp.g + (A.fault_inject ? 1u : 0u);
    if (!group_barrier(gp, target, A.limit_ns, A.fault_inject != 0)) {
        if (threadIdx.x == 0 && A.status) A.status[inst] = CQK_TIMEOUT;
        return;
    }
    double red[2];
    grid_reduce<2>(gp.part, gp.g, 0, -1, red, sh, bc);
    const bool nondiff = !inside && !(red[1] > 0.0);
    const double mu = (inside || nondiff) ? 0.0 : red[0] / red[1];

    // ---- pass 2: the gradients
    for (int64_t it = 0; it < sw.count; it++) {
        const int64_t base = sw.base(it, true);
        T vg[U][V], vx[U][V], vb[U][V], vd[U][V], vl[U][V], vu[U][V];
        bool ok[U][V];
#pragma unroll
        for (int w = 0; w < U; w++) {
            const int64_t q = base + w * 32 + lane;
            load_vec<T>(static_cast<const T*>(A.g), sp, q, aligned, vg[w], ok[w]);
            load_or<T>(A.x, sp, q, aligned, vx[w], ok[w], T(0));
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
            const unsigned fb = inside ? ((1u << V) - 1u) : free_bits<T, KIND>(A, sp, q, vx[w], vl[w], vu[w]);
            T oa[V], ob[V], od[V], ol[V], ou[V];
#pragma unroll
            for (int j = 0; j < V; j++) {
                const bool fr = (fb >> j) & 1u;
                const double gj = (double)vg[w][j], xj = (double)vx[w][j];
                if (KIND == kBwdGeneral) {
                    const double bj = (double)vb[w][j], dj = (double)vd[w][j];
                    const double res = gj - mu * bj;
                    const double daj = fr ? res / dj : 0.0;
                    oa[j] = (T)daj;
                    od[j] = (T)(-xj * daj);
                    ob[j] = (T)(lam * daj - mu * xj);
                    bool lower = false;
                    if (!fr && need_lu && ok[w][j]) {
                        lower = vx[w][j] == vl[w][j];
                        if (lower && vl[w][j] == vu[w][j] && A.a) {
                            // a fixed variable (l = u) is at its lower bound when (a + lambda b)/d <= l
                            const double aj = (double)static_cast<const T*>(A.a)[q * V + j];
                            lower = (aj + lam * bj) / dj <= (double)vl[w][j];
                        }
                    }
                    ol[j] = (T)(!fr && lower ? res : 0.0);
                    ou[j] = (T)(!fr && !lower ? res : 0.0);
                } else if (KIND == kBwdSimplex) {
                    oa[j] = (T)(fr ? gj - mu : 0.0);
                } else {
                    oa[j] = (T)(inside ? gj : (fr ? gj - (vx[w][j] > T(0) ? mu : -mu) : 0.0));
                }
            }
            store_or<T>(A.ga, sp, q, aligned, oa);
            if (KIND == kBwdGeneral) {
                store_or<T>(A.gb, sp, q, aligned, ob);
                store_or<T>(A.gd, sp, q, aligned, od);
                store_or<T>(A.gl, sp, q, aligned, ol);
                store_or<T>(A.gu, sp, q, aligned, ou);
            }
        }
    }
    if (gp.member == 0 && threadIdx.x == 0) {
        if (A.gr) A.gr[inst] = mu;
        if (A.status) {
            const int e = *(volatile int*)&gp.hdr->error;
            A.status[inst] = e ? e : (nondiff ? CQK_NONDIFF : CQK_OK);
        }
    }
}

template <typename T, int KIND, bool BATCHED>
__global__ void __launch_bounds__(NT, 2) backward_kernel(BwdArgs A) {
    if constexpr (!BATCHED) {
        Grp gp;
        gp.member = blockIdx.x;
        gp.g = gridDim.x;
        gp.sp = Span{0, A.n};
        gp.hdr = A.hdr;
        gp.part = A.part;
        bwd_instance<T, KIND>(A, gp, 0);
        return;
    } else {
        while (true) {
            const Slot sl = next_slot(A.R, A.B);
            if (sl.inst < 0) break;
            const Grp gp = slot_group(A.R, A.offsets, sl);
            if (gp.sp.hi < gp.sp.lo) {
                if (sl.member == 0 && threadIdx.x == 0) {
                    if (A.gr) A.gr[sl.inst] = 0.0;
                    if (A.status) A.status[sl.inst] = CQK_BAD_ARG;
                }
                continue;
            }
            bwd_instance<T, KIND>(A, gp, sl.inst);
        }
    }
}

template <typename T, int KIND>
const void* pick_kernel(bool batched) {
    return batched ? (const void*)backward_kernel<T, KIND, true> : (const void*)backward_kernel<T, KIND, false>;
}

}  // namespace

int launch_backward(int kind, int64_t B, const int64_t* offsets, int64_t n, int dtype, const void* g, const void* x,
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
    if (dtype == CQK_F64) {
        kern = kind == kBwdGeneral ? pick_kernel<double, kBwdGeneral>(batched)
               : kind == kBwdSimplex ? pick_kernel<double, kBwdSimplex>(batched)
                                     : pick_kernel<double, kBwdL1>(batched);
    } else {
        kern = kind == kBwdGeneral ? pick_kernel<float, kBwdGeneral>(batched)
               : kind == kBwdSimplex ? pick_kernel<float, kBwdSimplex>(batched)
                                     : pick_kernel<float, kBwdL1>(batched);
    }
    const int64_t vec = dtype == CQK_F64 ? 2 : 4;
    int grid;
    cudaError_t e;
    if (batched) {
        A.offsets = offsets;
        A.B = B;
        A.R = BatchRefs::at(ws, B);
        grid = persistent_grid(kern, NT, 0, INT64_MAX / 2, o.max_blocks);
        if (grid <= 0) return CQK_CUDA_ERROR;
        if ((int64_t)grid > B * kMaxGroup) grid = (int)(B * kMaxGroup);
        const int64_t per_block = o.group_elems > 0 ? o.group_elems : kBackwardGroupElems;
        const int rc = plan_batch(offsets, B, per_block, grid, ws, s);
        if (rc != CQK_OK) return rc;
    } else {
        A.n = n;
        A.hdr = static_cast<WsHeader*>(ws);
        A.part = reinterpret_cast<double*>(static_cast<char*>(ws) + sizeof(WsHeader));
        grid = persistent_grid(kern, NT, 0, (n + vec - 1) / vec, o.max_blocks);
        if (grid <= 0) return CQK_CUDA_ERROR;
        e = cudaMemsetAsync(ws, 0, sizeof(WsHeader), s);
        if (e != cudaSuccess) {
            set_last_cuda_error(e);
            return CQK_CUDA_ERROR;
        }
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
