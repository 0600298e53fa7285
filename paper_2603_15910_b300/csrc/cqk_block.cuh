// cqk_block.cuh -- streaming loads and deterministic reductions shared by the persistent
// kernels of libcqk.
//
// Work is done by a "group" of co-resident blocks on one element range [lo, hi) of arrays
// that are 16-byte aligned at element 0 (a single solve: one group of all blocks on [0, n);
// a batch: one group per instance on that instance's range of the concatenated arrays).
// Vectors are indexed globally: vector q holds elements q*V ... q*V+V-1, so every 128-bit
// access stays aligned whatever lo is; elements outside [lo, hi) are masked off.
#pragma once

#include "cqk_device.cuh"
#include "cqk_internal.h"

namespace cqk {

template <typename T>
struct VecOf;
template <>
struct VecOf<double> {
    using type = double2;
    static constexpr int V = 2;
};
template <>
struct VecOf<float> {
    using type = float4;
    static constexpr int V = 4;
};

constexpr int NT = kBlockThreads;
constexpr int NWARP = NT / 32;

struct Span {
    int64_t lo, hi;
};

// the vectors [qlo, qhi) that meet the span
template <int V>
__device__ __forceinline__ int64_t span_qlo(const Span& s) { return s.lo / V; }
template <int V>
__device__ __forceinline__ int64_t span_qhi(const Span& s) { return (s.hi + V - 1) / V; }

// One group of blocks working on one span: block `member` of `g`, its barrier / ticket /
// flags header and its per-block partial sums [2][kPartialQ][g].
struct Grp {
    int member, g;
    Span sp;
    WsHeader* hdr;
    double* part;
};

// Barrier of a group at arrival count `target`.  A group of one block needs no device-wide
// arrival counter: a block barrier around a fence by thread 0 orders the partial sums that
// thread 0 wrote before it against the reads after it.  `force_grid` keeps the counter
// (the fault-injection path of the tests).
__device__ __forceinline__ bool group_barrier(const Grp& gp, unsigned target, unsigned long long limit_ns,
                                              bool force_grid) {
    if (gp.g == 1 && !force_grid) {
        __syncthreads();
        if (threadIdx.x == 0) __threadfence();
        __syncthreads();
        return true;
    }
    return grid_barrier(&gp.hdr->bar_count, target, &gp.hdr->error, limit_ns, CQK_TIMEOUT);
}

// Load the V elements of vector q; elements outside the span get ok = false.  One 128-bit
// load when the arrays are 16-byte aligned and the vector lies inside the span.
template <typename T>
__device__ __forceinline__ void load_vec(const T* __restrict__ p, const Span& sp, int64_t q, bool aligned,
                                         T (&v)[VecOf<T>::V], bool (&ok)[VecOf<T>::V]) {
    constexpr int V = VecOf<T>::V;
    const int64_t e0 = q * V;
    if (aligned && e0 >= sp.lo && e0 + V <= sp.hi) {
        using VT = typename VecOf<T>::type;
        VT w = __ldg(reinterpret_cast<const VT*>(p) + q);
        const T* s = reinterpret_cast<const T*>(&w);
#pragma unroll
        for (int j = 0; j < V; j++) {
            v[j] = s[j];
            ok[j] = true;
        }
    } else {
#pragma unroll
        for (int j = 0; j < V; j++) {
            ok[j] = e0 + j >= sp.lo && e0 + j < sp.hi;
            v[j] = ok[j] ? __ldg(p + e0 + j) : T(0);
        }
    }
}
template <typename T>
__device__ __forceinline__ void load_vec(const T* __restrict__ p, int64_t n, int64_t q, bool aligned,
                                         T (&v)[VecOf<T>::V], bool (&ok)[VecOf<T>::V]) {
    load_vec<T>(p, Span{0, n}, q, aligned, v, ok);
}

// Store the elements of vector q that lie inside the span.
template <typename T>
__device__ __forceinline__ void store_vec(T* __restrict__ p, const Span& sp, int64_t q, bool aligned,
                                          const T (&v)[VecOf<T>::V]) {
    constexpr int V = VecOf<T>::V;
    const int64_t e0 = q * V;
    if (aligned && e0 >= sp.lo && e0 + V <= sp.hi) {
        using VT = typename VecOf<T>::type;
        VT w;
        T* s = reinterpret_cast<T*>(&w);
#pragma unroll
        for (int j = 0; j < V; j++) s[j] = v[j];
        reinterpret_cast<VT*>(p)[q] = w;
    } else {
#pragma unroll
        for (int j = 0; j < V; j++)
            if (e0 + j >= sp.lo && e0 + j < sp.hi) p[e0 + j] = v[j];
    }
}

// Free-mask words of a warp's 32 consecutive vectors (starting at vector qw, a multiple of
// 32): bit e % 32 of word e / 32 is set iff sel of element e.  Words that lie entirely inside
// the span are stored; a word shared with a neighbouring span is updated atomically on this
// span's bits only.  Called by all lanes.
template <int V>
__device__ __forceinline__ void store_mask(uint32_t* mask, const Span& sp, int64_t qw, const bool (&sel)[V]) {
    const int lane = threadIdx.x & 31;
    unsigned bitsv = 0;
#pragma unroll
    for (int j = 0; j < V; j++) bitsv |= (sel[j] ? 1u : 0u) << ((lane * V + j) & 31);
    constexpr int LPW = 32 / V;  // lanes per mask word
#pragma unroll
    for (int o = 1; o < LPW; o <<= 1) bitsv |= __shfl_xor_sync(0xffffffffu, bitsv, o);
    if ((lane % LPW) == 0) {
        const int64_t word = (qw * V) / 32 + lane / LPW;
        const int64_t w0 = word * 32;
        if (w0 >= sp.hi || w0 + 32 <= sp.lo) return;
        if (w0 >= sp.lo && w0 + 32 <= sp.hi) {
            mask[word] = bitsv;
        } else {
            const int64_t a = sp.lo > w0 ? sp.lo - w0 : 0, b = sp.hi < w0 + 32 ? sp.hi - w0 : 32;
            const unsigned in = (b >= 32 ? 0xFFFFFFFFu : ((1u << b) - 1u)) & ~((1u << a) - 1u);
            atomicAnd(&mask[word], ~in | bitsv);
            atomicOr(&mask[word], bitsv & in);
        }
    }
}

// The free-mask bits of U consecutive rows of 32 vectors (row u holds the vectors
// base + 32u ... base + 32u + 31, lane L the vector base + 32u + L; base a multiple of 32),
// written as whole words: the U*V words of the rows, word w by lane w, one store per lane
// instead of one shuffle chain and one 4-byte store per row.  Each lane packs its U*V bits
// (bit u*V + j = element j of its vector of row u); the lane of word w gathers its V-bit
// pieces from the 32/V lanes that hold the word's elements.  Words shared with another span
// are merged with atomics on this span's bits.
template <int V, int U>
__device__ __forceinline__ void store_mask_rows(uint32_t* mask, const Span& sp, int64_t base,
                                                const bool (&sel)[U][V]) {
    static_assert(U * V <= 32 && 32 % V == 0, "the rows' words fit one per lane");
    constexpr int LPW = 32 / V;  // lanes per mask word
    constexpr int NW = U * V;    // words of the U rows
    const int lane = threadIdx.x & 31;
    unsigned p = 0;
#pragma unroll
    for (int u = 0; u < U; u++)
#pragma unroll
        for (int j = 0; j < V; j++) p |= (sel[u][j] ? 1u : 0u) << (u * V + j);
    const int ru = lane / V, rk = lane % V;  // this lane's word: row ru, word rk of the row
    const unsigned piece = (1u << V) - 1u;
    unsigned word = 0;
#pragma unroll
    for (int i = 0; i < LPW; i++) {
        const unsigned q = __shfl_sync(0xffffffffu, p, (rk * LPW + i) & 31);
        word |= ((q >> ((ru * V) & 31)) & piece) << (i * V);
    }
    if (lane >= NW) return;
    const int64_t wi = base * V / 32 + lane;  // global word index
    const int64_t w0 = wi * 32;
    if (w0 >= sp.hi || w0 + 32 <= sp.lo) return;
    if (w0 >= sp.lo && w0 + 32 <= sp.hi) {
        mask[wi] = word;
    } else {
        const int64_t a = sp.lo > w0 ? sp.lo - w0 : 0, b = sp.hi < w0 + 32 ? sp.hi - w0 : 32;
        const unsigned in = (b >= 32 ? 0xFFFFFFFFu : ((1u << b) - 1u)) & ~((1u << a) - 1u);
        atomicAnd(&mask[wi], ~in | word);
        atomicOr(&mask[wi], word & in);
    }
}

// Warp-contiguous traversal of the vectors [qlo, qhi) by the warps of a group: iteration i of
// warp w (of W = g * NWARP) covers the vectors [base, base + 32*U) with
// base = floor(qlo/32)*32 + (w + i*W)*32*U, lane L taking base + k*32 + L (k < U), so every
// load instruction of a warp reads 512 contiguous bytes and each lane has U independent
// 16-byte loads in flight.  rev = true visits the same iterations in reverse order: a pass
// that follows a forward pass then starts on the data that the forward pass read last,
// which is still in L2.
struct WarpSweep {
    int64_t first, step, count;
    __device__ __forceinline__ WarpSweep(int64_t qlo, int64_t qhi, int U, int member, int g) {
        const int64_t w = (int64_t)member * NWARP + (threadIdx.x >> 5);
        first = (qlo / 32) * 32 + w * 32 * U;
        step = (int64_t)g * NWARP * 32 * U;
        count = first < qhi ? (qhi - first + step - 1) / step : 0;
    }
    // one warp alone (a warp-level solve): warp index w of W warps
    __device__ __forceinline__ static WarpSweep solo(int64_t qlo, int64_t qhi, int U) {
        WarpSweep s(qlo, qhi, U, 0, 0);
        s.first = (qlo / 32) * 32;
        s.step = (int64_t)32 * U;
        s.count = s.first < qhi ? (qhi - s.first + s.step - 1) / s.step : 0;
        return s;
    }
    __device__ __forceinline__ int64_t base(int64_t i, bool rev) const { return first + (rev ? count - 1 - i : i) * step; }
};

// a[j] for a runtime index j without dynamic register indexing (unrolled selects)
template <typename X, int N>
__device__ __forceinline__ X pick(const X (&a)[N], int j) {
    X v = a[0];
#pragma unroll
    for (int t = 1; t < N; t++) v = (t == j) ? a[t] : v;
    return v;
}
template <typename X, int N, int M>
__device__ __forceinline__ X pick2(const X (&a)[N][M], int uj) {
    X v = a[0][0];
#pragma unroll
    for (int t = 1; t < N * M; t++) v = (t == uj) ? a[t / M][t % M] : v;
    return v;
}
template <typename X, int N>
__device__ __forceinline__ void put(X (&a)[N], int j, X v) {
#pragma unroll
    for (int t = 0; t < N; t++)
        if (t == j) a[t] = v;
}

__device__ __forceinline__ unsigned long long bits_of(double v) { return opaque_bits(v); }

// Combine the per-warp values sh[q][0..NWARP) in warp 0 with a fixed butterfly, so every lane
// of warp 0 ends with the same bits (q == qmax takes the maximum, the others the sum).  Called
// by the threads of warp 0 only.
template <int NQ>
__device__ __forceinline__ void warp0_combine(const double (*sh)[NWARP], int qmax, double (&out)[NQ]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < NQ; q++) out[q] = lane < NWARP ? sh[q][lane] : ((q == qmax) ? -INFINITY : 0.0);
#pragma unroll
    for (int o = NWARP / 2; o > 0; o >>= 1) {
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            const double t = __shfl_xor_sync(0xffffffffu, out[q], o);
            out[q] = (q == qmax) ? fmax(out[q], t) : out[q] + t;
        }
    }
}

// Sum NQ doubles over the block (fixed order); result valid in thread 0.
template <int NQ>
__device__ __forceinline__ void block_sum(double (&v)[NQ], double (*sh)[NWARP]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; q++) v[q] = warp_sum(v[q]);
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NQ; q++) sh[q][wid] = v[q];
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        double t[NQ];
        warp0_combine<NQ>(sh, -1, t);
#pragma unroll
        for (int q = 0; q < NQ; q++) v[q] = t[q];
    }
    __syncthreads();
}

// Sum NQ doubles over the block (fixed order); result valid in thread 0.  Every thread stores
// its values in scr (NQ x NT doubles of shared memory); warp 0 alone adds them, lane l the
// threads l, l + 32, ... in turn, then one butterfly.  The FP64 pipe, the scarce unit of this
// GPU, sees NWARP + 5 adds per value in one warp instead of a 5-level butterfly in every warp
// (at n = 1e4, ~4.5 -> ~1.5 us per Newton pass of the general solve).
template <int NQ>
__device__ __forceinline__ void block_sum_smem(double (&v)[NQ], double* scr) {
#pragma unroll
    for (int q = 0; q < NQ; q++) scr[q * NT + threadIdx.x] = v[q];
    __syncthreads();
    if (threadIdx.x < 32) {
        double t[NQ];
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            t[q] = scr[q * NT + threadIdx.x];
#pragma unroll
            for (int k = 1; k < NWARP; k++) t[q] += scr[q * NT + k * 32 + threadIdx.x];
        }
#pragma unroll
        for (int q = 0; q < NQ; q++) v[q] = warp_sum(t[q]);
    }
    __syncthreads();
}

// Totals of the group's g partials of pass parity `par` (sums, and a max for q == qmax), in
// a fixed order; valid in every lane of warp 0, computed by warp 0 alone (the other threads
// return at once): lane l takes blocks l, l + 32, ... in turn, then a butterfly.  Every block
// computes the same bits.  (Loading the partials with every thread and reducing them with a
// butterfly per warp issued ~8x the FP64 instructions, and the FP64 pipe is the scarce unit
// on this GPU.)
template <int NQ>
__device__ __forceinline__ void grid_totals_warp0(const double* part, int g, int par, int qmax, double (&out)[NQ],
                                                  double (*sh)[NWARP]) {
    (void)sh;
    if (threadIdx.x >= 32) return;
    double v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; q++) v[q] = (q == qmax) ? -INFINITY : 0.0;
#pragma unroll 4
    for (int b = threadIdx.x; b < g; b += 32) {
        double t[NQ];
#pragma unroll
        for (int q = 0; q < NQ; q++) t[q] = ld_cg(part + ((size_t)par * kPartialQ + q) * g + b);
#pragma unroll
        for (int q = 0; q < NQ; q++) v[q] = (q == qmax) ? fmax(v[q], t[q]) : v[q] + t[q];
    }
#pragma unroll
    for (int q = 0; q < NQ; q++) out[q] = (q == qmax) ? warp_max(v[q]) : warp_sum(v[q]);
}

// Reduce the partials of the group's g blocks for pass parity `par` (sums, and a max for
// q == qmax); every block computes the same values in the same order.  Result in out[] (all
// threads).
template <int NQ>
__device__ __forceinline__ void grid_reduce(const double* part, int g, int par, int qmax, double (&out)[NQ],
                                            double (*sh)[NWARP], double* bc) {
    double t[NQ];
    grid_totals_warp0<NQ>(part, g, par, qmax, t, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NQ; q++) bc[q] = t[q];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NQ; q++) out[q] = bc[q];
    __syncthreads();
}

template <int NQ>
__device__ __forceinline__ void write_partials(double* part, int member, int g, int par, const double (&v)[NQ]) {
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NQ; q++) part[((size_t)par * kPartialQ + q) * g + member] = v[q];
    }
}

// Last-block-done reduction of NQ <= 3 sums stored in slots 5..5+NQ of parity 0; returns
// true in the group's last block, whose out[] then holds the group sums (thread 0).
template <int NQ>
__device__ __forceinline__ bool last_block_sums(double* part, int member, int g, unsigned* ticket, double (&v)[NQ],
                                                double (&out)[NQ], double (*sh)[NWARP]) {
    __shared__ unsigned s_last;
    block_sum<NQ>(v, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NQ; q++) part[(size_t)(5 + q) * g + member] = v[q];
        __threadfence();
        unsigned t = atomicAdd(ticket, 1u);
        s_last = (t == (unsigned)g - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    double w[NQ];
#pragma unroll
    for (int q = 0; q < NQ; q++) w[q] = 0.0;
    for (int b = threadIdx.x; b < g; b += NT)
#pragma unroll
        for (int q = 0; q < NQ; q++) w[q] += ld_cg(part + (size_t)(5 + q) * g + b);
    block_sum<NQ>(w, sh);
#pragma unroll
    for (int q = 0; q < NQ; q++) out[q] = w[q];
    return true;
}

}  // namespace cqk
