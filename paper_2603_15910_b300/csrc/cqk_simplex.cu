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
//                    CQK_INIT_CONDAT   Alg. 2 on every chunk of a partition by tiles (exact,
//                                      see condat_block); lambda_0 from eq. (lambdaJ) on
//                                      the union of the J's (Sec. 4)
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
#include "cqk_stage.cuh"

namespace cqk {
namespace {

// 16-byte vectors in flight per lane in the streaming passes (half-unroll build: 4)
#ifdef CQK_UNROLL_HALF
constexpr int kStreamU = 4;
#else
constexpr int kStreamU = 8;
#endif
static_assert(NT == 256, "the pipelined Alg. 2 start gives its 8 warps fixed roles");


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
    int scan_warps;        // chunks (scan warps) per block of the pipelined start; 0 = automatic
    const void* xbar;      // CQK_INIT_WARM: primal estimate
    WsHeader* hdr;
    double* part;  // [2][kPartialQ][gridDim.x]
};

// ---- sum and max of y (l1: |y|) and the NaN check, accumulated per element -----------------
// FP64 data: values in the df operating range go to a lazily normalised float pair that is
// folded into FP64 once per tile or sweep; others are added in FP64 (one trip per element).
// FP32 data: a double-float sum.  The maximum is kept as an order key (integer pipe).
struct SumAcc {
    df acc;
    LazyDf lz;
    double acc64, acc_wide;
    long long mxk;
    float mxf;
    bool bad;
    __device__ void init() {
        acc = df_make(0.0f);
        lz = LazyDf{0.0f, 0.0f};
        acc64 = acc_wide = 0.0;
        mxk = order_key(-INFINITY);
        mxf = -INFINITY;
        bad = false;
    }
    __device__ void fold() {
        acc64 += df_to_f64_int(df{lz.hi, lz.lo});
        lz = LazyDf{0.0f, 0.0f};
    }
    __device__ double sum() const { return df_to_f64_int_all(acc) + acc64 + df_to_f64_int(df{lz.hi, lz.lo}) + acc_wide; }
};

// one element; returns true when an FP64 value lies outside the df range (the caller adds it
// with sum_wide)
template <typename T, bool L1>
__device__ __forceinline__ bool sum_elem(SumAcc& a, T v) {
    if constexpr (sizeof(T) == 8) {
        const double t = L1 ? __longlong_as_double((long long)(bits_of(v) & 0x7FFFFFFFFFFFFFFFull)) : (double)v;
        const bool inr = df_in_range(t, false);
        const df st = split_f64_finite(t);
        lazy_add(a.lz, df{inr ? st.hi : 0.0f, inr ? st.lo : 0.0f});
        a.bad |= f64_is_nan(t);
        const long long kk = order_key(t);
        a.mxk = kk > a.mxk ? kk : a.mxk;
        return !inr;
    } else {
        const float t = L1 ? fabsf((float)v) : (float)v;
        a.acc = df_add_f(a.acc, t);
        a.bad |= (t != t);
        a.mxf = fmaxf(a.mxf, t);
        return false;
    }
}
template <typename T, bool L1>
__device__ __forceinline__ void sum_wide(SumAcc& a, T v) {
    a.acc_wide += L1 ? fabs((double)v) : (double)v;
}
template <typename T>
__device__ __forceinline__ double sum_max(const SumAcc& a) {
    if constexpr (sizeof(T) == 8) return from_order_key(a.mxk);
    else return (double)a.mxf;
}

// ---- Alg. 2 per chunk ---------------------------------------------------------------------
// Tile c holds elements [c*TILE, (c+1)*TILE) (16 KB); the span's tiles are dealt round robin to
// the chunks (W = blocks x scan warps per block), and each chunk is scanned in increasing index
// order.  The tiles stream into shared memory by bulk copies (kCondatStages stages, bounded
// waits).
//
// Exactness: both branches of the first loop of Alg. 2 lower lambda (adding j with
// y_j + lambda > 0 gives lambda - (y_j + lambda)/(|J|+1); a restart gives r - y_j, below the
// rejected lambda_{J u {j}}), so once J is started an element that fails the test fails it
// for the rest of the scan.  A filter with any threshold the scan has already reached
// therefore passes a superset of the elements the scan can accept: the filter warps test each
// tile against the threshold the chunk's scan last published, and the chunk's scan warp runs
// the sequential scan over the passing elements only, in index order, testing each against
// the lambda current when it is reached, and publishes the new threshold.  (A block chunk of
// kSplitTiles tiles or more gives the walk over the passing elements and the scan to two
// warps joined by a queue in index order; the scan is the same.)  Before J is started every
// element passes (the first element of the chunk starts J unconditionally).  The final loop of Alg. 2 over J~ visits, in order, the elements
// of J~ that pass the test with the current lambda.  J~ is the set of values accepted before
// the last restart; the scan warp keeps every accepted value in acceptance (= index) order, so
// the loop runs over that list.  When J~ outgrows the list, the loop is a re-scan of the chunk
// prefix before the last restart with the same test instead: every element there that is
// not in J~ failed the test with a larger lambda and fails it again.
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

constexpr int kCondatStages = 5;
template <typename T>
__host__ __device__ constexpr int condat_tile() { return 16384 / (int)sizeof(T); }  // elements per tile
constexpr size_t kCondatSmem = (size_t)kCondatStages * 16384;                      // dynamic shared memory
constexpr int kJList = 1024;  // accepted values kept for the final loop
constexpr int kStartBit = 16;  // bit of the first start barrier's phase in the ring parity word
constexpr int kMaxScan = 4;    // scan warps (chunks) per block in the pipelined Alg. 2

constexpr int kQueue = 128;     // survivors queued between the walking and the taking warp
constexpr int kSplitTiles = 64; // tiles of a block's chunk from which the scan is split in two

struct CondatShared {
    unsigned msk[NWARP][16];  // filter ballots of each warp, (k, j) -> bit lane
    unsigned pmsk[kCondatStages][32 * 4];  // pipelined filter: ballots of group g, (g, j) -> bit lane
    double list[kJList];
    unsigned long long tb[kMaxScan];  // the published test thresholds (FP64 data: bit patterns)
    float trd[kMaxScan];              // (FP32 data)
    // one chunk per block: the survivors in index order, written by the walking warp (values
    // as the scan uses them, element indices), taken by the scanning warp; counters only grow
    double qv[kQueue];
    long long qe[kQueue];
    unsigned qtail, qhead, qdone, qabort;
    long long qklo;  // the scan's current klo (certain failures are not queued)
};

__device__ __forceinline__ unsigned ld_acquire_cta(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.cta.shared::cta.b32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_cta(unsigned* p, unsigned v) {
    asm volatile("st.release.cta.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v) : "memory");
}

// ---- the scalar recurrence of Alg. 2 --------------------------------------------------------
// The scan is one long dependency chain (lambda_{k+1} from lambda_k) run by one warp, so its
// cost is the latency and the instruction count of one step.  The scan's own FP64 operations
// are kept except the division: S (the sum of J in scan order), r - S and t = (r - S) - y are
// formed exactly as the sequential scan forms them, and lambda = fl(t / (|J|+1)) is replaced
// by the product t * w with w within 2^-46 of 1/(|J|+1) (a float reciprocal and one Newton
// correction, formed while the previous step runs), which lies within kLamUlps units in the
// last place of the scan's quotient (2^-46 + 2^-52 relative, at most ~2^8 units across a
// binade boundary).  Every decision of the scan — y > -lambda (l1: |y| > max{0, -lambda}) and
// the restart test lambda < r - y — is taken from the product when it holds for every value
// within kLamUlps units of it (integer compares of order keys), and from the exact quotient
// otherwise (out of line, rare).  The decisions, hence J, J~, |J| and S, are those of the
// FP64 scan.  The test thresholds are kept as order keys (klo, khi): v > c for every c within
// the margin iff key(v) > khi, and v <= c for all of them iff key(v) <= klo, since for any two
// bit patterns v > c (FP64, c != -0) iff key(v) > key(c).  On the critical path of one step
// are then two FP64 operations (t, then the product) and a few integer ones; S + y and
// r - (S + y) are formed beside them, before the decision.  (A double-float version of the
// step measured ~800 cycles in one warp, an FP64 one with a correctly rounded reciprocal
// ~1160.)
constexpr long long kLamUlps = 512;
constexpr long long kKeyNegInf = -0x7FF0000000000000ll - 1;  // order_key(-inf)
constexpr long long kKeyPosInf = 0x7FF0000000000000ll;       // order_key(+inf)

struct CondatState {
    double S;     // the FP64 sum of J in scan order
    double rmS;   // fl(r - S)
    long long nJ;
    int64_t rs;   // index of the last restart
    double w1;    // ~1/(|J|+1) (relative error below 2^-46; |J|+1 < 2^24)
    // the scan's lambda is fl(t / en) (en > 0) or t itself (en == 0); lk = order key of the
    // approximation, within kLamUlps of the key of lambda (exact when en == 0)
    double t;
    long long en, lk;
    long long klo, khi;  // key(v) <= klo: v certainly fails; key(v) > khi: certainly passes
    double* list;  // accepted values in acceptance order (the first cap of them)
    int cap, cnt, jt_end;
};

__device__ __forceinline__ void condat_init(CondatState& st, double* list, int cap) {
    st.S = 0.0;
    st.rmS = 0.0;
    st.nJ = 0;
    st.rs = -1;
    st.w1 = 1.0;
    st.t = 0.0;
    st.en = 0;
    st.lk = 0;
    st.klo = kKeyNegInf;  // before J starts every element passes
    st.khi = kKeyNegInf;
    st.list = list;
    st.cap = cap;
    st.cnt = 0;
    st.jt_end = 0;
}

// 1/k correctly rounded for 1 <= k < kRecipN (entry 0 unused), folded by the compiler from
// IEEE division; read with a warp-uniform index (constant cache broadcast)
constexpr int kRecipN = 4096;
struct RecipTable {
    double v[kRecipN];
    constexpr RecipTable() : v() {
        for (int k = 1; k < kRecipN; k++) v[k] = 1.0 / (double)k;
    }
};
__constant__ RecipTable kRecip = RecipTable();

// ~1/n for 1 <= n < 2^24 (relative error below 2^-46): the table, else the float reciprocal
// and one Newton correction as a double (the float parts converted on the integer pipe)
__device__ __forceinline__ double condat_recip(long long n) {
    if (n < kRecipN) return kRecip.v[n];
    const float nf = (float)(int)n;
    const float r0 = __frcp_rn(nf);
    const float e0 = fmaf(-nf, r0, 1.0f);
    return f32_to_f64_bits(r0) + f32_to_f64_bits(__fmul_rn(r0, e0));
}

// the keys of the test thresholds from the key of lambda, +-m keys (l1: c = max{0, -lambda});
// the key -1 (c = -0) becomes the key of +0, as FP64 compares
template <bool L1>
__device__ __forceinline__ void condat_thresholds(CondatState& st, long long m) {
    // c = -lambda: key(-x) = -key(x) - 1; the larger keys of lambda give the smaller c
    long long klo = -(st.lk + m) - 1, khi = -(st.lk - m) - 1;
    if (L1) {
        klo = klo < 0 ? 0 : klo;
        khi = khi < 0 ? 0 : khi;
    } else {
        klo = klo == -1 ? 0 : klo;
        khi = khi == -1 ? 0 : khi;
    }
    st.klo = klo;
    st.khi = khi;
}

// the bit pattern of the threshold klo (a GtThreshold for the block filters)
__device__ __forceinline__ unsigned long long condat_lo_bits(const CondatState& st) {
    const long long k = st.klo;
    return k >= 0 ? (unsigned long long)k : 0x8000000000000000ull - (unsigned long long)(k + 1);
}

// the approximation's neighbourhood stays inside the finite range (else FP64 decides)
__device__ __forceinline__ bool condat_lam_ok(double lam_approx) {
    return ((hi_word(lam_approx) >> 20) & 0x7FFu) < 0x7FEu;
}

// lambda of the current (t, en) and its thresholds
template <bool L1>
__device__ __forceinline__ void condat_set_lambda(CondatState& st, double lam_approx) {
    st.lk = order_key(lam_approx);
    if (st.en == 0) {
        condat_thresholds<L1>(st, 0);
    } else if (!condat_lam_ok(lam_approx) || st.en >= (1ll << 24)) {  // no certain decision
        st.klo = kKeyNegInf;
        st.khi = kKeyPosInf;
    } else {
        condat_thresholds<L1>(st, kLamUlps);
    }
}

// The exact FP64 decisions, out of line: inlined, the compiler evaluates the FP64 division
// speculatively on every test.
template <bool L1>
__device__ __noinline__ bool condat_exact_gt(unsigned long long vb, double t, long long en) {
    const double le = en == 0 ? t : t / (double)en;
    unsigned long long cb = opaque_bits(le) ^ 0x8000000000000000ull;
    if (L1 && (cb >> 63)) cb = 0ull;
    return gt_bits(vb, make_gt(__longlong_as_double((long long)cb)));
}
__device__ __noinline__ bool condat_exact_less(double t, long long en, double rmy) {
    return t / (double)en < rmy;
}

// the test v > c(lambda) of the FP64 scan (v = y_j, l1: |y_j|)
template <bool L1>
__device__ __forceinline__ bool condat_gt(double v, const CondatState& st, double r) {
    const long long kv = order_key(v);
    if (kv > st.khi) return true;
    if (kv <= st.klo) return false;
    return condat_exact_gt<L1>(opaque_bits(v), st.t, st.en);  // rare
}

__device__ __forceinline__ void condat_record(CondatState& st, double v) {
    if ((threadIdx.x & 31) == 0 && st.cnt < st.cap) st.list[st.cnt] = v;
    st.cnt++;
}

// J <- {y} (the first element of the chunk, or a restart): lambda = r - y exactly
template <bool L1>
__device__ __forceinline__ void condat_start_j(CondatState& st, double r, double y) {
    st.S = y;
    st.rmS = r - y;
    st.nJ = 1;
    st.w1 = 0.5;
    st.t = st.rmS;
    st.en = 0;
    condat_set_lambda<L1>(st, st.rmS);
    st.jt_end = st.cnt;
}

// one element taken by the first loop of Alg. 2 (J started): add it or restart with it
template <bool L1>
__device__ __forceinline__ void condat_take(CondatState& st, double r, double y, int64_t e) {
    const double t = st.rmS - y;
    const double lam = t * st.w1;
    const double rmy = r - y;
    const double S1 = st.S + y;  // the addition's S and r - S, beside the decision
    const double rmS1 = r - S1;
    const double w2 = condat_recip(st.nJ + 2);  // for the step after an addition
    const long long lk = order_key(lam), ky = order_key(rmy);
    // restart test lambda < r - y, from the approximation unless within its uncertainty
    const bool sure = condat_lam_ok(lam) && st.nJ + 1 < (1ll << 24);
    bool acc;
    if (sure && lk + kLamUlps < ky) acc = true;
    else if (sure && lk - kLamUlps >= ky) acc = false;
    else acc = condat_exact_less(t, st.nJ + 1, rmy);  // rare
    if (acc) {
        st.S = S1;
        st.rmS = rmS1;
        st.nJ += 1;
        st.w1 = w2;
        st.t = t;
        st.en = st.nJ;
        condat_set_lambda<L1>(st, lam);
    } else {  // restart: J~ <- J~ u J, J <- {j}
        st.rs = e;
        condat_start_j<L1>(st, r, y);
    }
    condat_record(st, y);
}

// the final loop of Alg. 2: J <- J u {y} (no restart test)
template <bool L1>
__device__ __forceinline__ void condat_add(CondatState& st, double r, double y) {
    const double t = st.rmS - y;
    const double lam = t * st.w1;
    st.S += y;
    st.rmS = r - st.S;
    st.nJ += 1;
    st.w1 = condat_recip(st.nJ + 1);
    st.t = t;
    st.en = st.nJ;
    condat_set_lambda<L1>(st, lam);
}

// the block filter's threshold for FP32 data: a float at or below every c the scan can still
// use (the FP64 data take the bit pattern of klo)
__device__ __forceinline__ float condat_filter_rd(const CondatState& st) {
    return __double2float_rd(__longlong_as_double((long long)condat_lo_bits(st)));
}

// The next survivor in index order (lane, j) of the masks m[j] (warp-uniform): its lane and
// j, and the bit cleared; false when none is left.
template <int V>
__device__ __forceinline__ bool condat_next(unsigned (&m)[V], int& L, int& jn) {
    unsigned any = 0;
#pragma unroll
    for (int j = 0; j < V; j++) any |= m[j];
    if (!any) return false;
    L = __ffs(any) - 1;
    jn = 0;
#pragma unroll
    for (int j = V - 1; j >= 0; j--)
        if ((m[j] >> L) & 1u) jn = j;
#pragma unroll
    for (int j = 0; j < V; j++)
        if (j == jn) m[j] &= m[j] - 1u;  // L is the lowest bit of m[jn]
    return true;
}

// Warp 0: the first loop of Alg. 2 over one group of 32 vectors in index order (lane, j);
// okv marks the elements that passed the block's filter.  The survivors of the test against
// the lambda of the group's start are visited in order, each tested again against the lambda
// current when it is reached (c(lambda) only grows, so this is the scan's own test), with the
// next survivor's value fetched while the current step runs.
template <typename T, bool L1>
__device__ __forceinline__ void condat_slab(const T (&vals)[VecOf<T>::V], const bool (&okv)[VecOf<T>::V],
                                            int64_t eidx0, double r, CondatState& st) {
    constexpr int V = VecOf<T>::V;
    const int lane = threadIdx.x & 31;
    const int64_t e0 = eidx0 - (int64_t)lane * V;  // element (lane, j) of the group is e0 + lane*V + j
    double av[V];
#pragma unroll
    for (int j = 0; j < V; j++) {
        const double dv = (double)vals[j];
        av[j] = L1 ? __longlong_as_double((long long)(opaque_bits(dv) & 0x7FFFFFFFFFFFFFFFull)) : dv;
    }
    unsigned m[V];
    if (st.nJ == 0) {
        // the first element of the chunk starts J unconditionally (first line of Alg. 2)
#pragma unroll
        for (int j = 0; j < V; j++) m[j] = __ballot_sync(0xffffffffu, okv[j]);
        int L0, j0;
        if (!condat_next<V>(m, L0, j0)) return;
        const double y0 = __shfl_sync(0xffffffffu, pick(av, j0), L0);
        st.rs = e0 + L0 * V + j0;
        condat_start_j<L1>(st, r, y0);
        condat_record(st, y0);
#pragma unroll
        for (int j = 0; j < V; j++) {
            const bool after = (lane > L0) || (lane == L0 && j > j0);
            m[j] = __ballot_sync(0xffffffffu, okv[j] && after && condat_gt<L1>(av[j], st, r));
        }
    } else {
#pragma unroll
        for (int j = 0; j < V; j++) m[j] = __ballot_sync(0xffffffffu, okv[j] && condat_gt<L1>(av[j], st, r));
    }
    int L, jn;
    bool have = condat_next<V>(m, L, jn);
    double v = 0.0;
    if (have) v = __shfl_sync(0xffffffffu, pick(av, jn), L);
    while (have) {
        const int64_t e = e0 + L * V + jn;
        const double y = v;
        have = condat_next<V>(m, L, jn);
        if (have) v = __shfl_sync(0xffffffffu, pick(av, jn), L);
        if (condat_gt<L1>(y, st, r)) condat_take<L1>(st, r, y, e);
    }
}

// The scan warp over one whole staged tile, group by group in index order (bit lane of
// mk[g*V + j] = the filters' result for element (g*32 + lane)*V + j of the tile).  A group with
// many survivors (the tiles filtered before J had a threshold) goes through condat_slab, whose
// lanes test the whole group at once; the few survivors of any other group are visited one
// by one, their values loaded from the stage by every lane (one address) and tested against
// the lambda current when each is reached (the first one of the chunk starts J).  ebase =
// index of the tile's first element.
constexpr int kScanSparse = 4;  // survivors of a group visited one by one
template <typename T, bool L1>
__device__ __forceinline__ void condat_scan_tile(const T* stage, const unsigned* mk, unsigned groups, int64_t ebase,
                                                 double r, CondatState& st) {
    constexpr int V = VecOf<T>::V;
    const int lane = threadIdx.x & 31;
    for (unsigned gs = groups; gs; gs &= gs - 1) {
        const int gi = __ffs(gs) - 1;
        unsigned m[V];
        int cnt = 0;
#pragma unroll
        for (int j = 0; j < V; j++) {
            m[j] = mk[gi * V + j];
            cnt += __popc(m[j]);
        }
        if (cnt > kScanSparse) {
            using VT = typename VecOf<T>::type;
            const VT w = reinterpret_cast<const VT*>(stage)[gi * 32 + lane];
            T v[V];
            bool ok[V];
#pragma unroll
            for (int j = 0; j < V; j++) {
                v[j] = reinterpret_cast<const T*>(&w)[j];
                ok[j] = ((m[j] >> lane) & 1u) != 0u;
            }
            condat_slab<T, L1>(v, ok, ebase + (int64_t)(gi * 32 + lane) * V, r, st);
            continue;
        }
        int L, j;
        while (condat_next<V>(m, L, j)) {
            const int q = gi * 32 + L;
            const int64_t e = ebase + (int64_t)q * V + j;
            double y = (double)stage[q * V + j];
            if (L1) y = __longlong_as_double((long long)(opaque_bits(y) & 0x7FFFFFFFFFFFFFFFull));
            if (st.nJ == 0) {  // the first element of the chunk starts J (first line of Alg. 2)
                st.rs = e;
                condat_start_j<L1>(st, r, y);
                condat_record(st, y);
            } else if (condat_gt<L1>(y, st, r)) {
                condat_take<L1>(st, r, y, e);
            }
        }
    }
}

// warp 0: the final loop of Alg. 2 over the first n entries of the J~ list, 32 at a time: every
// lane tests its entry against the current lambda, and the passing entries are visited in list
// order, each tested again when it is reached (an addition only raises c(lambda), so an entry
// that fails stays out)
template <bool L1>
__device__ __forceinline__ void condat_final_list(const double* list, int n, double r, CondatState& st) {
    const int lane = threadIdx.x & 31;
    for (int base = 0; base < n; base += 32) {
        const int e = base + lane;
        const double val = e < n ? list[e] : 0.0;
        unsigned m[1] = {__ballot_sync(0xffffffffu, e < n && condat_gt<L1>(val, st, r))};
        int L, j0;
        bool have = condat_next<1>(m, L, j0);
        double v = 0.0;
        if (have) v = __shfl_sync(0xffffffffu, val, L);
        while (have) {
            const double y = v;
            have = condat_next<1>(m, L, j0);
            if (have) v = __shfl_sync(0xffffffffu, val, L);
            if (condat_gt<L1>(y, st, r)) condat_add<L1>(st, r, y);
        }
    }
}

// warp 0, J~ outgrew the list: the final loop of Alg. 2 as a re-scan of one slab (32 vectors)
// of the chunk prefix before the last restart
template <typename T, bool L1>
__device__ __forceinline__ void condat_rescan_slab(const T (&vals)[VecOf<T>::V], const bool (&okv)[VecOf<T>::V],
                                                   int64_t eidx0, double r, CondatState& st) {
    constexpr int V = VecOf<T>::V;
    const int lane = threadIdx.x & 31;
    double av[V];
#pragma unroll
    for (int j = 0; j < V; j++) {
        const double dv = (double)vals[j];
        av[j] = L1 ? __longlong_as_double((long long)(opaque_bits(dv) & 0x7FFFFFFFFFFFFFFFull)) : dv;
    }
    bool pass[V];
#pragma unroll
    for (int j = 0; j < V; j++) pass[j] = okv[j] && (eidx0 + j < st.rs) && condat_gt<L1>(av[j], st, r);
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
        const double yv = __shfl_sync(0xffffffffu, pick(av, jf), Lf);
        condat_add<L1>(st, r, yv);
#pragma unroll
        for (int j = 0; j < V; j++) {
            const bool after = (lane > Lf) || (lane == Lf && j > jf);
            pass[j] = pass[j] && after && condat_gt<L1>(av[j], st, r);
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

// the V values of tile vector ql (from the stage when the bulk copy delivered it, else directly)
template <typename T>
__device__ __forceinline__ void tile_vec(const T* __restrict__ y, const Span& sp, const T* stage, bool staged,
                                         int64_t c, int ql, int64_t sb0, int64_t sb1, T (&v)[VecOf<T>::V],
                                         bool (&ok)[VecOf<T>::V]) {
    constexpr int V = VecOf<T>::V;
    constexpr int TT = condat_tile<T>();
    using VT = typename VecOf<T>::type;
    const int64_t q = c * (TT / V) + ql;
    if (staged && q * V >= sb0 && (q + 1) * V <= sb1) {
        const VT w = reinterpret_cast<const VT*>(stage)[ql];
#pragma unroll
        for (int j = 0; j < V; j++) {
            v[j] = reinterpret_cast<const T*>(&w)[j];
            ok[j] = true;
        }
    } else {
        load_vec<T>(y, sp, q, false, v, ok);
    }
}

// The block filter of one tile against the published threshold (tb: the exact 64-bit
// test of FP64 data; trd: FP32 data): the ballots of the passing elements go to s.msk, and
// the NaN check of the data rides along into sacc.bad.  Returns whether this thread's elements
// passed.
template <typename T, bool L1>
__device__ __forceinline__ bool condat_filter_exact(const T* __restrict__ y, const T* __restrict__ xb,
                                                    const Span& sp, bool aligned, const T* stage, bool staged,
                                                    int64_t c, int64_t sb0, int64_t sb1, CondatShared& s,
                                                    SumAcc& sacc) {
    constexpr int V = VecOf<T>::V;
    constexpr int TT = condat_tile<T>();
    constexpr int KC = TT / V / NT;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const GtThreshold g{s.tb[0], (s.tb[0] >> 63) != 0ull};
    const float rd = s.trd[0];
    bool anyp = false;
#pragma unroll
    for (int k = 0; k < KC; k++) {
        const int ql = k * NT + (int)threadIdx.x;
        T v[V];
        bool ok[V];
        tile_vec<T>(y, sp, stage, staged, c, ql, sb0, sb1, v, ok);
#pragma unroll
        for (int j = 0; j < V; j++) {
            if constexpr (sizeof(T) == 8) sacc.bad |= ok[j] && u64_is_nan(bits_of((double)v[j]));
            else sacc.bad |= ok[j] && (v[j] != v[j]);
        }
        support_mask<T, L1>(xb, sp, c * (TT / V) + ql, aligned, ok);
#pragma unroll
        for (int j = 0; j < V; j++) {
            const bool p = ok[j] && condat_test<T, L1>(v[j], g, rd);
            const unsigned bal = __ballot_sync(0xffffffffu, p);
            if (lane == 0) s.msk[wid][k * V + j] = bal;
            anyp |= p;
        }
    }
    return anyp;
}

// A cheaper test of one vector of a tile in the stage: whether it holds an element that may
// pass the exact filter.  FP64 data: the high words alone (y > c implies hi(y) >= hi(c) as
// signed words for c >= 0, hi(y) <= hi(c) as unsigned words for c < 0), and a NaN always
// passes (so that the exact filter, which checks for NaN, sees it); FP32 data: the unordered
// comparison (a NaN passes).  A superset of the exact filter, so a tile it rejects has no
// element the scan can accept.
template <typename T, bool L1>
__device__ __forceinline__ bool condat_prefilter(const T* stage, const T* __restrict__ xb, const Span& sp,
                                                 int64_t c, int ql, bool aligned, unsigned long long tb, float trd) {
    constexpr int V = VecOf<T>::V;
    constexpr int TT = condat_tile<T>();
    const uint4 w = reinterpret_cast<const uint4*>(stage)[ql];
    bool ok[V];
#pragma unroll
    for (int j = 0; j < V; j++) ok[j] = true;
    support_mask<T, L1>(xb, sp, c * (TT / V) + ql, aligned, ok);
    bool p = false;
    if constexpr (sizeof(T) == 8) {
        const unsigned th = (unsigned)(tb >> 32);
        const bool tneg = (tb >> 63) != 0ull;
        const unsigned h[2] = {w.y, w.w};
#pragma unroll
        for (int j = 0; j < 2; j++) {
            bool q;
            if (L1) q = (int)(h[j] & 0x7FFFFFFFu) >= (int)th;  // |y|: a NaN has the largest word
            else if (!tneg) q = ((int)h[j] >= (int)th) | (h[j] >= 0xFFF00000u);
            else q = (h[j] <= th) | (h[j] >= 0xFFF00000u);
            p |= ok[j] && q;
        }
    } else {
        const unsigned u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int j = 0; j < 4; j++) {
            float f = __uint_as_float(u[j]);
            if (L1) f = fabsf(f);
            p |= ok[j] && !(f <= trd);
        }
    }
    return p;
}

// Alg. 2 on the chunks of block `member` of `nchunk` (blocks with member >= nchunk have none):
// the block's tiles i = 0, 1, ... (tile member + i*nchunk of the span) are dealt to nscan
// chunks, tile i to chunk i mod nscan, so that chunk k of block m is chunk m + nchunk*k of a
// partition into nchunk*nscan chunks by tiles taken round robin.  Called by all threads;
// (S_out, nJ_out) = (sum_J y, |J|) of each chunk, valid in lane 0 of scan warp k (zero
// elsewhere); the NaN check of the data rides on this pass, into sacc.bad.
template <typename T, bool L1>
__device__ void condat_block(const T* __restrict__ y, const T* __restrict__ xb, const Span& sp, bool aligned,
                             double r, int member, int nchunk, int nscan, T* smem, uint64_t* bars, unsigned& parity,
                             int* err, unsigned long long limit_ns, bool qfault, SumAcc& sacc, double& S_out,
                             long long& nJ_out) {
    constexpr int V = VecOf<T>::V;
    constexpr int TT = condat_tile<T>();
    constexpr int KC = TT / V / NT;
    constexpr int S = kCondatStages;
    static_assert(KC * V * NT == TT && KC * V <= 16, "tile layout");
    __shared__ CondatShared s;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const bool staged = aligned;
    if (!staged) nscan = 1;
    const int cap = kJList / nscan;
    CondatState st;
    condat_init(st, s.list + (wid < nscan ? wid : 0) * cap, cap);
    if (threadIdx.x < kMaxScan) {  // before J starts every element passes the filter
        s.tb[threadIdx.x] = make_gt(-INFINITY).bits;  // the sign bit of the pattern is the sign of the threshold
        s.trd[threadIdx.x] = -INFINITY;
    }
    if (threadIdx.x == 0) {
        s.qtail = s.qhead = s.qdone = s.qabort = 0u;
        s.qklo = kKeyNegInf;
    }
    TileRing<T, 1, TT> ring;
    ring.setup(sp.lo, sp.hi, smem, bars, member, nchunk);
    if (member >= nchunk) ring.count = 0;
    ring.parity = parity;
    const T* src[1] = {y};
    __syncthreads();
    if (staged) {
        // Pipelined: warps nscan..NWARP-1 filter the tiles as they land and signal the stage's
        // second mbarrier; scan warp k runs the scan of chunk k over the groups with survivors
        // of its tiles, then refills the stage it is done with.  The filters read the threshold
        // that chunk's scan last published, which can only be lower than the scan's own
        // (c(lambda) only grows during the first loop), so they pass a superset.
        constexpr int NVEC = TT / V;  // vectors of a tile
        constexpr int NG = NVEC / 32;  // groups of 32 vectors, in index order
        static_assert(NG == 32 && V <= 32 && kMaxScan < S, "one lane per group; a scan warp steps by less than the ring");
        // one chunk per block of at least kSplitTiles tiles: warp 1 walks the tiles after the
        // first (survivors into the queue, refills), warp 0 scans the first tile, then takes the
        // queued survivors (shorter chunks keep seven filters)
        const bool split = nscan == 1 && ring.count >= kSplitTiles;
        const int nfw = split ? 2 : nscan;  // warps before the filters
        const int NP = NWARP - nfw;         // filtering warps; group g belongs to filter g % NP
        uint64_t* fullb = bars + S;
        uint64_t* startb = bars + 2 * S;  // [k]: scan k is done with its first tile
        const unsigned base = ring.parity;
        if (threadIdx.x == 0)
            for (int k = 0; k < S; k++)
                if (k < ring.count) ring.issue(ring.tile(k, false), k, src);
        if (wid >= nfw) {
            const int pw = wid - nfw;
            // stage, chunk and phase parities advance with i (no divisions in the loop)
            int stg = 0, k = 0;
            unsigned phs = base;  // bit s: parity of stage s's next phase
            for (int64_t i = 0; i < ring.count; i++, stg = stg + 1 == S ? 0 : stg + 1, k = k + 1 == nscan ? 0 : k + 1) {
                const unsigned ph = (phs >> stg) & 1u;
                phs ^= 1u << stg;
                // before J starts every element passes: the filters wait for the threshold of
                // chunk k's first tile before filtering its second
                if (i >= nscan && i < 2 * nscan)
                    mbar_wait(&startb[k], (base >> (kStartBit + k)) & 1u, err, limit_ns, CQK_TIMEOUT);
                mbar_wait(&ring.bar[stg], ph, err, limit_ns, CQK_TIMEOUT);
                const int64_t c = ring.tile(i, false);
                const int64_t sb0 = ring.b0(c), sb1 = ring.b1(c);
                const T* stage = ring.stage(stg, 0);
                const unsigned long long tb = *reinterpret_cast<volatile unsigned long long*>(&s.tb[k]);
                const float trd = *reinterpret_cast<volatile float*>(&s.trd[k]);
                bool may = !(sb0 == c * TT && sb1 == (c + 1) * TT);  // a partial tile: exact filter
                if (!may)
                    for (int gi = pw; gi < NG; gi += NP)
                        may |= condat_prefilter<T, L1>(stage, xb, sp, c, gi * 32 + lane, aligned, tb, trd);
                unsigned* mk = s.pmsk[stg];
                if (__any_sync(0xffffffffu, may)) {
                    const GtThreshold g{tb, (tb >> 63) != 0ull};
                    for (int gi = pw; gi < NG; gi += NP) {
                        const int ql = gi * 32 + lane;
                        T v[V];
                        bool ok[V];
                        tile_vec<T>(y, sp, stage, true, c, ql, sb0, sb1, v, ok);
#pragma unroll
                        for (int j = 0; j < V; j++) {
                            if constexpr (sizeof(T) == 8) sacc.bad |= ok[j] && u64_is_nan(bits_of((double)v[j]));
                            else sacc.bad |= ok[j] && (v[j] != v[j]);
                        }
                        support_mask<T, L1>(xb, sp, c * NVEC + ql, aligned, ok);
#pragma unroll
                        for (int j = 0; j < V; j++) {
                            const unsigned bal = __ballot_sync(0xffffffffu, ok[j] && condat_test<T, L1>(v[j], g, trd));
                            if (lane == 0) mk[gi * V + j] = bal;
                        }
                    }
                } else if (lane == 0) {
                    for (int gi = pw; gi < NG; gi += NP)
#pragma unroll
                        for (int j = 0; j < V; j++) mk[gi * V + j] = 0u;
                }
                __syncwarp();
                // release: the ballots of this warp (the barrier counts NWARP - 1 arrivals: the
                // first filter also arrives for the warps before the filters beyond the first)
                if (lane == 0) mbar_arrive_cnt(&fullb[stg], pw == 0 ? (unsigned)nfw : 1u);
            }
        } else if (split && wid == 1) {
            // the walking warp: tiles i = 1, 2, ... (stage i mod S); the survivors of each group
            // that are not certain failures against the scan's current threshold go to the queue
            // in index order; the stage is refilled as soon as its survivors are queued
            const unsigned lt = (1u << lane) - 1u;
            unsigned tail = 0u, head = 0u;
            int stg = 1 % S;
            unsigned flip = 0u;
            for (int64_t i = 1; i < ring.count; i++) {
                const unsigned ph = ((base >> stg) ^ flip) & 1u;
                mbar_wait(&fullb[stg], ph, err, limit_ns, CQK_TIMEOUT);
                mbar_wait(&ring.bar[stg], ph, err, limit_ns, CQK_TIMEOUT);
                const unsigned* mk = s.pmsk[stg];
                unsigned gany = 0;
#pragma unroll
                for (int j = 0; j < V; j++) gany |= mk[lane * V + j];
                const unsigned groups = __ballot_sync(0xffffffffu, gany != 0u);
                if (groups) {
                    const int64_t c = ring.tile(i, false);
                    const int64_t sb0 = ring.b0(c), sb1 = ring.b1(c);
                    const T* stage = ring.stage(stg, 0);
                    const bool whole = sb0 == c * TT && sb1 == (c + 1) * TT;
                    const long long qklo = *reinterpret_cast<volatile long long*>(&s.qklo);
                    for (unsigned gs = groups; gs; gs &= gs - 1) {
                        const int gi = __ffs(gs) - 1;
                        const int ql = gi * 32 + lane;
                        T v[V];
                        bool ok[V];
                        if (whole) {
                            using VT = typename VecOf<T>::type;
                            const VT w = reinterpret_cast<const VT*>(stage)[ql];
#pragma unroll
                            for (int j = 0; j < V; j++) v[j] = reinterpret_cast<const T*>(&w)[j];
                        } else {
                            tile_vec<T>(y, sp, stage, true, c, ql, sb0, sb1, v, ok);
                        }
                        double av[V];
                        unsigned b[V];
                        int before = 0, cnt = 0;
#pragma unroll
                        for (int j = 0; j < V; j++) {
                            const double dv = (double)v[j];
                            av[j] = L1 ? __longlong_as_double((long long)(opaque_bits(dv) & 0x7FFFFFFFFFFFFFFFull)) : dv;
                            const bool p = ((mk[gi * V + j] >> lane) & 1u) && order_key(av[j]) > qklo;
                            b[j] = __ballot_sync(0xffffffffu, p);
                            before += __popc(b[j] & lt);
                            cnt += __popc(b[j]);
                        }
                        if (!cnt) continue;
                        // room for cnt entries (bounded wait for the scanning warp)
                        if (tail + (unsigned)cnt - head > (unsigned)kQueue) {
                            // the entries queued so far become visible, then the wait for room
                            // (lane 0 reads, the warp decides together)
                            __syncwarp();
                            if (lane == 0 && !qfault) st_release_cta(&s.qtail, tail);
                            const unsigned long long t0 = globaltimer_ns();
                            while (true) {
                                head = __shfl_sync(0xffffffffu, lane == 0 ? ld_acquire_cta(&s.qhead) : 0u, 0);
                                if (tail + (unsigned)cnt - head <= (unsigned)kQueue) break;
                                const bool quit = lane == 0 && (*reinterpret_cast<volatile unsigned*>(&s.qabort) != 0u ||
                                                                globaltimer_ns() - t0 > limit_ns);
                                if (__any_sync(0xffffffffu, quit)) {
                                    if (lane == 0) {
                                        atomicExch(err, CQK_TIMEOUT);
                                        s.qabort = 1u;
                                    }
                                    break;
                                }
                                __nanosleep(64);
                            }
                        }
                        unsigned pos = tail + (unsigned)before;
                        const int64_t e0 = (c * NVEC + ql) * V;
#pragma unroll
                        for (int j = 0; j < V; j++) {
                            if ((b[j] >> lane) & 1u) {
                                s.qv[pos % kQueue] = av[j];
                                s.qe[pos % kQueue] = e0 + j;
                                pos++;
                            }
                        }
                        tail += (unsigned)cnt;
                    }
                    __syncwarp();
                    if (lane == 0 && !qfault) st_release_cta(&s.qtail, tail);  // the tile's survivors
                }
                __syncwarp();
                // the stage is free (its filters signalled, its survivors are queued): the next tile
                if (lane == 0 && i + S < ring.count) ring.issue(ring.tile(i + S, false), stg, src);
                if (++stg == S) {
                    stg = 0;
                    flip ^= 1u;
                }
            }
            __syncwarp();
            // (qfault, testing only: nothing is published, and the scanning warp's bounded wait
            // ends with CQK_TIMEOUT)
            if (lane == 0 && !qfault) st_release_cta(&s.qdone, 1u);
        } else if (split) {
            // the scanning warp: the first tile from its stage, then the queue
            if (ring.count > 0) {
                const unsigned ph = base & 1u;
                mbar_wait(&fullb[0], ph, err, limit_ns, CQK_TIMEOUT);
                mbar_wait(&ring.bar[0], ph, err, limit_ns, CQK_TIMEOUT);
                const unsigned* mk = s.pmsk[0];
                unsigned gany = 0;
#pragma unroll
                for (int j = 0; j < V; j++) gany |= mk[lane * V + j];
                const unsigned groups = __ballot_sync(0xffffffffu, gany != 0u);
                if (groups) {
                    const int64_t c = ring.tile(0, false);
                    const int64_t sb0 = ring.b0(c), sb1 = ring.b1(c);
                    const T* stage = ring.stage(0, 0);
                    if (sb0 == c * TT && sb1 == (c + 1) * TT) {
                        condat_scan_tile<T, L1>(stage, mk, groups, c * TT, r, st);
                    } else {
                        for (unsigned gs = groups; gs; gs &= gs - 1) {
                            const int gi = __ffs(gs) - 1;
                            const int ql = gi * 32 + lane;
                            T v[V];
                            bool ok[V];
                            tile_vec<T>(y, sp, stage, true, c, ql, sb0, sb1, v, ok);
#pragma unroll
                            for (int j = 0; j < V; j++) ok[j] = ((mk[gi * V + j] >> lane) & 1u) != 0u;
                            condat_slab<T, L1>(v, ok, (c * NVEC + ql) * V, r, st);
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) {
                    if (S < ring.count) ring.issue(ring.tile(S, false), 0, src);
                    if (st.nJ > 0) {
                        *reinterpret_cast<volatile long long*>(&s.qklo) = st.klo;
                        if constexpr (sizeof(T) == 8)
                            *reinterpret_cast<volatile unsigned long long*>(&s.tb[0]) = condat_lo_bits(st);
                        else
                            *reinterpret_cast<volatile float*>(&s.trd[0]) = condat_filter_rd(st);
                    }
                    mbar_arrive(&startb[0]);  // release: the published threshold
                }
            }
            unsigned head = 0u;
            unsigned long long t0 = 0ull;
            while (ring.count > 1) {
                // (lane 0 reads, the warp decides together)
                unsigned tail = __shfl_sync(0xffffffffu, lane == 0 ? ld_acquire_cta(&s.qtail) : 0u, 0);
                if (tail == head) {
                    const unsigned done = __shfl_sync(0xffffffffu, lane == 0 ? ld_acquire_cta(&s.qdone) : 0u, 0);
                    if (done) {
                        tail = __shfl_sync(0xffffffffu, lane == 0 ? ld_acquire_cta(&s.qtail) : 0u, 0);
                        if (tail == head) break;
                    } else {
                        // bounded wait for the walking warp
                        const unsigned long long now = globaltimer_ns();
                        if (t0 == 0ull) t0 = now;
                        const bool quit = lane == 0 && (now - t0 > limit_ns ||
                                                        *reinterpret_cast<volatile unsigned*>(&s.qabort) != 0u);
                        if (__any_sync(0xffffffffu, quit)) {
                            if (lane == 0) {
                                atomicExch(err, CQK_TIMEOUT);
                                s.qabort = 1u;
                            }
                            break;
                        }
                        __nanosleep(32);
                        continue;
                    }
                }
                t0 = 0ull;
                const long long klo0 = st.klo;
                for (; head != tail; head++) {
                    const double yq = s.qv[head % kQueue];
                    const long long e = s.qe[head % kQueue];
                    if (st.nJ == 0) {  // the first element of the chunk starts J (first line of Alg. 2)
                        st.rs = e;
                        condat_start_j<L1>(st, r, yq);
                        condat_record(st, yq);
                    } else if (condat_gt<L1>(yq, st, r)) {
                        condat_take<L1>(st, r, yq, e);
                    }
                }
                __syncwarp();
                if (lane == 0) {
                    st_release_cta(&s.qhead, head);
                    if (st.nJ > 0 && st.klo != klo0) {
                        *reinterpret_cast<volatile long long*>(&s.qklo) = st.klo;
                        if constexpr (sizeof(T) == 8)
                            *reinterpret_cast<volatile unsigned long long*>(&s.tb[0]) = condat_lo_bits(st);
                        else
                            *reinterpret_cast<volatile float*>(&s.trd[0]) = condat_filter_rd(st);
                    }
                }
            }
        } else {
            const int k = wid;
            int stg = k;          // i mod S (k < nscan <= kMaxScan < S)
            unsigned flip = 0u;   // (i / S) mod 2
            for (int64_t i = k; i < ring.count; i += nscan) {
                const unsigned ph = ((base >> stg) ^ flip) & 1u;
                mbar_wait(&fullb[stg], ph, err, limit_ns, CQK_TIMEOUT);
                mbar_wait(&ring.bar[stg], ph, err, limit_ns, CQK_TIMEOUT);
                const unsigned* mk = s.pmsk[stg];
                unsigned gany = 0;
#pragma unroll
                for (int j = 0; j < V; j++) gany |= mk[lane * V + j];
                const unsigned groups = __ballot_sync(0xffffffffu, gany != 0u);
                if (groups) {
                    const int64_t c = ring.tile(i, false);
                    const int64_t sb0 = ring.b0(c), sb1 = ring.b1(c);
                    const T* stage = ring.stage(stg, 0);
                    if (sb0 == c * TT && sb1 == (c + 1) * TT) {  // the stage holds every element
                        condat_scan_tile<T, L1>(stage, mk, groups, c * TT, r, st);
                    } else {
                        for (unsigned gs = groups; gs; gs &= gs - 1) {
                            const int gi = __ffs(gs) - 1;
                            const int ql = gi * 32 + lane;
                            T v[V];
                            bool ok[V];
                            tile_vec<T>(y, sp, stage, true, c, ql, sb0, sb1, v, ok);
#pragma unroll
                            for (int j = 0; j < V; j++) ok[j] = ((mk[gi * V + j] >> lane) & 1u) != 0u;
                            condat_slab<T, L1>(v, ok, (c * NVEC + ql) * V, r, st);
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) {
                    // the stage is free (its filters signalled, its scan is done): the next tile
                    if (i + S < ring.count) ring.issue(ring.tile(i + S, false), stg, src);
                    // the threshold the filters use for this type of data
                    if (groups && st.nJ > 0) {
                        if constexpr (sizeof(T) == 8)
                            *reinterpret_cast<volatile unsigned long long*>(&s.tb[k]) = condat_lo_bits(st);
                        else
                            *reinterpret_cast<volatile float*>(&s.trd[k]) = condat_filter_rd(st);
                    }
                    if (i == k) mbar_arrive(&startb[k]);  // release: the published threshold
                }
                stg += nscan;
                if (stg >= S) {
                    stg -= S;
                    flip ^= 1u;
                }
            }
        }
        // every thread: the phases completed in this call (one per tile of each stage, one per
        // chunk with a tile on its start barrier)
        unsigned p = base;
        for (int k = 0; k < S; k++)
            if (k < ring.count) p ^= (unsigned)(((ring.count - 1 - k) / S + 1) & 1) << k;
        for (int k = 0; k < nscan; k++)
            if (k < ring.count) p ^= 1u << (kStartBit + k);
        ring.parity = p;
        __syncthreads();
    } else {
        // data not 16-byte aligned: no staging; per tile the exact filter of the whole block,
        // then warp 0 scans the survivors while the block waits
        for (int64_t i = 0; i < ring.count; i++) {
            const int64_t c = ring.tile(i, false);
            const bool anyp = condat_filter_exact<T, L1>(y, xb, sp, aligned, nullptr, false, c, 0, 0, s, sacc);
            // a tile with no survivor needs no scan (the vote is also the barrier after which the
            // ballots may be rewritten)
            if (!__syncthreads_or(anyp)) continue;
            if (wid == 0) {
                // lane g looks at group g = (k, w) of 32 vectors; the groups are visited in order
                static_assert(KC * NWARP <= 32, "one lane per group");
                unsigned gany = 0;
                if (lane < KC * NWARP)
#pragma unroll
                    for (int j = 0; j < V; j++) gany |= s.msk[lane % NWARP][(lane / NWARP) * V + j];
                for (unsigned groups = __ballot_sync(0xffffffffu, gany != 0u); groups; groups &= groups - 1) {
                    const int gi = __ffs(groups) - 1;
                    const int k = gi / NWARP, w = gi % NWARP;
                    const int ql = k * NT + w * 32 + lane;
                    T v[V];
                    bool ok[V];
                    tile_vec<T>(y, sp, nullptr, false, c, ql, 0, 0, v, ok);
#pragma unroll
                    for (int j = 0; j < V; j++) ok[j] = ((s.msk[w][k * V + j] >> lane) & 1u) != 0u;
                    condat_slab<T, L1>(v, ok, (c * (TT / V) + ql) * V, r, st);
                }
                if (lane == 0 && st.nJ > 0) {
                    s.tb[0] = condat_lo_bits(st);
                    s.trd[0] = condat_filter_rd(st);
                }
            }
            __syncthreads();
        }
    }
    parity = ring.parity;
    // final loop of Alg. 2 over J~ (scan warp k: its chunk)
    if (wid < nscan && st.nJ > 0) {
        if (st.jt_end <= st.cap) {
            __syncwarp();
            condat_final_list<L1>(st.list, st.jt_end, r, st);
        } else if (st.rs >= 0) {
            // the chunk's tiles up to the last restart: block tiles i = wid, wid + nscan, ...
            for (int64_t i = wid; i < ring.count; i += nscan) {
                const int64_t c = ring.tile(i, false);
                if (c * TT > st.rs) break;
                for (int sl = 0; sl < TT / V / 32; sl++) {
                    const int64_t q = c * (TT / V) + sl * 32 + lane;
                    T vals[V];
                    bool okv[V];
                    load_vec<T>(y, sp, q, aligned, vals, okv);
                    support_mask<T, L1>(xb, sp, q, aligned, okv);
                    condat_rescan_slab<T, L1>(vals, okv, q * V, r, st);
                }
            }
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
__device__ __forceinline__ void newton_sweep(const T* __restrict__ y, const Span& sp, const WarpSweep& sw,
                                             bool aligned, bool rev, unsigned long long tb, float rd, float ru,
                                             double lam, df Lm, PassAcc& pa) {
    constexpr int V = VecOf<T>::V;
    constexpr int U = kStreamU;
    using VT = typename VecOf<T>::type;
    const int lane = threadIdx.x & 31;
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

// one Newton pass at lambda: picks the comparison form (FP64: sign of the threshold; FP32:
// directed roundings) and whether ties / NaN are counted (first)
template <typename T, bool L1>
__device__ __forceinline__ void newton_pass(const T* __restrict__ y, const Span& sp, const WarpSweep& sw, bool aligned,
                                            bool rev, bool first, double lam, PassAcc& pa) {
    pa.acc64 = 0.0;
    pa.acc32 = df_make(0.0f);
    pa.cm = pa.ct = 0u;
    pa.nan = false;
    if constexpr (sizeof(T) == 8) {
        const GtThreshold g = make_gt(-lam);
        const df Lm = df_make(0.0f);
        if (g.neg) {
            if (first) newton_sweep<T, L1, true, true>(y, sp, sw, aligned, rev, g.bits, 0.f, 0.f, lam, Lm, pa);
            else newton_sweep<T, L1, true, false>(y, sp, sw, aligned, rev, g.bits, 0.f, 0.f, lam, Lm, pa);
        } else {
            if (first) newton_sweep<T, L1, false, true>(y, sp, sw, aligned, rev, g.bits, 0.f, 0.f, lam, Lm, pa);
            else newton_sweep<T, L1, false, false>(y, sp, sw, aligned, rev, g.bits, 0.f, 0.f, lam, Lm, pa);
        }
    } else {
        const float rd = f32_rd(-lam), ru = f32_ru(-lam);
        const df Lm = df_from_f64(lam);
        if (first) newton_sweep<T, L1, false, true>(y, sp, sw, aligned, rev, 0ull, rd, ru, lam, Lm, pa);
        else newton_sweep<T, L1, false, false>(y, sp, sw, aligned, rev, 0ull, rd, ru, lam, Lm, pa);
        pa.acc64 = df_to_f64_int_all(pa.acc32);
    }
}

// The scalar part of one Alg. 4 iteration from phi(lambda_k) and its lateral slopes: bracket,
// Newton step, the stopping tests of Sec. 4.  Returns true when the loop stops; then fin is
// the final multiplier, else next is lambda_{k+1}.
struct Alg4State {
    double lower, upper, slope;
    int stop;
};
__device__ __forceinline__ bool alg4_update(Alg4State& a, int k, double lam, double phi, double dminus, double dplus,
                                            double r, double eps34, bool final_step, double& next, double& fin) {
    const double gk = phi - r;
    double step = 0.0;
    bool done = false;
    next = lam;
    fin = lam;
    if (k == 0) {
        if (gk == 0.0) {
            a.stop = CQK_STOP_EXACT;
            done = true;
        } else if (gk < 0.0) {
            a.lower = lam;
            a.slope = dplus;
            step = -gk / dplus;
        } else {
            a.upper = lam;
            a.slope = dminus;
            step = -gk / dminus;
        }
    } else if (gk <= 0.0) {
        a.stop = CQK_STOP_BELOW;
        done = true;
    } else {
        a.upper = lam;
        a.slope = dminus;
        step = -gk / dminus;
    }
    if (!done && a.upper - a.lower < eps34 * fmax(fabs(a.upper), fabs(a.lower))) {
        a.stop = CQK_STOP_BRACKET;
        done = true;
    }
    if (!done && fabs(step) < eps34) {
        a.stop = CQK_STOP_STEP;
        done = true;
        if (final_step) fin = lam + step;  // the Newton step already computed
    }
    if (!done) {
        next = lam + step;
        if (next == lam) {
            a.stop = CQK_STOP_SAME;
            done = true;
        }
    }
    return done;
}

// per-block totals of a pass (fixed order) -> partials slot `par`, and into blk (warp 0); a
// one-block group (solo) keeps them in registers only.  The sum is an FP64 butterfly over the
// warps; the two counts are integers, stored as 64-bit integer bit patterns in their double
// slots and summed as integers (B300's FP64 pipe is the scarce unit here).
__device__ __forceinline__ void write_pass_partials(const Grp& gp, int par, double acc, unsigned cm, unsigned ct,
                                                    double (*sh)[NWARP], bool solo, double (&blk)[3]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    acc = warp_sum(acc);
    cm = __reduce_add_sync(0xffffffffu, cm);
    ct = __reduce_add_sync(0xffffffffu, ct);
    if (lane == 0) {
        sh[0][wid] = acc;
        sh[1][wid] = __longlong_as_double((long long)cm);
        sh[2][wid] = __longlong_as_double((long long)ct);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        double sum = lane < NWARP ? sh[0][lane] : 0.0;
#pragma unroll
        for (int o = NWARP / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        // (64-bit: a one-block group over more than 2^32 elements)
        unsigned long long c1 = lane < NWARP ? (unsigned long long)__double_as_longlong(sh[1][lane]) : 0ull;
        unsigned long long c2 = lane < NWARP ? (unsigned long long)__double_as_longlong(sh[2][lane]) : 0ull;
#pragma unroll
        for (int o = NWARP / 2; o > 0; o >>= 1) {
            c1 += __shfl_xor_sync(0xffffffffu, c1, o);
            c2 += __shfl_xor_sync(0xffffffffu, c2, o);
        }
        const unsigned long long c12 = c1 + c2;
        if (!solo && lane == 0) {
            gp.part[((size_t)par * kPartialQ + 0) * gp.g + gp.member] = sum;
            gp.part[((size_t)par * kPartialQ + 1) * gp.g + gp.member] = __longlong_as_double((long long)c1);
            gp.part[((size_t)par * kPartialQ + 2) * gp.g + gp.member] = __longlong_as_double((long long)c12);
        }
        blk[0] = sum;
        blk[1] = (double)c1;
        blk[2] = (double)c12;
    }
}

// The group totals of a pass from the partials of write_pass_partials (warp 0; every block
// computes the same values in the same order): lane l takes blocks l, l + 32, ... in turn,
// then an FP64 butterfly for the sum and integer sums for the counts.
__device__ __forceinline__ void grid_totals_pass(const double* part, int g, int par, double (&out)[3]) {
    const int lane = threadIdx.x & 31;
    const double* p0 = part + ((size_t)par * kPartialQ + 0) * g;
    const double* p1 = part + ((size_t)par * kPartialQ + 1) * g;
    const double* p2 = part + ((size_t)par * kPartialQ + 2) * g;
    double sum = 0.0;
    unsigned long long c1 = 0ull, c2 = 0ull;
#pragma unroll 4
    for (int b = lane; b < g; b += 32) {
        sum += ld_cg(p0 + b);
        c1 += (unsigned long long)__double_as_longlong(ld_cg(p1 + b));
        c2 += (unsigned long long)__double_as_longlong(ld_cg(p2 + b));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        c1 += __shfl_xor_sync(0xffffffffu, c1, o);
        c2 += __shfl_xor_sync(0xffffffffu, c2, o);
    }
    out[0] = sum;
    out[1] = (double)c1;
    out[2] = (double)c2;
}

// the final pass: x_i = max{0, y_i + lambda} (l1: sgn(y_i) max{0, |y_i| + lambda}; copy: x = y),
// the free mask, and the sum of the stored |x| and the count of nonzero x
template <typename T, bool L1>
__device__ __forceinline__ void final_sweep(const T* __restrict__ y, T* __restrict__ x, uint32_t* mask,
                                            const Span& sp, const WarpSweep& sw, bool aligned, bool rev, bool copy,
                                            double lamf, double& sx, df& sx32, long long& nz) {
    constexpr int V = VecOf<T>::V;
    const int lane = threadIdx.x & 31;
    {
        const GtThreshold g = make_gt(-lamf);
        const float rd = f32_rd(-lamf);
        const df Lm = df_from_f64(lamf);
        for (int64_t it = 0; it < sw.count; it++) {
            const int64_t base = sw.base(it, rev);
            T vv[kStreamU][V];
            bool okk[kStreamU][V];
            bool sela[kStreamU][V];  // the iteration's mask bits, stored together after the rows
#pragma unroll
            for (int u = 0; u < kStreamU; u++) load_vec<T>(y, sp, base + u * 32 + lane, aligned, vv[u], okk[u]);
#pragma unroll
            for (int u = 0; u < kStreamU; u++) {
                const int64_t qw = base + u * 32;
                const int64_t q = qw + lane;
                const T(&v)[V] = vv[u];
                const bool(&ok)[V] = okk[u];
                T o[V];
                bool(&sel)[V] = sela[u];
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
            }
            if (mask) store_mask_rows<V, kStreamU>(mask, sp, base, sela);
        }
    }
}

// one pass over the group's span accumulating the sum and maximum of y (l1: |y|) and the NaN
// check (every thread of the group)
template <typename T, bool L1>
__device__ __forceinline__ void sum_sweep(const T* __restrict__ y, const Span& sp, const Grp& gp, bool aligned,
                                          SumAcc& sacc) {
    constexpr int V = VecOf<T>::V;
    const int lane = threadIdx.x & 31;
    const WarpSweep sw(span_qlo<V>(sp), span_qhi<V>(sp), kStreamU, gp.member, gp.g);
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
            if (okk[u][j] && sum_elem<T, L1>(sacc, vv[u][j])) widem |= 1u << uj;
        }
        if constexpr (sizeof(T) == 8) {
            // values outside the df operating range: exact FP64, one trip per element
            for (unsigned m = widem; m; m &= m - 1) sum_wide<T, L1>(sacc, pick2(vv, __ffs(m) - 1));
            // fold the lazy pair (at most 64 terms) into FP64: one FP64 add per 4 sweeps
            if ((it & 3) == 3) sacc.fold();
        }
    }
}

// sum_sweep by one warp alone
template <typename T, bool L1>
__device__ __forceinline__ void sum_sweep_warp(const T* __restrict__ y, const Span& sp, bool aligned, SumAcc& sacc) {
    constexpr int V = VecOf<T>::V;
    const int lane = threadIdx.x & 31;
    const WarpSweep sw = WarpSweep::solo(span_qlo<V>(sp), span_qhi<V>(sp), kStreamU);
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
            if (okk[u][j] && sum_elem<T, L1>(sacc, vv[u][j])) widem |= 1u << uj;
        }
        if constexpr (sizeof(T) == 8) {
            for (unsigned m = widem; m; m &= m - 1) sum_wide<T, L1>(sacc, pick2(vv, __ffs(m) - 1));
            if ((it & 3) == 3) sacc.fold();
        }
    }
}

// ---- one projection by one group of blocks ------------------------------------------------
// A supplies the arrays, r, the options and the info slot; gp the group (member, size, span,
// header and partial sums).  The instance is the span [gp.sp.lo, gp.sp.hi) of y and x.
template <typename T, bool L1>
__device__ __forceinline__ void simplex_solve(const SimplexArgs& A, const Grp& gp, T* smem, uint64_t* bars,
                                              unsigned& ring_parity) {
    constexpr int V = VecOf<T>::V;
    __shared__ double sh[kPartialQ][NWARP];
    __shared__ double bc[kPartialQ];
    // loop state written by thread 0 after each update, read by all threads
    __shared__ double s_lam, s_final;
    __shared__ int s_done, s_bad, s_redo;
    const T* __restrict__ y = static_cast<const T*>(A.y);
    const Span sp = gp.sp;
    const int64_t n = sp.hi - sp.lo;
    const int64_t qlo = span_qlo<V>(sp), qhi = span_qhi<V>(sp);
    const int lane = threadIdx.x & 31;
    const int G = gp.g;
    const bool aligned = A.aligned != 0;
    unsigned bar_target = (unsigned)G + (A.fault_inject == 1 ? 1u : 0u);
    const double r = A.r;

    // ------------------------------------------------------------------ pass 0: start
    double lam0 = 0.0, abs_sum = 0.0;
    int passes = 0, nchunks = 0, tile = 0;
    bool condat_start = false;  // lambda_0 from the Alg. 2 union (>= lambda*)
    int par0 = 1;               // partial-sum slot of the first Newton pass
    {
        double q[4] = {0.0, 0.0, 0.0, -INFINITY};  // sum y (l1: |y|), union sum, union size, max y (l1: |y|)
        const bool warm = A.init == CQK_INIT_WARM;
        const bool condat = A.init == CQK_INIT_CONDAT || warm;
        // the formula and given starts need sum y and max y (l1: |y|), which also serve the l1
        // ball's inside test; after an Alg. 2 start the l1 ball sums |y| only when needed (below)
        const bool sum_pass = !condat;
        bool bad = false;
        SumAcc sacc;
        sacc.init();
        if (sum_pass) {
            sum_sweep<T, L1>(y, sp, gp, aligned, sacc);
            passes++;
        }
        // chunks of at least condat_chunk elements (the J updates are scalar FP64 work, which
        // a partition into many small chunks multiplies, and larger chunks give a better
        // lambda_0), at most one per block
        const int nchunk = (int)min((int64_t)G, max((int64_t)1, (n + A.condat_chunk - 1) / A.condat_chunk));
        // chunks per block (option scan_warps, default 1): the scan of a chunk is one warp's
        // dependency chain, and a block that alone holds a short instance may split it over
        // several scan warps, but each doubling of the chunks loosens the union's lambda_0 by
        // about one Newton step (ragged FP32 batches: 3.4 -> 4.5 -> 5.3 steps); on the 4096-
        // instance batch one scan warp per block is the fastest (2.30 ms; 2.35 ms with four for
        // one-block instances of 4 to 15 tiles, 2.56 / 2.80 ms with two / four everywhere)
        int nscan = 1;
        if (condat && aligned) nscan = A.scan_warps > 0 ? A.scan_warps : 1;
        if (condat) {
            double Sw = 0.0;
            long long nJw = 0;
            condat_block<T, L1>(y, warm ? static_cast<const T*>(A.xbar) : nullptr, sp, aligned, r, gp.member,
                                nchunk, nscan, smem, bars, ring_parity, &gp.hdr->error, A.limit_ns,
                                A.fault_inject == 2, sacc, Sw, nJw);
            q[1] = lane == 0 ? Sw : 0.0;  // each scan warp's chunk (zero elsewhere)
            q[2] = lane == 0 ? (double)nJw : 0.0;
            passes++;
        }
        bad = sacc.bad;
        q[0] = sacc.sum();
        q[3] = sum_max<T>(sacc);
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
        if (threadIdx.x < 32) {
            double pv[4];
            warp0_combine<4>(sh, 3, pv);
            write_partials<4>(gp.part, gp.member, G, 0, pv);
        }
        __syncthreads();
        if (!group_barrier(gp, bar_target, A.limit_ns, A.fault_inject == 1)) {
            if (threadIdx.x == 0) A.info->status = CQK_TIMEOUT;
            return;
        }
        bar_target += (unsigned)G;
        double red[4];
        grid_reduce<4>(gp.part, G, 0, 3, red, sh, bc);
        abs_sum = red[0];
        if (condat && red[2] > 0.0) {
            lam0 = (r - red[1]) / red[2];  // eq. (lambdaJ) on the union of the chunks' J
            condat_start = true;
            nchunks = (int)nchunk * nscan;
            tile = condat_tile<T>();
        } else if (condat) {
            // warm start with an empty J_+ (no element of the estimate's support): Sec. 3.3
            const double y1 = (double)y[sp.lo];
            lam0 = fmax(r / (double)n, L1 ? -fabs(y1) : -y1);
            nchunks = (int)nchunk * nscan;
            tile = condat_tile<T>();
        } else if (A.init == CQK_INIT_GIVEN) {
            lam0 = fmax(A.lambda0, -red[3]);  // Alg. 4, line 1
        } else {
            lam0 = fmax((r - red[0]) / (double)n, -red[3]);  // eq. (CQKlambda0) with b = d = 1; Alg. 4 line 1
        }
        // The l1 ball's inside test needs sum |y|, except when the Alg. 2 start already proves
        // sum |y| > r: lambda_0 >= lambda* (eq. (lambdaJ)), and lambda* >= 0 whenever sum |y| <= r
        // (then phi(0) = sum |y| <= r).  lambda_0 = (r - S)/C < 0 is taken as proven only when
        // r - S is negative beyond the rounding of S.
        if (L1 && condat) {
            const bool outside = condat_start && (r - red[1]) < -1e-13 * (fabs(r) + fabs(red[1]));
            if (outside) {
                abs_sum = INFINITY;
            } else {
                SumAcc s2;
                s2.init();
                sum_sweep<T, L1>(y, sp, gp, aligned, s2);
                passes++;
                double pv[1] = {s2.sum()};
                block_sum<1>(pv, sh);
                write_partials<1>(gp.part, gp.member, G, 1, pv);
                if (!group_barrier(gp, bar_target, A.limit_ns, A.fault_inject == 1)) {
                    if (threadIdx.x == 0) A.info->status = CQK_TIMEOUT;
                    return;
                }
                bar_target += (unsigned)G;
                double red1[1];
                grid_reduce<1>(gp.part, G, 1, -1, red1, sh, bc);
                abs_sum = red1[0];
                par0 = 0;  // slot 1 holds this reduction: the Newton loop starts on slot 0
            }
        }
    }
    bool bad_input = A.validate && (__ldcg(&gp.hdr->flags) & kFlagBadInput);
    // Compiler barriers between the start, the Newton loop and the final pass: without them the
    // l1-ball kernel's code came out ~80 us slower per solve at n = 1e8 (the simplex kernel's
    // did not change), though every phase computes the same.
    asm volatile("" ::: "memory");

    // ------------------------------------------------------------------ Newton loop (Alg. 4)
    // thread 0 keeps the bracket and the stopping logic; every thread keeps lambda
    double lam = lam0, final_lam = lam0;
    Alg4State a4{-INFINITY, INFINITY, 0.0, CQK_STOP_NONE};  // thread 0
    int status = CQK_OK, k = 0;                              // status: all threads
    bool copy = false;                                       // l1 ball, y inside
    if (bad_input) {
        status = CQK_BAD_INPUT;
    } else if (L1 && abs_sum <= r) {
        copy = true;
        a4.stop = CQK_STOP_INSIDE;
        lam = final_lam = 0.0;
    } else {
        int par = par0;
        // ties (phi'_+) are needed only when the first step goes right; from the Alg. 2 start
        // (lambda_0 >= lambda*) it goes left, and the pass is redone with ties if it does not
        bool ties = !condat_start;
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
            const bool first = (k == 0) && ties;
            newton_pass<T, L1>(y, sp, WarpSweep(qlo, qhi, kStreamU, gp.member, gp.g), aligned, rev, first, lam, pa);
            passes++;
            if (A.validate && first && __any_sync(0xffffffffu, pa.nan) && lane == 0)
                atomicOr(&gp.hdr->flags, kFlagBadInput);
            // a one-block group needs neither the partials in memory nor a barrier: thread 0
            // already holds the totals (bit-identical to the one-partial grid sum)
            const bool solo = G == 1 && A.fault_inject != 1;
            double blk[3];
            write_pass_partials(gp, par, pa.acc64, pa.cm, pa.ct, sh, solo, blk);
            if (!solo) {
                if (!group_barrier(gp, bar_target, A.limit_ns, A.fault_inject == 1)) {
                    if (threadIdx.x == 0) A.info->status = CQK_TIMEOUT;
                    return;
                }
                bar_target += (unsigned)G;
            }
            double red[3] = {blk[0], blk[1], blk[2]};
            if (!solo && threadIdx.x < 32) grid_totals_pass(gp.part, G, par, red);
            {
                if (threadIdx.x == 0) {
                    int done = 0, bad = 0, redo = 0;
                    double next = lam;
                    if (A.validate && first && (__ldcg(&gp.hdr->flags) & kFlagBadInput)) {
                        bad = 1;
                        done = 1;
                    } else if (k == 0 && !first && red[0] - r < 0.0) {
                        redo = 1;  // phi(lambda_0) < r: the step needs phi'_+, count the ties
                    } else {
                        double fin;
                        done = alg4_update(a4, k, lam, red[0], red[1], red[2], r, A.eps34, A.final_step != 0, next,
                                           fin) ? 1 : 0;
                        s_final = fin;
                    }
                    s_lam = next;
                    s_done = done;
                    s_bad = bad;
                    s_redo = redo;
                }
            }
            __syncthreads();
            par ^= 1;
            if (s_redo) {
                ties = true;
                k--;
                __syncthreads();
                continue;
            }
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
    asm volatile("" ::: "memory");
    double sx = 0.0;
    df sx32 = df_make(0.0f);
    long long nz = 0;
    T* __restrict__ x = static_cast<T*>(A.x);
    if (!bad_input)
        final_sweep<T, L1>(y, x, A.mask, sp, WarpSweep(qlo, qhi, kStreamU, gp.member, gp.g), aligned, (k & 1) == 0,
                           copy, final_lam, sx, sx32, nz);
    if constexpr (sizeof(T) == 4) sx = df_to_f64_int_all(sx32);
    double pv[2] = {sx, (double)nz}, tot[2];
    if (last_block_sums<2>(gp.part, gp.member, G, &gp.hdr->ticket, pv, tot, sh) && threadIdx.x == 0) {
        cqk_info inf;
        const double sumx = copy ? abs_sum : tot[0];  // inside the l1 ball x = y
        inf.lambda = final_lam;
        inf.residual = sumx - r;
        inf.abs_bx = sumx;
        inf.slope = a4.slope;
        inf.lambda0 = lam0;
        inf.nfree = (int64_t)tot[1];
        inf.iters = k;
        const int e = *(volatile int*)&gp.hdr->error;
        inf.status = e ? e : status;
        inf.passes = passes + (bad_input ? 0 : 1);
        inf.stop = a4.stop;
        inf.nchunks = nchunks;
        inf.tile = tile;
        *A.info = inf;
    }
}

// ---- one small projection by one warp ------------------------------------------------------
// The same method as simplex_solve for an instance that one warp streams quickly: the Alg. 2
// start is one chunk (the whole instance, tiles of 32 vectors in index order), the Newton
// loop reduces with warp shuffles only, and every lane runs the same scalar update (no
// barrier, no shared state but the warp's accepted-value list).  Called by the 32 lanes of
// one warp; list has kWarpList entries.
constexpr int kWarpList = 1024;
static_assert(kWarpList * NWARP * sizeof(double) <= kCondatSmem, "warp lists fit the stage memory");

template <typename T, bool L1>
__device__ void simplex_warp_solve(const SimplexArgs& A, const Span& sp, double* list) {
    constexpr int V = VecOf<T>::V;
    const T* __restrict__ y = static_cast<const T*>(A.y);
    const int lane = threadIdx.x & 31;
    const int64_t n = sp.hi - sp.lo;
    const int64_t qlo = span_qlo<V>(sp), qhi = span_qhi<V>(sp);
    const bool aligned = A.aligned != 0;
    const double r = A.r;
    const bool warm = A.init == CQK_INIT_WARM;
    const bool condat = A.init == CQK_INIT_CONDAT || warm;
    const T* __restrict__ xb = warm ? static_cast<const T*>(A.xbar) : nullptr;
    int passes = 0;

    // ---- pass 0: start
    SumAcc sacc;
    sacc.init();
    double lam0 = 0.0, abs_sum = 0.0, Sunion = 0.0;
    bool condat_start = false;
    if (!condat) {
        sum_sweep_warp<T, L1>(y, sp, aligned, sacc);
        passes++;
    } else {
        CondatState st;
        condat_init(st, list, kWarpList);
        for (int64_t q0 = (qlo / 32) * 32; q0 < qhi; q0 += 32) {
            const int64_t q = q0 + lane;
            T v[V];
            bool ok[V];
            load_vec<T>(y, sp, q, aligned, v, ok);
#pragma unroll
            for (int j = 0; j < V; j++) {
                if constexpr (sizeof(T) == 8) sacc.bad |= ok[j] && u64_is_nan(bits_of((double)v[j]));
                else sacc.bad |= ok[j] && (v[j] != v[j]);
            }
            support_mask<T, L1>(xb, sp, q, aligned, ok);
            condat_slab<T, L1>(v, ok, q * V, r, st);
        }
        passes++;
        if (st.nJ > 0) {
            if (st.jt_end <= kWarpList) {  // the final loop of Alg. 2 over J~
                __syncwarp();
                condat_final_list<L1>(list, st.jt_end, r, st);
            } else {
                for (int64_t q0 = (qlo / 32) * 32; q0 * V <= st.rs; q0 += 32) {
                    const int64_t q = q0 + lane;
                    T v[V];
                    bool ok[V];
                    load_vec<T>(y, sp, q, aligned, v, ok);
                    support_mask<T, L1>(xb, sp, q, aligned, ok);
                    condat_rescan_slab<T, L1>(v, ok, q * V, r, st);
                }
            }
            lam0 = (r - st.S) / (double)st.nJ;  // eq. (lambdaJ)
            condat_start = true;
            Sunion = st.S;
        } else {
            // warm start with an empty J_+ (Sec. 3.3)
            const double y1 = (double)y[sp.lo];
            lam0 = fmax(r / (double)n, L1 ? -fabs(y1) : -y1);
        }
    }
    const bool bad_input = A.validate && __any_sync(0xffffffffu, sacc.bad);
    if (!condat) {
        const double sum = warp_sum(sacc.sum()), mx = warp_max(sum_max<T>(sacc));
        abs_sum = sum;
        if (A.init == CQK_INIT_GIVEN) lam0 = fmax(A.lambda0, -mx);  // Alg. 4, line 1
        else lam0 = fmax((r - sum) / (double)n, -mx);                // eq. (CQKlambda0); Alg. 4 line 1
    } else if (L1) {
        // the inside test of the l1 ball (see simplex_solve)
        const bool outside = condat_start && (r - Sunion) < -1e-13 * (fabs(r) + fabs(Sunion));
        if (outside) {
            abs_sum = INFINITY;
        } else {
            SumAcc s2;
            s2.init();
            sum_sweep_warp<T, L1>(y, sp, aligned, s2);
            passes++;
            abs_sum = warp_sum(s2.sum());
        }
    }

    // ---- Newton loop (Alg. 4): every lane holds the same state
    double lam = lam0, final_lam = lam0;
    Alg4State a4{-INFINITY, INFINITY, 0.0, CQK_STOP_NONE};
    int status = CQK_OK, k = 0;
    bool copy = false;
    if (bad_input) {
        status = CQK_BAD_INPUT;
    } else if (L1 && abs_sum <= r) {
        copy = true;
        a4.stop = CQK_STOP_INSIDE;
        lam = final_lam = 0.0;
    } else {
        bool ties = !condat_start;
        for (k = 0;; k++) {
            if (k >= A.max_iter) {
                status = CQK_MAXITER;
                break;
            }
            const bool first = (k == 0) && ties;
            PassAcc pa;
            newton_pass<T, L1>(y, sp, WarpSweep::solo(qlo, qhi, kStreamU), aligned, (k & 1) == 0, first, lam, pa);
            passes++;
            const double phi = warp_sum(pa.acc64);
            const double dminus = (double)__reduce_add_sync(0xffffffffu, pa.cm);
            const double dplus = dminus + (double)__reduce_add_sync(0xffffffffu, pa.ct);
            if (A.validate && first && __any_sync(0xffffffffu, pa.nan)) {
                status = CQK_BAD_INPUT;
                k++;
                copy = false;
                final_lam = lam;
                break;
            }
            if (k == 0 && !first && phi - r < 0.0) {  // the first step needs phi'_+: count the ties
                ties = true;
                k--;
                continue;
            }
            double next, fin;
            if (alg4_update(a4, k, lam, phi, dminus, dplus, r, A.eps34, A.final_step != 0, next, fin)) {
                final_lam = fin;
                k++;
                break;
            }
            lam = next;
            final_lam = lam;
        }
    }

    // ---- final pass: x, mask, sums
    double sx = 0.0;
    df sx32 = df_make(0.0f);
    long long nz = 0;
    if (status != CQK_BAD_INPUT)
        final_sweep<T, L1>(y, static_cast<T*>(A.x), A.mask, sp, WarpSweep::solo(qlo, qhi, kStreamU), aligned,
                           (k & 1) == 0, copy, final_lam, sx, sx32, nz);
    if constexpr (sizeof(T) == 4) sx = df_to_f64_int_all(sx32);
    sx = warp_sum(sx);
    const long long nzt = (long long)__reduce_add_sync(0xffffffffu, (unsigned)nz);
    if (lane == 0) {
        cqk_info inf;
        const double sumx = copy ? abs_sum : sx;
        inf.lambda = final_lam;
        inf.residual = sumx - r;
        inf.abs_bx = sumx;
        inf.slope = a4.slope;
        inf.lambda0 = lam0;
        inf.nfree = nzt;
        inf.iters = k;
        inf.status = status;
        inf.passes = passes + (status == CQK_BAD_INPUT ? 0 : 1);
        inf.stop = a4.stop;
        inf.nchunks = condat ? 1 : 0;
        inf.tile = condat ? condat_tile<T>() : 0;
        *A.info = inf;
    }
}

// the bulk-copy stages of the Alg. 2 start: kCondatSmem bytes of dynamic shared memory and
// their mbarriers, initialised once per block
__device__ __forceinline__ void init_condat_bars(uint64_t* bars) {
    if (threadIdx.x == 0) {
        for (int k = 0; k < kCondatStages; k++) {
            mbar_init(&bars[k], 1);                           // the stage's bulk copy
            mbar_init(&bars[kCondatStages + k], NWARP - 1);  // the filtering warps (pipelined Alg. 2)
        }
        for (int k = 0; k < kMaxScan; k++) mbar_init(&bars[2 * kCondatStages + k], 1);  // scan k's first tile
        fence_barrier_init();
    }
    __syncthreads();
}

#ifndef CQK_BATCH_ONLY
template <typename T, bool L1>
__global__ void __launch_bounds__(NT, kMinBlocksPerSM) simplex_kernel(SimplexArgs A) {
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    __shared__ uint64_t bars[2 * kCondatStages + kMaxScan];
    unsigned parity = 0;
    init_condat_bars(bars);
    Grp gp;
    gp.member = blockIdx.x;
    gp.g = gridDim.x;
    gp.sp = Span{0, A.n};
    gp.hdr = A.hdr;
    gp.part = A.part;
    simplex_solve<T, L1>(A, gp, reinterpret_cast<T*>(dyn_smem), bars, parity);
}

#endif  // CQK_BATCH_ONLY

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
__global__ void __launch_bounds__(NT, kMinBlocksPerSM) simplex_batched_kernel(SimplexBatchArgs P) {
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    __shared__ uint64_t bars[2 * kCondatStages + kMaxScan];
    unsigned parity = 0;
    init_condat_bars(bars);
    while (true) {
        const Slot sl = next_slot(P.R, P.B);
        if (sl.pack_first >= 0) {  // a pack of small instances, one per warp
            const long long p = sl.pack_first + (threadIdx.x >> 5);
            if (p < P.B) {
                const int inst = P.R.order[p];
                const Span sp{P.offsets[inst], P.offsets[inst + 1]};
                SimplexArgs A = P.base;
                A.r = P.r[inst];
                A.info = P.info + inst;
                const int64_t len = sp.hi - sp.lo;
                const bool r_ok = A.r > 0.0 && A.r < INFINITY;
                if (len <= 0 || !r_ok) {
                    if ((threadIdx.x & 31) == 0) {
                        if (len < 0 || !r_ok) write_plain_info(A.info, CQK_BAD_ARG, CQK_STOP_NONE, A.r);
                        else if (L1) write_plain_info(A.info, CQK_OK, CQK_STOP_INSIDE, A.r);
                        else write_plain_info(A.info, CQK_INFEASIBLE, CQK_STOP_NONE, A.r);
                    }
                } else {
                    simplex_warp_solve<T, L1>(A, sp, reinterpret_cast<double*>(dyn_smem) + (threadIdx.x >> 5) * kWarpList);
                }
            }
            continue;
        }
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
        simplex_solve<T, L1>(A, gp, reinterpret_cast<T*>(dyn_smem), bars, parity);
    }
}

}  // namespace

int CQK_VFN(launch_simplex_batched)(int64_t B, const int64_t* offsets, int dtype, const void* y, const double* r, int l1,
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
    A.scan_warps = o.scan_warps;
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
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCondatSmem);
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return CQK_CUDA_ERROR;
    }
    int grid = persistent_grid(kern, NT, kCondatSmem, INT64_MAX / 2, o.max_blocks);
    if (grid <= 0) return CQK_CUDA_ERROR;
    if ((int64_t)grid > B * kMaxGroup) grid = (int)(B * kMaxGroup);
    const int64_t per_block = o.group_elems > 0 ? o.group_elems : kSimplexGroupElems;
    // instances shorter than 2^warp_log2 are solved one per warp
    int rc = CQK_VFN(plan_batch)(offsets, B, per_block, grid, ws, s, o.warp_log2);
    if (rc != CQK_OK) return rc;
    void* args[] = {&P};
    e = cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(NT), args, kCondatSmem, s);
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return CQK_CUDA_ERROR;
    }
    return CQK_OK;
}

#ifndef CQK_BATCH_ONLY
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
    A.scan_warps = o.scan_warps;
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
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCondatSmem);
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return CQK_CUDA_ERROR;
    }
    const int grid = persistent_grid(kern, NT, kCondatSmem, (n + vec - 1) / vec, o.max_blocks);
    if (grid <= 0) return CQK_CUDA_ERROR;
    e = cudaMemsetAsync(ws, 0, sizeof(WsHeader), s);
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return CQK_CUDA_ERROR;
    }
    void* args[] = {&A};
    e = cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(NT), args, kCondatSmem, s);
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return CQK_CUDA_ERROR;
    }
    return CQK_OK;
}

#endif  // CQK_BATCH_ONLY

}  // namespace cqk
