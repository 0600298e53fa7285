// cqk_device.cuh -- device building blocks of libcqk (sm_103a).
//
// B300 executes FP64 at ~1.6 operations per clock per SM against ~114 for FP32
// (measured), so a per-element FP64 map would run 5-30x below the HBM roofline.
// The per-element work of the map-reduce therefore uses:
//   * exact comparisons of FP64 values on their bit patterns (integer pipe);
//   * double-float ("df") arithmetic: a value is an unevaluated sum hi + lo of
//     two floats, combined with the error-free transformations TwoSum
//     (Knuth), Fast-TwoSum (Dekker) and TwoProd via FMA, giving ~46-48
//     significant bits on the FP32 pipe;
//   * FP64 only for per-thread flushes of df accumulators, for the few
//     elements whose value must be exact in FP64, and for the scalar Newton
//     update.
// Nothing here depends on the problem.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cqk {

// ------------------------------------------------------------------------------------------
// The words of a double as opaque integers.  Bit tests written on __double_as_longlong are
// recognised by the compiler as floating-point classifications and emitted as FP64
// instructions, the scarcest unit of this GPU; a move through inline PTX hides the origin of
// the bits so that the tests below stay on the integer pipe.
__device__ __forceinline__ unsigned hi_word(double x) {
    unsigned h;
    asm("mov.b32 %0, %1;" : "=r"(h) : "r"(__double2hiint(x)));
    return h;
}
__device__ __forceinline__ unsigned lo_word(double x) {
    unsigned l;
    asm("mov.b32 %0, %1;" : "=r"(l) : "r"(__double2loint(x)));
    return l;
}
__device__ __forceinline__ unsigned long long opaque_bits(double x) {
    unsigned long long b;
    asm("mov.b64 %0, %1;" : "=l"(b) : "l"(__double_as_longlong(x)));
    return b;
}

// double-float arithmetic (round to nearest; never contracted: the library is compiled with
// -fmad=false and fused operations are written as explicit fmaf)
struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_make(float h) { return {h, 0.0f}; }

// Knuth TwoSum: s + e == a + b exactly.
__device__ __forceinline__ df two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// Dekker Fast-TwoSum, requires |a| >= |b| (or a == 0): s + e == a + b exactly.
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

// TwoProd with FMA: p + e == a * b exactly (barring underflow).
__device__ __forceinline__ df two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    float e = fmaf(a, b, -p);
    return {p, e};
}

// (a.hi + a.lo) + (b.hi + b.lo), relative error <= ~2^-47 of the result.
__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    df t = two_sum(a.lo, b.lo);
    float e = __fadd_rn(s.lo, t.hi);
    df u = fast_two_sum(s.hi, e);
    e = __fadd_rn(t.lo, u.lo);
    return fast_two_sum(u.hi, e);
}

// df + float, relative error <= ~2^-47.
__device__ __forceinline__ df df_add_f(df a, float b) {
    df s = two_sum(a.hi, b);
    float e = __fadd_rn(s.lo, a.lo);
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

// df * df, relative error <= ~2^-46.
__device__ __forceinline__ df df_mul(df a, df b) {
    df p = two_prod(a.hi, b.hi);
    float e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
    return fast_two_sum(p.hi, e);
}

// df * df without the final renormalisation (hi = product of the high parts, lo = all the
// correction terms): for feeding lazily normalised accumulators.
__device__ __forceinline__ df df_mul_lazy(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    return {p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, fmaf(a.hi, b.hi, -p)))};
}

// df * float, relative error <= ~2^-47.
__device__ __forceinline__ df df_mul_f(df a, float b) {
    df p = two_prod(a.hi, b);
    float e = fmaf(a.lo, b, p.lo);
    return fast_two_sum(p.hi, e);
}

// Approximate reciprocal of a float (MUFU, ~1 ulp); subnormals are outside the
// operating range of the df path (see df_in_range).
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// a / b by long division in df: q1 = a.hi/b.hi, then two corrections with the exact
// remainder.  rb = rcp_approx(b.hi).  Relative error <= ~2^-45.
__device__ __forceinline__ df df_div(df a, df b, float rb) {
    float q1 = __fmul_rn(a.hi, rb);
    df r = df_add(a, df_neg(df_mul_f(b, q1)));
    float q2 = __fmul_rn(r.hi, rb);
    df q = fast_two_sum(q1, q2);
    df r2 = df_add(a, df_neg(df_mul(b, q)));
    float q3 = __fmul_rn(r2.hi, rb);
    return df_add_f(q, q3);
}

// order of normalised df values
__device__ __forceinline__ bool df_lt(df a, df b) { return (a.hi < b.hi) || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool df_eq(df a, df b) { return a.hi == b.hi && a.lo == b.lo; }

// df -> double (one FP64 add).
__device__ __forceinline__ double df_to_f64(df a) { return (double)a.hi + (double)a.lo; }

// float -> double on the integer pipe (exact for 0 and normal floats; the df path never
// produces subnormal or non-finite parts for values it keeps).
__device__ __forceinline__ double f32_to_f64_bits(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xFFu;
    const unsigned hi = (u & 0x80000000u) | (e ? (((e + 896u) << 20) | ((u >> 3) & 0xFFFFFu)) : 0u);
    const unsigned lo = e ? (u << 29) : 0u;
    return __hiloint2double((int)hi, (int)lo);
}
// df -> double with one FP64 add and no conversion instruction.
__device__ __forceinline__ double df_to_f64_int(df a) { return f32_to_f64_bits(a.hi) + f32_to_f64_bits(a.lo); }

// double -> df with FP64 arithmetic (per-call scalars only): the pair rounds x to ~48 bits.
__device__ __forceinline__ df df_from_f64(double x) {
    float h = __double2float_rn(x);
    if (isinf(h) || h == 0.0f) return {h, 0.0f};
    float l = __double2float_rn(x - (double)h);
    return {h, l};
}

// ------------------------------------------------------------------------------------------
// FP64 -> df on the integer pipe.  hi = the leading 24 significant bits (truncated),
// lo = the next 23 bits (truncated); |x - hi - lo| < 2^-46 |x|.  Valid for
// 2^-103 <= |x| < 2^128 and for x = +-0 (-> 0) and +-inf (-> +-inf, lo = 0).
// Operating range of the df path: finite nonzero magnitudes in [2^-60, 2^60].
__device__ __forceinline__ df split_f64(double x) {
    unsigned lo = (unsigned)__double2loint(x);
    unsigned hi = (unsigned)__double2hiint(x);
    unsigned sgn = hi & 0x80000000u;
    unsigned e = (hi >> 20) & 0x7FFu;
    unsigned fh = sgn | (((hi & 0x7FFFFFFFu) - (896u << 20)) << 3) | (lo >> 29);
    unsigned base = sgn | ((e - 919u) << 23);
    float flo = __fsub_rn(__uint_as_float(base | ((lo >> 6) & 0x7FFFFFu)), __uint_as_float(base));
    float fhi = __uint_as_float(fh);
    if (e == 0u) { fhi = __uint_as_float(sgn); flo = 0.0f; }
    if (e == 0x7FFu) { fhi = __uint_as_float(sgn | 0x7F800000u | (hi & 0xFFFFFu) | lo); flo = 0.0f; }
    return {fhi, flo};
}

// split_f64 for values known to be finite (0 allowed) inside the df operating range.
__device__ __forceinline__ df split_f64_finite(double x) {
    const unsigned lo = (unsigned)__double2loint(x);
    const unsigned hi = (unsigned)__double2hiint(x);
    const unsigned sgn = hi & 0x80000000u;
    const unsigned fh = sgn | (((hi & 0x7FFFFFFFu) - (896u << 20)) << 3) | (lo >> 29);
    const unsigned base = (fh & 0xFF800000u) - (23u << 23);
    float flo = __fsub_rn(__uint_as_float(base | ((lo >> 6) & 0x7FFFFFu)), __uint_as_float(base));
    float fhi = __uint_as_float(fh);
    if ((hi & 0x7FF00000u) == 0u) { fhi = __uint_as_float(sgn); flo = 0.0f; }
    return {fhi, flo};
}

// split_f64_finite for positive values inside the df operating range (no zero test)
__device__ __forceinline__ df split_f64_pos(double x) {
    const unsigned lo = (unsigned)__double2loint(x);
    const unsigned hi = (unsigned)__double2hiint(x);
    const unsigned fh = ((hi - (896u << 20)) << 3) | (lo >> 29);
    const unsigned base = (fh & 0xFF800000u) - (23u << 23);
    const float flo = __fsub_rn(__uint_as_float(base | ((lo >> 6) & 0x7FFFFFu)), __uint_as_float(base));
    return {__uint_as_float(fh), flo};
}

// Lazily normalised df accumulator: the high part is kept exact with TwoSum, the low parts
// are summed in float and folded in when the accumulator is flushed (a few dozen terms at
// most), which costs 8 FP32 operations per term instead of the 11 of df_add.
struct LazyDf {
    float hi, lo;
};
__device__ __forceinline__ void lazy_add(LazyDf& a, df x) {
    const df s = two_sum(a.hi, x.hi);
    a.hi = s.hi;
    a.lo = __fadd_rn(a.lo, __fadd_rn(s.lo, x.lo));
}
__device__ __forceinline__ double lazy_value(LazyDf a) { return (double)a.hi + (double)a.lo; }
// float -> double on the integer pipe for every finite float, subnormals included (normalised
// by the position of their leading one)
__device__ __forceinline__ double f32_to_f64_bits_all(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned m = u & 0x7FFFFFu;
    if ((u & 0x7F800000u) != 0u || m == 0u) return f32_to_f64_bits(f);
    const int p = 31 - __clz((int)m);  // f = m 2^-149, leading one at bit p
    const unsigned long long bits = ((unsigned long long)(u & 0x80000000u) << 32) |
                                    ((unsigned long long)(p + 874) << 52) |
                                    ((unsigned long long)(m ^ (1u << p)) << (52 - p));
    return __longlong_as_double((long long)bits);
}
// df -> double as df_to_f64 (one FP64 add) with the parts widened on the integer pipe, exact for
// every finite part (pass-end sums; the per-element conversion is df_to_f64_int)
__device__ __forceinline__ double df_to_f64_int_all(df a) { return f32_to_f64_bits_all(a.hi) + f32_to_f64_bits_all(a.lo); }
// the same sum as lazy_value with the parts widened on the integer pipe (one FP64 add, no
// conversion instruction: F2F runs on the FP64 pipe, this GPU's scarce unit)
__device__ __forceinline__ double lazy_value_int(LazyDf a) {
    return f32_to_f64_bits_all(a.hi) + f32_to_f64_bits_all(a.lo);
}

// true iff x is 0, +-inf (when allow_inf) or a finite value with 2^-60 <= |x| <= 2^60
__device__ __forceinline__ bool df_in_range(double x, bool allow_inf) {
    unsigned hi = hi_word(x);
    unsigned lo = lo_word(x);
    unsigned e = (hi >> 20) & 0x7FFu;
    bool zero = ((hi & 0x7FFFFFFFu) | lo) == 0u;
    bool inf = allow_inf && ((hi & 0x7FFFFFFFu) == 0x7FF00000u) && (lo == 0u);
    return zero || inf || (e - 963u <= 120u);
}

// ------------------------------------------------------------------------------------------
// Exact comparison y > c of doubles on bit patterns (no FP64 instruction).  For c < 0 the
// relation is an unsigned compare of the bit patterns, for c >= 0 a signed one.  -0
// thresholds are canonicalised to +0 so that the result equals the IEEE relation y > c for
// every non-NaN y (including y = +-0).
struct GtThreshold {
    unsigned long long bits;
    bool neg;
};
__device__ __forceinline__ GtThreshold make_gt(double c) {
    unsigned long long b = opaque_bits(c);
    if ((b << 1) == 0ull) b = 0ull;  // -0 -> +0
    GtThreshold t;
    t.bits = b;
    t.neg = (b >> 63) != 0ull;
    return t;
}
__device__ __forceinline__ bool gt_bits(unsigned long long ybits, const GtThreshold& t) {
    return t.neg ? (ybits < t.bits) : ((long long)ybits > (long long)t.bits);
}

// Order-preserving integer key of a double (non-NaN): x < y  <=>  key(x) < key(y) (as signed
// 64-bit integers; -0 and +0 map to adjacent keys).  Used for max/min without FP64 instructions.
__device__ __forceinline__ long long order_key(double x) {
    const long long b = (long long)opaque_bits(x);
    return b >= 0 ? b : (long long)(0x8000000000000000ull - (unsigned long long)b) - 1;
}
__device__ __forceinline__ double from_order_key(long long k) {
    return __longlong_as_double(k >= 0 ? k : (long long)(0x8000000000000000ull - (unsigned long long)(k + 1)));
}

// FP64 classification on the bit pattern (integer pipe).
__device__ __forceinline__ bool u64_is_nan(unsigned long long b) {
    const unsigned h = (unsigned)(b >> 32) & 0x7FFFFFFFu, l = (unsigned)b;
    return (h > 0x7FF00000u) | ((h == 0x7FF00000u) & (l != 0u));
}
__device__ __forceinline__ bool f64_is_nan(double x) {
    const unsigned h = hi_word(x) & 0x7FFFFFFFu;
    return (h > 0x7FF00000u) | ((h == 0x7FF00000u) & (lo_word(x) != 0u));
}
__device__ __forceinline__ bool f64_is_finite(double x) { return (hi_word(x) & 0x7FF00000u) != 0x7FF00000u; }
// finite and > 0
__device__ __forceinline__ bool f64_pos_finite(double x) {
    const unsigned h = hi_word(x);
    return ((int)h >= 0) & (h < 0x7FF00000u) & ((h | lo_word(x)) != 0u);
}

// Largest float <= c: for a float y, y > c  <=>  y > rd(c).
__device__ __forceinline__ float f32_rd(double c) { return __double2float_rd(c); }
// Smallest float >= c: for a float y, y >= c  <=>  y >= ru(c).
__device__ __forceinline__ float f32_ru(double c) { return __double2float_ru(c); }

// ------------------------------------------------------------------------------------------
// Warp reductions with a fixed order (deterministic).
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ------------------------------------------------------------------------------------------
// Time and bounded waits.
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Device-wide barrier for a co-resident (cooperatively launched) grid.  `count` only
// grows; a barrier completes when it reaches `target` (the caller adds gridDim.x per
// barrier).  Every wait is bounded by limit_ns; on expiry the block sets *error and the
// function returns false (the caller must leave the kernel).  Called by all threads of
// the block.
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned target, int* error,
                                             unsigned long long limit_ns, int timeout_code) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        // the release orders this block's writes (ordered before it by the block barrier)
        // before the arrival; the acquire orders the other blocks' writes before the block
        // barrier that ends the wait
        red_release_add_u32(count, 1u);
        int ok = 1;
        unsigned long long t0 = globaltimer_ns();
        while (ld_acquire_u32(count) < target) {
            if (globaltimer_ns() - t0 > limit_ns) {
                atomicExch(error, timeout_code);
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Coherent load of data written by other blocks during this launch (bypasses L1).
__device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }

}  // namespace cqk
