// Double-word ("float-float") arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi)/2, about 48 significant bits carried on the FP32 pipe.
//
// The building blocks are the published ones:
//   2Sum (Knuth; Moller), Fast2Sum (Dekker 1971), the FMA-based exact product;
//   AccurateDWPlusDW, DWTimesFP3 and DWTimesDW3 of M. Joldes, J.-M. Muller, V. Popescu,
//   "Tight and rigorous error bounds for basic building blocks of double-word arithmetic",
//   ACM Trans. Math. Softw. 44(2), 2017 (Algorithms 6, 9 and 12), with relative error bounds
//   3u^2 + 13u^3, 2u^2 and 4u^2 (u = 2^-24) while no operand underflows.
// Every FP32 operation uses an _rn intrinsic, so the compiler neither contracts a product and
// a sum into one FMA nor reorders the error-free transformations.
#pragma once
#include <cuda_runtime.h>

namespace ddnls {

struct dw {
    float h, l;
};
struct cdw {   // complex double-word
    dw x, y;
};

__device__ __forceinline__ dw two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float av = __fsub_rn(s, bv);
    return {s, __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv))};
}
// exact when the exponent of a is at least that of b (or a = 0)
__device__ __forceinline__ dw fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dw dw_add(dw x, dw y) {
    const dw s = two_sum(x.h, y.h);
    const dw t = two_sum(x.l, y.l);
    const dw v = fast_two_sum(s.h, __fadd_rn(s.l, t.h));
    return fast_two_sum(v.h, __fadd_rn(t.l, v.l));
}
// SloppyDWPlusDW (Algorithm 5 of the same paper): 11 operations instead of 20.  Its relative
// error is unbounded when x ~ -y, but its absolute error stays within a few u^2 (|x| + |y|)
// (2Sum is exact; the low words enter with one rounding each), which is the accuracy a
// residual b - A zeta needs: every term is known to u^2 of its own size, not of the result.
__device__ __forceinline__ dw dw_add_s(dw x, dw y) {
    const dw s = two_sum(x.h, y.h);
    const float w = __fadd_rn(s.l, __fadd_rn(x.l, y.l));
    return fast_two_sum(s.h, w);
}
__device__ __forceinline__ dw dw_neg(dw x) { return {-x.h, -x.l}; }
__device__ __forceinline__ dw dw_sub_s(dw x, dw y) { return dw_add_s(x, {-y.h, -y.l}); }
__device__ __forceinline__ dw dw_sub(dw x, dw y) { return dw_add(x, dw_neg(y)); }
__device__ __forceinline__ dw dw_mul_f(dw x, float y) {
    const float ch = __fmul_rn(x.h, y);
    const float cl1 = __fmaf_rn(x.h, y, -ch);
    return fast_two_sum(ch, __fmaf_rn(x.l, y, cl1));
}
__device__ __forceinline__ dw dw_mul(dw x, dw y) {
    const float ch = __fmul_rn(x.h, y.h);
    const float cl1 = __fmaf_rn(x.h, y.h, -ch);
    const float tl1 = __fmaf_rn(x.h, y.l, __fmul_rn(x.l, y.l));
    const float cl2 = __fmaf_rn(x.l, y.h, tl1);
    return fast_two_sum(ch, __fadd_rn(cl1, cl2));
}
// multiplication by a power of two: exact (both words scale)
__device__ __forceinline__ dw dw_pow2(dw x, float p2) { return {__fmul_rn(x.h, p2), __fmul_rn(x.l, p2)}; }
// FP64 -> double word (the FP64 value to within 2^-48 relative) and back
__device__ __forceinline__ dw dw_from(double v) {
    const float h = __double2float_rn(v);
    return {h, __double2float_rn(v - (double)h)};
}
__device__ __forceinline__ double dw_to(dw x) { return (double)x.h + (double)x.l; }
// The same split with integer operations only (GB300 issues FP64 instructions, conversions
// included, at ~1/64 of the FP32 rate): hi = the leading 24 significant bits of v, truncated;
// lo = the next 29 bits, rounded to 24 and scaled by 2^(e-1075) in two exact power-of-two
// steps; then normalized by Fast2Sum.  Exact to 2^-47 relative for 2^-102 <= |v| < 2^128; for
// 2^-126 <= |v| < 2^-102 the low word is FP32-subnormal and the error stays below 2^-149 in
// absolute terms; zero, smaller values and non-finite values take dw_from.
__device__ __forceinline__ dw dw_from_bits(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned e = (unsigned)(b >> 52) & 0x7ffu;
    if (e < 897u || e > 1150u) return dw_from(v);
    const unsigned sgn = (unsigned)(b >> 63) << 31;
    const unsigned long long m = b & 0xfffffffffffffull;
    const float h = __uint_as_float(sgn | ((e - 896u) << 23) | (unsigned)(m >> 29));
    const unsigned k = e >= 949u ? 0u : 64u;
    const float p1 = __uint_as_float((e + k - 948u) << 23);   // 2^(e - 1075 + k)
    const float p2 = __uint_as_float((127u - k) << 23);       // 2^-k
    const float l = __fmul_rn(__fmul_rn(__uint2float_rn((unsigned)(m & 0x1fffffffu)), p1), p2);
    return fast_two_sum(h, __uint_as_float(__float_as_uint(l) | sgn));
}

// 1/b: the FP32 reciprocal r0 refined by one Newton step carried in double words,
// r = r0 + r0 (1 - b r0); relative error O(u^2) while b and 1/b stay normal
__device__ __forceinline__ dw dw_recip(dw b) {
    const float r0 = __frcp_rn(b.h);
    const dw e = dw_sub({1.f, 0.f}, dw_mul_f(b, r0));
    return dw_add({r0, 0.f}, dw_mul_f(e, r0));
}

__device__ __forceinline__ cdw cdw_add(const cdw& a, const cdw& b) { return {dw_add(a.x, b.x), dw_add(a.y, b.y)}; }
// complex products and quotients of double words (the Krylov scalar recurrences)
__device__ __forceinline__ cdw cdw_mul(const cdw& a, const cdw& b) {
    return {dw_sub(dw_mul(a.x, b.x), dw_mul(a.y, b.y)), dw_add(dw_mul(a.x, b.y), dw_mul(a.y, b.x))};
}
__device__ __forceinline__ dw cdw_abs2(const cdw& a) { return dw_add(dw_mul(a.x, a.x), dw_mul(a.y, a.y)); }
// a / b = a conj(b) / |b|^2 with b scaled by a power of two so that |b|^2 neither overflows nor
// underflows; b = 0 gives a non-finite result
__device__ __forceinline__ cdw cdw_div(const cdw& a, const cdw& b) {
    const float m = fmaxf(fabsf(b.x.h), fabsf(b.y.h));
    int e = 0;
    if (m > 0.f && m < INFINITY) e = ((__float_as_int(m) >> 23) & 0xff) - 127;
    e = max(-120, min(120, e));
    const float p2 = __int_as_float((127 - e) << 23);   // 2^-e
    const cdw bs = {dw_pow2(b.x, p2), dw_pow2(b.y, p2)};
    const dw inv = dw_recip(cdw_abs2(bs));
    const cdw t = cdw_mul(a, {bs.x, dw_neg(bs.y)});
    return {dw_pow2(dw_mul(t.x, inv), p2), dw_pow2(dw_mul(t.y, inv), p2)};
}
// 1 / b = conj(b) / |b|^2, with b scaled by a power of two as in cdw_div
__device__ __forceinline__ cdw cdw_recip(const cdw& b) {
    const float m = fmaxf(fabsf(b.x.h), fabsf(b.y.h));
    int e = 0;
    if (m > 0.f && m < INFINITY) e = ((__float_as_int(m) >> 23) & 0xff) - 127;
    e = max(-120, min(120, e));
    const float p2 = __int_as_float((127 - e) << 23);   // 2^-e
    const cdw bs = {dw_pow2(b.x, p2), dw_pow2(b.y, p2)};
    const dw inv = dw_recip(cdw_abs2(bs));
    return {dw_pow2(dw_mul(bs.x, inv), p2), dw_pow2(dw_mul(dw_neg(bs.y), inv), p2)};
}
__device__ __forceinline__ bool cdw_nonzero(const cdw& a) { return a.x.h != 0.f || a.y.h != 0.f; }
__device__ __forceinline__ bool cdw_finite(const cdw& a) { return isfinite(a.x.h) && isfinite(a.y.h); }
__device__ __forceinline__ cdw cdw_sub(const cdw& a, const cdw& b) { return {dw_sub(a.x, b.x), dw_sub(a.y, b.y)}; }
__device__ __forceinline__ cdw cdw_add_s(const cdw& a, const cdw& b) { return {dw_add_s(a.x, b.x), dw_add_s(a.y, b.y)}; }
__device__ __forceinline__ cdw cdw_sub_s(const cdw& a, const cdw& b) { return {dw_sub_s(a.x, b.x), dw_sub_s(a.y, b.y)}; }
__device__ __forceinline__ cdw cdw_pow2(const cdw& a, float p2) { return {dw_pow2(a.x, p2), dw_pow2(a.y, p2)}; }
__device__ __forceinline__ cdw cdw_zero() { return {{0.f, 0.f}, {0.f, 0.f}}; }
// storage: one float4 per complex node value {re.h, re.l, im.h, im.l}
__device__ __forceinline__ cdw cdw_ld(const float4* p) {
    const float4 v = *p;
    return {{v.x, v.y}, {v.z, v.w}};
}
__device__ __forceinline__ void cdw_st(float4* p, const cdw& a) { *p = make_float4(a.x.h, a.x.l, a.y.h, a.y.l); }

}  // namespace ddnls
