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
__device__ __forceinline__ dw dw_neg(dw x) { return {-x.h, -x.l}; }
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

__device__ __forceinline__ cdw cdw_add(const cdw& a, const cdw& b) { return {dw_add(a.x, b.x), dw_add(a.y, b.y)}; }
__device__ __forceinline__ cdw cdw_sub(const cdw& a, const cdw& b) { return {dw_sub(a.x, b.x), dw_sub(a.y, b.y)}; }
__device__ __forceinline__ cdw cdw_pow2(const cdw& a, float p2) { return {dw_pow2(a.x, p2), dw_pow2(a.y, p2)}; }
__device__ __forceinline__ cdw cdw_zero() { return {{0.f, 0.f}, {0.f, 0.f}}; }
// storage: one float4 per complex node value {re.h, re.l, im.h, im.l}
__device__ __forceinline__ cdw cdw_ld(const float4* p) {
    const float4 v = *p;
    return {{v.x, v.y}, {v.z, v.w}};
}
__device__ __forceinline__ void cdw_st(float4* p, const cdw& a) { *p = make_float4(a.x.h, a.x.l, a.y.h, a.y.l); }

}  // namespace ddnls
