// Double-word FP32 arithmetic: a value is hi + lo (two floats, |lo| <= ulp(hi)/2, about 48
// significant bits).  Built from error-free transformations: Knuth's TwoSum, the FMA TwoProduct,
// Dekker's Fast2Sum, and the double-word sums and products of Joldes, Muller and Popescu, "Tight
// and rigorous error bounds for basic building blocks of double-word arithmetic" (ACM TOMS, 2017).
// Dot products accumulate as in Ogita, Rump and Oishi, "Accurate sum and dot product" (SIAM J.
// Sci. Comput., 2005), Dot2: the high parts of the products are summed by TwoSum, the errors of
// the products and of the sums in a second float.
//
// GB300 issues 128 FP32 FMAs per clock per SM against about 2 FP64 FMAs, so FP64-accurate work
// done this way on the FP32 pipe runs several times faster than plain FP64.  The _rn intrinsics
// keep the compiler from contracting or reassociating the transformations.
#pragma once

namespace rte {

struct DW {
    float h, l;
};

__device__ __forceinline__ DW dw_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
    return DW{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DW dw_fast_two_sum(float a, float b) {   // |a| >= |b| or a == 0
    const float s = __fadd_rn(a, b);
    return DW{s, __fsub_rn(b, __fsub_rn(s, a))};
}
// sum of two double-words (the cheap form: small absolute error against |x| + |y| even where
// x and y cancel)
__device__ __forceinline__ DW dw_add(DW x, DW y) {
    const DW s = dw_two_sum(x.h, y.h);
    return dw_fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l)));
}
__device__ __forceinline__ DW dw_mul_f(DW x, float a) {             // x * a, a exact in FP32
    const float p = __fmul_rn(x.h, a);
    const float e = __fmaf_rn(x.h, a, -p);
    return dw_fast_two_sum(p, __fmaf_rn(x.l, a, e));
}
__device__ __forceinline__ DW dw_mul(DW x, DW y) {
    const float p = __fmul_rn(x.h, y.h);
    const float e = __fmaf_rn(x.h, y.h, -p);
    return dw_fast_two_sum(p, __fadd_rn(e, __fmaf_rn(x.l, y.h, __fmul_rn(x.h, y.l))));
}
__device__ __forceinline__ DW dw_of(double v) {
    const float h = (float)v;
    return DW{h, (float)(v - (double)h)};
}
__device__ __forceinline__ DW dw_neg(DW x) { return DW{-x.h, -x.l}; }
__device__ __forceinline__ double dw_to_double(DW x) { return (double)x.h + (double)x.l; }   // exact
__device__ __forceinline__ DW dw_load(const float2* p) {
    const float2 v = *p;
    return DW{v.x, v.y};
}
__device__ __forceinline__ void dw_store(float2* p, DW x) { *p = make_float2(x.h, x.l); }

// Dot2 step: acc += x * y.  acc.h carries the TwoSum of the high product parts, acc.l the
// rounding errors (product error by FMA, cross terms x.h y.l + x.l y.h, sum error); the
// x.l y.l term (2^-48 relative) is dropped.  Normalise with dw_norm before using acc.
__device__ __forceinline__ void dw_mac(DW& acc, DW x, DW y) {
    const float p = __fmul_rn(x.h, y.h);
    float e = __fmaf_rn(x.h, y.h, -p);
    e = __fmaf_rn(x.h, y.l, e);
    e = __fmaf_rn(x.l, y.h, e);
    const DW s = dw_two_sum(acc.h, p);
    acc.h = s.h;
    acc.l = __fadd_rn(acc.l, __fadd_rn(s.l, e));
}
__device__ __forceinline__ DW dw_norm(DW acc) { return dw_fast_two_sum(acc.h, acc.l); }

__device__ __forceinline__ DW dw_warp_sum(DW v) {
    for (int o = 16; o > 0; o >>= 1) {
        const DW w{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
        v = dw_add(v, w);
    }
    return v;
}

}  // namespace rte
