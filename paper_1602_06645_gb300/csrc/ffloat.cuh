// Float-float ("double-single") arithmetic: a value is the unevaluated sum
// hi + lo of two binary32 numbers, about 48 significant bits.  Built from the
// error-free transformations of Knuth (TwoSum: a + b = s + e exactly) and
// Dekker (FastTwoSum, for |a| >= |b|), with the product error taken by one
// fused multiply-add (a * b = p + fmaf(a, b, -p) exactly, Ogita, Rump and
// Oishi 2005).  Correct only without contraction or reassociation of the
// written operations: the library is compiled with --fmad=false and no
// fast-math.
#pragma once

namespace tsdf {

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // |a| >= |b| (or a == 0)
    const float s = a + b;
    return {s, b - (s - a)};
}

__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ ff two_prod(float a, float b) {
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const ff s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ ff ff_add(ff a, float b) {
    const ff s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, s.lo + a.lo);
}

__device__ __forceinline__ ff ff_mul(ff a, float b) {
    const ff p = two_prod(a.hi, b);
    return fast_two_sum(p.hi, fmaf(a.lo, b, p.lo));
}

// y = R x + t for one row r of a binary32 3x3 R and t, x in float-float.
__device__ __forceinline__ ff ff_row(const float* R, float t, const ff x[3]) {
    ff acc = ff_mul(x[0], R[0]);
    acc = ff_add(acc, ff_mul(x[1], R[1]));
    acc = ff_add(acc, ff_mul(x[2], R[2]));
    return ff_add(acc, t);
}

// a / b to float-float accuracy: q = hi(a) / hi(b) corrected once by the
// residual a - q b (computed in float-float).
__device__ __forceinline__ ff ff_div(ff a, ff b) {
    const float q = __fdiv_rn(a.hi, b.hi);
    const ff qb = two_prod(q, b.hi);
    const ff r = ff_add(a, ff{-qb.hi, -fmaf(q, b.lo, qb.lo)});
    return fast_two_sum(q, __fdiv_rn(r.hi, b.hi));
}

}  // namespace tsdf
