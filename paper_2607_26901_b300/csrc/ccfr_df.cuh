// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// binary32 numbers with |lo| <= ulp(hi) / 2, about 48 significant bits.
// Built from error-free transformations:
//   TwoSum (Knuth): s = fl(a + b) and the exact error a + b - s, six adds,
//     no branch, any magnitudes;
//   Fast2Sum (Dekker): the same in three adds when |a| >= |b| (or a = 0);
//   TwoProd: p = fl(a b) and the exact error fma(a, b, -p).
// The sums and products below follow the double-word algorithms analysed by
// Joldes, Muller and Popescu ("Tight and rigorous error bounds for basic
// building blocks of double-word arithmetic", ACM TOMS 2017): relative errors
// of a few u^2 (u = 2^-24), far below what the callers need.  Every step uses
// the explicitly rounded intrinsics so that no contraction or reassociation
// can change them.
#pragma once

namespace ccfr {

struct dfl { float hi, lo; };

__device__ __forceinline__ dfl df_make(float a) { dfl r; r.hi = a; r.lo = 0.f; return r; }

__device__ __forceinline__ dfl two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    dfl r; r.hi = s; r.lo = e; return r;
}

__device__ __forceinline__ dfl fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    dfl r; r.hi = s; r.lo = e; return r;
}

__device__ __forceinline__ dfl two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    dfl r; r.hi = p; r.lo = __fmaf_rn(a, b, -p); return r;
}

// x + y, both double-float (accurate sum: TwoSum on both words).
__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
    const dfl s = two_sum(x.hi, y.hi);
    const dfl t = two_sum(x.lo, y.lo);
    const dfl v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}
__device__ __forceinline__ dfl df_neg(dfl x) { dfl r; r.hi = -x.hi; r.lo = -x.lo; return r; }
__device__ __forceinline__ dfl df_sub(dfl x, dfl y) { return df_add(x, df_neg(y)); }

// x * y, both double-float.
__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
    const dfl c = two_prod(x.hi, y.hi);
    const float t = __fmaf_rn(x.lo, y.hi, __fmul_rn(x.hi, y.lo));
    return fast_two_sum(c.hi, __fadd_rn(c.lo, t));
}

// x * y + z.
__device__ __forceinline__ dfl df_fma(dfl x, dfl y, dfl z) { return df_add(df_mul(x, y), z); }

// x / y: a binary32 quotient estimate q1, the remainder x - q1 y in
// double-float, and a second quotient word from it (long division with one
// correction step; y must be nonzero).
__device__ __forceinline__ dfl df_div(dfl x, dfl y) {
    const float q1 = __fdiv_rn(x.hi, y.hi);
    const dfl r = df_sub(x, df_mul(y, df_make(q1)));
    const float q2 = __fdiv_rn(r.hi, y.hi);
    return fast_two_sum(q1, q2);
}

// Nearest binary32 to x (hi + lo rounded once).
__device__ __forceinline__ float df_to_float(dfl x) { return __fadd_rn(x.hi, x.lo); }

struct df3 { dfl x, y, z; };
__device__ __forceinline__ df3 df3_make(dfl x, dfl y, dfl z) { df3 r; r.x = x; r.y = y; r.z = z; return r; }
__device__ __forceinline__ df3 df3_of(float x, float y, float z) { return df3_make(df_make(x), df_make(y), df_make(z)); }
__device__ __forceinline__ df3 df3_add(df3 a, df3 b) { return df3_make(df_add(a.x, b.x), df_add(a.y, b.y), df_add(a.z, b.z)); }
__device__ __forceinline__ df3 df3_sub(df3 a, df3 b) { return df3_make(df_sub(a.x, b.x), df_sub(a.y, b.y), df_sub(a.z, b.z)); }
__device__ __forceinline__ dfl df3_dot(df3 a, df3 b) { return df_fma(a.x, b.x, df_fma(a.y, b.y, df_mul(a.z, b.z))); }
// s a + b
__device__ __forceinline__ df3 df3_axpy(dfl s, df3 a, df3 b) {
    return df3_make(df_fma(s, a.x, b.x), df_fma(s, a.y, b.y), df_fma(s, a.z, b.z));
}

}  // namespace ccfr
