// Double-float ("float-float") arithmetic: a value is the unevaluated sum h + l of two
// binary32 numbers with |l| <= ulp(h) / 2, giving about 48 significant bits from FP32
// instructions only (GB300's FP64 rate is a small fraction of its FP32 rate).
//
// The error-free transformations are the published ones: Knuth's two-sum (TAOCP vol. 2,
// 4.2.2), Dekker's fast two-sum for |a| >= |b| (Dekker 1971, "A floating-point technique
// for extending the available precision"), and the product error of a fused multiply-add
// (the exact residual a*b - fl(a*b)).  Sums, products and quotients of double-float
// values follow the usual compositions of these (as in Dekker 1971 and Hida, Li and
// Bailey 2001); each result is renormalised so that h = fl(h + l).
//
// The explicit __fadd_rn / __fmul_rn intrinsics keep the compiler from contracting or
// reassociating the steps whose rounding errors are being captured.
#pragma once

#include <cuda_runtime.h>

namespace ms {

struct dfl {
    float h, l;
};

__device__ __forceinline__ dfl df_make(float h) { return dfl{h, 0.0f}; }

// s + e == a + b exactly (Knuth).
__device__ __forceinline__ dfl df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return dfl{s, e};
}

// s + e == a + b exactly, given |a| >= |b| or a == 0 (Dekker).
__device__ __forceinline__ dfl df_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return dfl{s, __fsub_rn(b, __fsub_rn(s, a))};
}

// p + e == a * b exactly (FMA residual).
__device__ __forceinline__ dfl df_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return dfl{p, fmaf(a, b, -p)};
}

__device__ __forceinline__ dfl df_neg(dfl a) { return dfl{-a.h, -a.l}; }

// a + b, both double-float: two-sums of the high and of the low parts, renormalised.
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
    dfl s = df_two_sum(a.h, b.h);
    const dfl t = df_two_sum(a.l, b.l);
    s.l = __fadd_rn(s.l, t.h);
    s = df_fast_two_sum(s.h, s.l);
    s.l = __fadd_rn(s.l, t.l);
    return df_fast_two_sum(s.h, s.l);
}

__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }

// a + b with one two-sum of the high parts and the low parts added in binary32: error
// O(u^2 (|a| + |b|)), enough wherever the result is not a near-total cancellation that
// must keep its own full relative precision.
__device__ __forceinline__ dfl df_add_fast(dfl a, dfl b) {
    const dfl s = df_two_sum(a.h, b.h);
    return df_fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}

__device__ __forceinline__ dfl df_add_f(dfl a, float b) {
    dfl s = df_two_sum(a.h, b);
    s.l = __fadd_rn(s.l, a.l);
    return df_fast_two_sum(s.h, s.l);
}

// a * b: exact product of the high parts plus the cross terms (the l * l term is below
// the precision kept).
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
    dfl p = df_two_prod(a.h, b.h);
    p.l = fmaf(a.h, b.l, p.l);
    p.l = fmaf(a.l, b.h, p.l);
    return df_fast_two_sum(p.h, p.l);
}

__device__ __forceinline__ dfl df_mul_f(dfl a, float b) {
    dfl p = df_two_prod(a.h, b);
    p.l = fmaf(a.l, b, p.l);
    return df_fast_two_sum(p.h, p.l);
}

// a / b: a first quotient from the high parts, the residual a - q1 b in double-float,
// and a correction quotient of the residual.
__device__ __forceinline__ dfl df_div(dfl a, dfl b) {
    const float q1 = __fdiv_rn(a.h, b.h);
    const dfl r = df_sub(a, df_mul_f(b, q1));
    const float q2 = __fdiv_rn(r.h, b.h);
    return df_fast_two_sum(q1, q2);
}

// a / b from one reciprocal of b.h: q1 = a.h / b.h to a few units, the residual a - q1 b
// from two FMAs (the high one exact or nearly so), and a correction quotient.
__device__ __forceinline__ dfl df_div_rcp(dfl a, dfl b) {
    const float r = __frcp_rn(b.h);
    const float q1 = __fmul_rn(a.h, r);
    const float res = __fadd_rn(fmaf(-q1, b.h, a.h), fmaf(-q1, b.l, a.l));
    return df_fast_two_sum(q1, __fmul_rn(res, r));
}

// Value order of normalised double-float numbers: lexicographic on (h, l).
__device__ __forceinline__ bool df_lt(dfl a, dfl b) { return a.h < b.h || (a.h == b.h && a.l < b.l); }

// Nearest binary32 value of h + l.
__device__ __forceinline__ float df_round(dfl a) { return __fadd_rn(a.h, a.l); }

// floor(h + l) as a binary32 integer value.
__device__ __forceinline__ float df_floor(dfl a) {
    const float f = floorf(a.h);
    return (f == a.h && a.l < 0.0f) ? f - 1.0f : f;
}

// Dot product of a binary32 row r with a double-float vector (dx, dy, dz).
__device__ __forceinline__ dfl df_dot3(const float *r, dfl dx, dfl dy, dfl dz) {
    return df_add(df_add(df_mul_f(dx, r[0]), df_mul_f(dy, r[1])), df_mul_f(dz, r[2]));
}

}  // namespace ms
