// df.cuh -- compensated FP32 arithmetic ("double-float": an unevaluated sum
// hi + lo of two floats, ~48 significant bits) built from the error-free
// transformations of Knuth (TwoSum), Dekker (FastTwoSum) and the FMA-based
// TwoProduct.  Used where FP32 alone cannot hold the geometry to the force
// tolerance: probe positions of ~4 cm must be known to ~1e-10 m so that
// k * depth (k = 1e4 N/m) stays within 1e-6 N.  No FP64 instruction is
// issued on the GPU.
#pragma once
#include <cuda_runtime.h>

struct df {
    float hi, lo;
};

__host__ __device__ __forceinline__ df df_from(float a) { return df{a, 0.0f}; }

__device__ __forceinline__ df two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return df{s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {  // |a| >= |b|
    float s = a + b;
    float e = b - (s - a);
    return df{s, e};
}

__device__ __forceinline__ df two_prod(float a, float b) {
    float p = a * b;
    float e = __fmaf_rn(a, b, -p);
    return df{p, e};
}

__device__ __forceinline__ df df_add(df x, df y) {
    df s = two_sum(x.hi, y.hi);
    df t = two_sum(x.lo, y.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}

// x + y with a single TwoSum, on the high parts.  Its error is at most
// ~2^-23 (|x.lo| + |y.lo|) + 2^-46 |x + y|: the accurate df_add's bound as
// a relative one, except where the high parts cancel, where it stays this
// absolute bound.  For query points and interpolated distances of a few
// centimetres, needed to ~1e-12 m, that is ~1e-15 m.
__device__ __forceinline__ df df_add_abs(df x, df y) {
    df s = two_sum(x.hi, y.hi);
    s.lo += x.lo + y.lo;
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_neg(df x) { return df{-x.hi, -x.lo}; }
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }
__device__ __forceinline__ df df_add_f(df x, float b) {
    df s = two_sum(x.hi, b);
    s.lo += x.lo;
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_mul(df x, df y) {
    df p = two_prod(x.hi, y.hi);
    p.lo = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, p.lo));
    return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ df df_mul_f(df x, float b) {
    df p = two_prod(x.hi, b);
    p.lo = __fmaf_rn(x.lo, b, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

// x / y by one Newton correction of the float quotient
__device__ __forceinline__ df df_div(df x, df y) {
    float q1 = x.hi / y.hi;
    df r = df_sub(x, df_mul_f(y, q1));
    float q2 = r.hi / y.hi;
    return fast_two_sum(q1, q2);
}

__device__ __forceinline__ df df_div_f(df x, float b) {
    float q1 = x.hi / b;
    df r = df_sub(x, two_prod(q1, b));
    float q2 = r.hi / b;
    return fast_two_sum(q1, q2);
}

// sqrt by one Newton correction of the float root: s + (x - s^2) / (2 s)
__device__ __forceinline__ df df_sqrt(df x) {
    if (!(x.hi > 0.0f)) return df{0.0f, 0.0f};
    float s = sqrtf(x.hi);
    df s2 = two_prod(s, s);
    float r = ((x.hi - s2.hi) - s2.lo + x.lo) / (2.0f * s);
    return fast_two_sum(s, r);
}

__device__ __forceinline__ bool df_lt(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool df_gt(df a, df b) { return df_lt(b, a); }
__device__ __forceinline__ bool df_le(df a, df b) { return !df_lt(b, a); }

// integer part of x rounded toward -inf (x well inside the int range)
__device__ __forceinline__ int df_floor_int(df x) {
    float f = floorf(x.hi);
    int i = (int)f;
    if (f == x.hi && x.lo < 0.0f) i -= 1;
    return i;
}

// 3-vectors
struct df3 {
    df x, y, z;
};

__device__ __forceinline__ df df_dot3(df3 a, df3 b) {
    return df_add(df_add(df_mul(a.x, b.x), df_mul(a.y, b.y)), df_mul(a.z, b.z));
}
__device__ __forceinline__ df3 df3_sub(df3 a, df3 b) { return df3{df_sub(a.x, b.x), df_sub(a.y, b.y), df_sub(a.z, b.z)}; }
__device__ __forceinline__ df3 df3_add(df3 a, df3 b) { return df3{df_add(a.x, b.x), df_add(a.y, b.y), df_add(a.z, b.z)}; }
__device__ __forceinline__ df3 df3_scale(df3 a, df s) { return df3{df_mul(a.x, s), df_mul(a.y, s), df_mul(a.z, s)}; }
__device__ __forceinline__ df3 df3_cross(df3 a, df3 b) {
    return df3{df_sub(df_mul(a.y, b.z), df_mul(a.z, b.y)), df_sub(df_mul(a.z, b.x), df_mul(a.x, b.z)),
               df_sub(df_mul(a.x, b.y), df_mul(a.y, b.x))};
}
__device__ __forceinline__ df3 df3_from(float x, float y, float z) { return df3{df_from(x), df_from(y), df_from(z)}; }

// sin and cos of a compensated angle: reduction by multiples of pi/2 (pi/2
// held as a float pair), then the Taylor series on |r| <= pi/4 by Horner's
// rule in r^2 up to the r^17 / r^18 terms (the first omitted term is below
// 2^-50).  inv_fact(n) is 1/n! as a float pair, folded from the
// definition at compile time.
struct DfConst {
    float hi, lo;
};
constexpr double kFactD[19] = {1.0, 1.0, 2.0, 6.0, 24.0, 120.0, 720.0, 5040.0, 40320.0, 362880.0, 3628800.0,
                               39916800.0, 479001600.0, 6227020800.0, 87178291200.0, 1307674368000.0,
                               20922789888000.0, 355687428096000.0, 6402373705728000.0};
__host__ __device__ constexpr DfConst inv_fact(int n) {
    return DfConst{(float)(1.0 / kFactD[n]), (float)(1.0 / kFactD[n] - (double)(float)(1.0 / kFactD[n]))};
}

__device__ inline void df_sincos(df x, df* s_out, df* c_out) {
    const df PIO2 = df{1.57079637050628662109375f, -4.37113882867379213008e-08f};
    float kf = rintf(x.hi / PIO2.hi);
    df r = df_sub(x, df_mul_f(PIO2, kf));
    df r2 = df_mul(r, r);
    // sin r = r (1 - r^2/3! + r^4/5! - ...), cos r = 1 - r^2/2! + r^4/4! - ...
    constexpr DfConst s17 = inv_fact(17), s15 = inv_fact(15), s13 = inv_fact(13), s11 = inv_fact(11), s9 = inv_fact(9),
                      s7 = inv_fact(7), s5 = inv_fact(5), s3 = inv_fact(3);
    constexpr DfConst c18 = inv_fact(18), c16 = inv_fact(16), c14 = inv_fact(14), c12 = inv_fact(12), c10 = inv_fact(10),
                      c8 = inv_fact(8), c6 = inv_fact(6), c4 = inv_fact(4), c2 = inv_fact(2);
    df ps = df{s17.hi, s17.lo};
    ps = df_sub(df{s15.hi, s15.lo}, df_mul(r2, ps));
    ps = df_sub(df{s13.hi, s13.lo}, df_mul(r2, ps));
    ps = df_sub(df{s11.hi, s11.lo}, df_mul(r2, ps));
    ps = df_sub(df{s9.hi, s9.lo}, df_mul(r2, ps));
    ps = df_sub(df{s7.hi, s7.lo}, df_mul(r2, ps));
    ps = df_sub(df{s5.hi, s5.lo}, df_mul(r2, ps));
    ps = df_sub(df{s3.hi, s3.lo}, df_mul(r2, ps));
    ps = df_sub(df_from(1.0f), df_mul(r2, ps));
    const df s = df_mul(r, ps);
    df pc = df{c18.hi, c18.lo};
    pc = df_sub(df{c16.hi, c16.lo}, df_mul(r2, pc));
    pc = df_sub(df{c14.hi, c14.lo}, df_mul(r2, pc));
    pc = df_sub(df{c12.hi, c12.lo}, df_mul(r2, pc));
    pc = df_sub(df{c10.hi, c10.lo}, df_mul(r2, pc));
    pc = df_sub(df{c8.hi, c8.lo}, df_mul(r2, pc));
    pc = df_sub(df{c6.hi, c6.lo}, df_mul(r2, pc));
    pc = df_sub(df{c4.hi, c4.lo}, df_mul(r2, pc));
    pc = df_sub(df{c2.hi, c2.lo}, df_mul(r2, pc));
    const df c = df_sub(df_from(1.0f), df_mul(r2, pc));
    int k = ((int)kf) & 3;
    if (k == 0) { *s_out = s; *c_out = c; }
    else if (k == 1) { *s_out = c; *c_out = df_neg(s); }
    else if (k == 2) { *s_out = df_neg(s); *c_out = df_neg(c); }
    else { *s_out = df_neg(c); *c_out = s; }
}
