// Float-float ("double-float") arithmetic for the complex128 fused kernels.
//
// GB300's FP64 pipe runs at a small fraction of its FP32 rate, so the complex128 tile
// passes keep amplitudes as FP64 in HBM but compute on pairs of floats (hi + lo, an
// unevaluated sum carrying ~48 significant bits) with the FP32 pipe.  The operations are
// built from the classic error-free transformations: Knuth's TwoSum (the exact rounding
// error of a floating-point sum) and the FMA form of Dekker's TwoProduct (the exact
// rounding error of a product, a*b - fl(a*b) = fma(a, b, -fl(a*b))), combined as in the
// double-double literature (Dekker 1971; Hida, Li & Bailey 2001).
//
// Error model.  Addition is the one-TwoSum ("sloppy") form and fma(a, b, c) is fused the
// same way: their absolute error is below about 2^-46 (|a| + |b|), resp. 2^-46 (|a b| + |c|),
// i.e. FP64's own bound u (|a| + |b|) with u = 2^-53 widened by 2^7.  A state-vector update
// only needs this absolute bound (amplitudes are bounded by the state's norm); relative
// accuracy of a sum that cancels to nearly zero is not kept (FP64 does not keep it
// either).  Conversion from FP64 splits d into hi = fl32(d) and lo = fl32(d - hi) (exact
// to 48 bits for |d| in the float range); conversion back is hi + lo in FP64.
#pragma once

#include "common.cuh"

namespace vqg {

struct df {
    float hi, lo;
    df() = default;
    __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr df(int v) : hi((float)v), lo(0.f) {}
    __host__ __device__ constexpr df(float v) : hi(v), lo(0.f) {}
    __device__ df(double d) {
        hi = __double2float_rn(d);
        lo = __double2float_rn(d - (double)hi);
    }
    __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly (Knuth's TwoSum, no magnitude condition)
VQG_DEV void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e = a + b exactly when |a| >= |b| or a == 0
VQG_DEV void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

VQG_DEV df operator+(df a, df b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    fast_two_sum(s, e, s, e);
    return df(s, e);
}
VQG_DEV df operator-(df a) { return df(-a.hi, -a.lo); }
VQG_DEV df operator-(df a, df b) { return a + (-b); }
VQG_DEV df operator*(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);                    // exact error of the product
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));    // cross terms (a.lo * b.lo dropped)
    float s;
    fast_two_sum(p, e, s, e);
    return df(s, e);
}
VQG_DEV df &operator+=(df &a, df b) { return a = a + b; }
VQG_DEV df &operator-=(df &a, df b) { return a = a - b; }
VQG_DEV df &operator*=(df &a, df b) { return a = a * b; }
// a * b + c with one normalisation: the product's exact error and cross terms join the
// low part of the sum (a.lo * b.lo is below the error bound and dropped).
VQG_DEV df fma(df a, df b, df c) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    float s, t;
    two_sum(p, c.hi, s, t);
    t = __fadd_rn(t, __fadd_rn(e, c.lo));
    fast_two_sum(s, t, s, t);
    return df(s, t);
}

struct df2 {
    df x, y;
};

// Packed float-float pairs for real-factor updates of a complex amplitude (RY): the real
// and imaginary parts run the same sequence, so each FP32 step is one packed instruction
// (sm_100 and later) on (re, im) lanes.  hi = (x.hi, y.hi), lo = (x.lo, y.lo).
struct dfp {
    float2 hi, lo;
};
VQG_DEV dfp to_dfp(const df2 &a) { return {make_float2(a.x.hi, a.y.hi), make_float2(a.x.lo, a.y.lo)}; }
VQG_DEV df2 from_dfp(const dfp &v) { return {df(v.hi.x, v.lo.x), df(v.hi.y, v.lo.y)}; }
VQG_DEV float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
VQG_DEV void two_sum2(float2 a, float2 b, float2 &s, float2 &e) {
    s = __fadd2_rn(a, b);
    const float2 bb = __fadd2_rn(s, neg2(a));
    e = __fadd2_rn(__fadd2_rn(a, neg2(__fadd2_rn(s, neg2(bb)))), __fadd2_rn(b, neg2(bb)));
}
VQG_DEV void fast_two_sum2(float2 a, float2 b, float2 &s, float2 &e) {
    s = __fadd2_rn(a, b);
    e = __fadd2_rn(b, neg2(__fadd2_rn(s, neg2(a))));
}
// lane-wise a * b + c with a.hi/a.lo given as (possibly broadcast) pairs; same error
// model as fma(df, df, df)
VQG_DEV dfp fma2(float2 ah, float2 al, const dfp &b, const dfp &c) {
    const float2 p = __fmul2_rn(ah, b.hi);
    float2 e = __ffma2_rn(ah, b.hi, neg2(p));
    e = __ffma2_rn(ah, b.lo, __ffma2_rn(al, b.hi, e));
    float2 s, t;
    two_sum2(p, c.hi, s, t);
    t = __fadd2_rn(t, __fadd2_rn(e, c.lo));
    fast_two_sum2(s, t, s, t);
    return {s, t};
}
VQG_DEV dfp mul2(float2 ah, float2 al, const dfp &b) {
    const float2 p = __fmul2_rn(ah, b.hi);
    float2 e = __ffma2_rn(ah, b.hi, neg2(p));
    e = __ffma2_rn(ah, b.lo, __ffma2_rn(al, b.hi, e));
    float2 s;
    fast_two_sum2(p, e, s, e);
    return {s, e};
}

}  // namespace vqg

template <> struct Amp<vqg::df> { using type = vqg::df2; };
