// Float-float ("double-float") arithmetic: a value is hi + lo with two floats,
// |lo| <= ulp(hi)/2, about 48 significant bits, built from the error-free
// transforms two-sum (Knuth) and two-product (with a fused multiply-add), as in
// Dekker (1971) and the double-double literature (Hida, Li & Bailey, 2001).
// GB300 executes FP32 at many times its FP64 rate, so transcendental work that
// needs more than FP32 but not the full FP64 accuracy runs faster this way.
//
// Included by device code and, for testing, by host C++ (plain IEEE float
// arithmetic without reassociation is all that is assumed).
#pragma once
#include <math.h>

#include <cmath>

#ifdef __CUDACC__
#define DF_HD __host__ __device__ __forceinline__
#else
#define DF_HD inline
#endif

namespace fbim {
namespace dfl {

struct df {
    float hi, lo;
};

DF_HD float fma_f(float a, float b, float c) {
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return std::fmaf(a, b, c);
#endif
}

DF_HD df from_double(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}
DF_HD double to_double(df a) { return (double)a.hi + (double)a.lo; }

// s + e = a + b exactly
DF_HD df two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
// same when |a| >= |b|
DF_HD df quick_two_sum(float a, float b) {
    const float s = a + b;
    return {s, b - (s - a)};
}
// p + e = a b exactly
DF_HD df two_prod(float a, float b) {
    const float p = a * b;
    return {p, fma_f(a, b, -p)};
}

DF_HD df add(df a, df b) {
    const df s = two_sum(a.hi, b.hi);
    const df t = two_sum(a.lo, b.lo);
    df u = quick_two_sum(s.hi, s.lo + t.hi);
    return quick_two_sum(u.hi, u.lo + t.lo);
}
// Cheaper sum (one two-sum on the leading parts): error bounded relative to
// |a| + |b| rather than |a + b|; used inside recurrences whose terms stay bounded.
DF_HD df add_fast(df a, df b) {
    const df s = two_sum(a.hi, b.hi);
    return quick_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
DF_HD df neg(df a) { return {-a.hi, -a.lo}; }
DF_HD df sub(df a, df b) { return add(a, neg(b)); }
DF_HD df add_f(df a, float b) {
    const df s = two_sum(a.hi, b);
    return quick_two_sum(s.hi, s.lo + a.lo);
}
DF_HD df mul(df a, df b) {
    df p = two_prod(a.hi, b.hi);
    p.lo = fma_f(a.hi, b.lo, fma_f(a.lo, b.hi, p.lo));
    return quick_two_sum(p.hi, p.lo);
}
DF_HD df mul_f(df a, float b) {
    df p = two_prod(a.hi, b);
    p.lo = fma_f(a.lo, b, p.lo);
    return quick_two_sum(p.hi, p.lo);
}
DF_HD df div(df a, df b) {
    const float q1 = a.hi / b.hi;
    const df r = sub(a, mul_f(b, q1));
    const float q2 = r.hi / b.hi;
    const df r2 = sub(r, mul_f(b, q2));
    const float q3 = r2.hi / b.hi;
    const df q = quick_two_sum(q1, q2);
    return add_f(q, q3);
}

// ln 2 = L2_HI + L2_MID + L2_LO; L2_HI has 16 significant bits, so n L2_HI is exact
// for |n| < 2^8.
constexpr float L2_HI = 0.693145751953125f;
constexpr float L2_MID = 1.428606765330187e-06f;
constexpr float L2_LO = 5.495603971894525e-14f;

DF_HD df n_ln2(float n) {
    return add(df{n * L2_HI, 0.0f}, add(two_prod(L2_MID, n), df{n * L2_LO, 0.0f}));
}

DF_HD float round_f(float x) {
#ifdef __CUDA_ARCH__
    return rintf(x);
#else
    return std::nearbyint(x);
#endif
}

// 1/k!, k = 0..14, and 1/(2k+1), k = 0..9, as float-float pairs
#ifdef __CUDA_ARCH__
#define DF_TABLE __device__ const
#else
#define DF_TABLE static const
#endif
DF_TABLE float kInvFact[15][2] = {
    {1.000000000e+00f, 0.000000000e+00f},   {1.000000000e+00f, 0.000000000e+00f},
    {5.000000000e-01f, 0.000000000e+00f},   {1.666666716e-01f, -4.967053879e-09f},
    {4.166666791e-02f, -1.241763470e-09f},  {8.333333768e-03f, -4.346172033e-10f},
    {1.388888923e-03f, -3.363109444e-11f},  {1.984127011e-04f, -2.725596875e-12f},
    {2.480158764e-05f, -3.406996094e-13f},  {2.755731884e-06f, 3.793571224e-14f},
    {2.755731998e-07f, -7.575112209e-15f},  {2.505210794e-08f, 4.417623045e-16f},
    {2.087675588e-09f, 1.108283981e-16f},   {1.605904437e-10f, -5.352526512e-18f},
    {1.147074536e-11f, 2.372207689e-19f}};
DF_TABLE float kInvOdd[10][2] = {
    {1.000000000e+00f, 0.000000000e+00f},  {3.333333433e-01f, -9.934107759e-09f},
    {2.000000030e-01f, -2.980232283e-09f}, {1.428571492e-01f, -6.386212004e-09f},
    {1.111111119e-01f, -8.278422947e-10f}, {9.090909362e-02f, -2.709302116e-09f},
    {7.692307979e-02f, -2.865607973e-09f}, {6.666667014e-02f, -3.476937627e-09f},
    {5.882352963e-02f, -2.191347243e-10f}, {5.263157934e-02f, -3.921358238e-10f}};

// e^{-z} for 0 <= z <= 80: z = n ln2 + r, |r| <= ln2/2, e^{-r} by its Taylor series
// (15 terms, truncation below 1e-18), times 2^{-n}.
DF_HD df exp_neg(df z) {
    const float n = round_f(z.hi * 1.44269504088896341f);
    const df mr = sub(n_ln2(n), z);  // -r
    df t = {kInvFact[14][0], kInvFact[14][1]};
#pragma unroll
    for (int k = 13; k >= 0; --k) t = add_fast(mul(t, mr), df{kInvFact[k][0], kInvFact[k][1]});
    return {ldexpf(t.hi, -(int)n), ldexpf(t.lo, -(int)n)};
}

// ln x for x > 0: ln(hi) + lo/hi; ln(hi) = e ln2 + ln m, m in [1/sqrt2, sqrt2), and
// ln m = 2 atanh(u) = 2 u sum_k u^{2k}/(2k+1) with u = (m-1)/(m+1), |u| <= 0.172
// (terms to u^18, truncation below 1e-15 of ln m).
DF_HD df log(df x) {
    int e = 0;
    float m = frexpf(x.hi, &e);  // x.hi = m 2^e, m in [0.5, 1)
    if (m < 0.70710678f) {
        m *= 2.0f;
        e -= 1;
    }
    const df num = {m - 1.0f, 0.0f};  // exact (Sterbenz)
    const df den = two_sum(m, 1.0f);
    const df u = div(num, den);
    const df v = mul(u, u);
    df s = {kInvOdd[9][0], kInvOdd[9][1]};
#pragma unroll
    for (int k = 8; k >= 0; --k) s = add_fast(mul(s, v), df{kInvOdd[k][0], kInvOdd[k][1]});
    const df lm = mul(mul_f(u, 2.0f), s);
    const df r = add(n_ln2((float)e), lm);
    return add_f(r, x.lo / x.hi);
}

}  // namespace dfl
}  // namespace fbim

