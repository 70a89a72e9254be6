// lb_mu.cuh -- arithmetic for the chemical potential on GB300.
//
// GB300 issues FP64 at about 1/64 of its FP32 rate, so the chemical-potential
// stage (the only place where the mixed-precision path needs more than FP32:
// eta = 1 - sum b rho, 1/eta and the logarithms) is given two cheaper forms:
//
//  * log64_tbl: an FP64 natural logarithm by table-driven argument reduction
//    (P. T. P. Tang, "Table-driven implementation of the logarithm function in
//    IEEE floating-point arithmetic", ACM TOMS 16(4), 1990): x = 2^e m, m in
//    [c_j, c_j + 1/128) with c_j = 1 + j/128 picked by the top 7 mantissa bits,
//    ln x = e ln 2 - ln r_j + log1p(m r_j - 1), r_j ~ 1/c_j, |m r_j - 1| < 2^-7,
//    log1p by its Taylor series to r^8.  About 13 FP64 instructions instead of a
//    general-purpose log.  Absolute error ~1e-16 max(1, |ln x|), which is what the
//    chemical potential needs (a relative-accuracy special case near x = 1, as in
//    Tang's paper, is not needed and not done).
//  * the "df" (double-float) forms: a value is an unevaluated sum hi + lo of two
//    FP32 numbers (T. J. Dekker, "A floating-point technique for extending the
//    available precision", Numer. Math. 18, 1971; error-free sums after Knuth,
//    products through fused multiply-add).  About 44 significant bits, all on
//    the FP32 pipe; the logarithm uses the same table reduction, with r and r^2/2
//    in df and the series tail r^3/3 - ... - r^6/6 in FP32.
//
// ln 2 splits and the tables -ln r_j are computed on the host in extended
// precision from the decimal expansion of ln 2 and the host's long-double log.
//
// Tables are filled on the host once per context (lb_api.cu) and copied into
// shared memory by every CTA.
#pragma once
#include <cuda_runtime.h>

namespace lbvdw {

constexpr int LOG_TBL = 128;  // sub-intervals of [1, 2)

struct LogTables {
    // FP64 table: r_j = 1/c_j rounded to double, T_j = -ln(r_j) as hi + lo
    double r64[LOG_TBL], t64_hi[LOG_TBL], t64_lo[LOG_TBL];
    // df table: r_j = 1/c_j rounded to float, T_j = -ln(r_j) as float hi + lo
    float r32[LOG_TBL], t32_hi[LOG_TBL], t32_lo[LOG_TBL];
    // ln 2 = hi + lo: FP64 hi short enough that e * hi is exact (|e| < 2^10);
    // float pair = ln 2 rounded to float plus the rounded remainder
    double ln2_hi_d, ln2_lo_d;
    float ln2_hi_f, ln2_lo_f;
};

// Fill the tables on the host (lb_api.cu).
void fill_log_tables(LogTables *t);

// ------------------------------------------------------------------ FP64 log
// x > 0, finite, normal.  s_r/s_hi/s_lo: the FP64 table in shared memory.
__device__ __forceinline__ double log64_tbl(double x, const double *s_r, const double *s_hi, const double *s_lo,
                                            double ln2_hi, double ln2_lo) {
    long long bits = __double_as_longlong(x);
    int e = (int)((bits >> 52) & 0x7ff) - 1023;
    long long mbits = (bits & 0x000fffffffffffffLL) | 0x3ff0000000000000LL;  // m in [1, 2)
    int j = (int)((bits >> 45) & (LOG_TBL - 1));                            // top 7 mantissa bits
    double m = __longlong_as_double(mbits);
    double r = fma(m, s_r[j], -1.0);  // m r_j - 1 in [0, 2^-7), rounded once
    // log1p(r) = r - r^2/2 + r^3/3 - ... - r^8/8
    double p = fma(r, -1.0 / 8.0, 1.0 / 7.0);
    p = fma(r, p, -1.0 / 6.0);
    p = fma(r, p, 1.0 / 5.0);
    p = fma(r, p, -1.0 / 4.0);
    p = fma(r, p, 1.0 / 3.0);
    p = fma(r, p, -0.5);
    p = p * (r * r);
    double ed = (double)e;
    double hi = fma(ed, ln2_hi, s_hi[j]);
    return hi + (r + (fma(ed, ln2_lo, s_lo[j]) + p));
}

// ------------------------------------------------------------------ double-float
struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_quick(float a, float b) {  // |a| >= |b|
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df df_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ df df_two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df df_add(df a, df b) {
    df s = df_two_sum(a.hi, b.hi);
    float lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return df_quick(s.hi, lo);
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ df df_mul(df a, df b) {
    df p = df_two_prod(a.hi, b.hi);
    float lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return df_quick(p.hi, lo);
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
    df p = df_two_prod(a.hi, b);
    float lo = __fmaf_rn(a.lo, b, p.lo);
    return df_quick(p.hi, lo);
}

__device__ __forceinline__ df df_from_double(double v) {
    float hi = __double2float_rn(v);
    return {hi, __double2float_rn(v - (double)hi)};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ float df_to_float(df a) { return __fadd_rn(a.hi, a.lo); }

// 1/a: float reciprocal refined by one Newton step in df arithmetic
__device__ __forceinline__ df df_recip(df a) {
    float y = __frcp_rn(a.hi);
    // e = 1 - a*y in df, then y + y*e
    df ay = df_mul_f(a, y);
    df e = df_add({1.0f, 0.0f}, df_neg(ay));
    df ye = df_two_prod(y, e.hi);
    ye.lo = __fmaf_rn(y, e.lo, ye.lo);
    return df_add({y, 0.0f}, df_quick(ye.hi, ye.lo));
}

// natural log of a positive, normal df value
__device__ __forceinline__ df df_log(df x, const float *s_r, const float *s_hi, const float *s_lo, float ln2_hi,
                                     float ln2_lo) {
    int bits = __float_as_int(x.hi);
    int e = ((bits >> 23) & 0xff) - 127;
    int j = (bits >> 16) & (LOG_TBL - 1);
    // scale by 2^-e (exact for both parts)
    float sc = __int_as_float((127 - e) << 23);
    float mh = __fmul_rn(x.hi, sc), ml = __fmul_rn(x.lo, sc);
    // t = m r_j in df; r = t - 1 (t.hi - 1 is exact: t.hi lies within 2^-7 of 1)
    df t = df_two_prod(mh, s_r[j]);
    t.lo = __fmaf_rn(ml, s_r[j], t.lo);
    df r = df_two_sum(__fsub_rn(t.hi, 1.0f), t.lo);
    // log1p(r) = r - r^2/2 + r^3 (1/3 - r/4 + r^2/5 - r^3/6), the tail in FP32
    df r2 = df_two_prod(r.hi, r.hi);
    r2.lo = __fmaf_rn(2.0f * r.hi, r.lo, r2.lo);
    df half_r2 = {0.5f * r2.hi, 0.5f * r2.lo};
    float rh = r.hi;
    float q = __fmaf_rn(rh, -1.0f / 6.0f, 0.2f);
    q = __fmaf_rn(rh, q, -0.25f);
    q = __fmaf_rn(rh, q, 1.0f / 3.0f);
    float tail = q * (rh * rh * rh);
    // |r| > |r^2/2| > |tail|: the ordered (quick) sums are exact here
    df l1p = df_quick(r.hi, -half_r2.hi);
    l1p = df_quick(l1p.hi, __fadd_rn(l1p.lo, __fsub_rn(r.lo, half_r2.lo)));
    l1p = df_quick(l1p.hi, __fadd_rn(l1p.lo, tail));
    // e ln 2 + T_j: |e ln 2| >= ln 2 > |T_j| unless e = 0, when the quick sum is exact too
    df eln2 = df_mul_f({ln2_hi, ln2_lo}, (float)e);
    df et = df_quick(eln2.hi, s_hi[j]);
    et = df_quick(et.hi, __fadd_rn(et.lo, __fadd_rn(eln2.lo, s_lo[j])));
    return df_add(et, l1p);
}

}  // namespace lbvdw
