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

#include "lb_lane.cuh"

namespace lbvdw {

constexpr int LOG_TBL = 128;  // sub-intervals of [1, 2)

struct LogTables {
    // FP64 table: r_j = 1/c_j rounded to double, T_j = -ln(r_j) as hi + lo
    double r64[LOG_TBL], t64_hi[LOG_TBL], t64_lo[LOG_TBL];
    // df table: (r_j = 1/c_j rounded to float, T_j = -ln(r_j) as float hi + lo, 0): one
    // 16-byte load per logarithm
    float4 t32[LOG_TBL];
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
// The double-float operations on lanes are in lb_lane.cuh; df is one scalar lane.
using df = DF<float>;

__device__ __forceinline__ df df_from_double(double v) {
    float hi = __double2float_rn(v);
    return {hi, __double2float_rn(v - (double)hi)};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// 1/a for a positive df a (possibly unnormalised).  y ~ 1/a.hi from the MUFU approximation
// and one Newton step lies within an ulp of 1/a.hi, so the residual 1 - a.hi y is exact in
// one fused multiply-add; with e = 1 - a y, 1/a = y (1 + e + e^2 + ...), and the e^3 term
// lies below the df precision.  The result is unnormalised: hi = y, |lo| ~ ulp(y).
__device__ __forceinline__ df df_recip(df a) {
    const float y0 = __fdividef(1.0f, a.hi);
    const float y = __fmaf_rn(y0, __fmaf_rn(-a.hi, y0, 1.0f), y0);
    const float e = __fmaf_rn(-a.lo, y, __fmaf_rn(-a.hi, y, 1.0f));
    return df{y, __fmul_rn(y, __fmaf_rn(e, e, e))};
}

// The per-lane part of the table reduction: x_hi = 2^e m, j = top 7 bits of the mantissa;
// returns the scale 2^-e, e and the table entry (r_j, T_j hi, T_j lo).
struct LogRed {
    float sc, e;
    float4 t;
};
__device__ __forceinline__ LogRed log_reduce(float xh, const float4 *s_t) {
    const int bits = __float_as_int(xh);
    const int e = ((bits >> 23) & 0xff) - 127;
    const int j = (bits >> 16) & (LOG_TBL - 1);
    return {__int_as_float((127 - e) << 23), (float)e, s_t[j]};
}

__device__ __forceinline__ void log_lanes(float xh, const float4 *s_t, float &sc, float &e, float &r, float &thi,
                                          float &tlo) {
    const LogRed q = log_reduce(xh, s_t);
    sc = q.sc, e = q.e, r = q.t.x, thi = q.t.y, tlo = q.t.z;
}
__device__ __forceinline__ void log_lanes(float2 xh, const float4 *s_t, float2 &sc, float2 &e, float2 &r, float2 &thi,
                                          float2 &tlo) {
    const LogRed a = log_reduce(xh.x, s_t), b = log_reduce(xh.y, s_t);
    sc = make_float2(a.sc, b.sc), e = make_float2(a.e, b.e), r = make_float2(a.t.x, b.t.x);
    thi = make_float2(a.t.y, b.t.y), tlo = make_float2(a.t.z, b.t.z);
}

// natural log of positive, normal df lanes.  s_t: the table (r_j, -ln r_j as hi + lo)
// in shared memory; a non-positive or non-finite input gives a meaningless value (the
// table index stays in range).
template <class V>
__device__ __forceinline__ DF<V> df_log(DF<V> x, const float4 *s_t, float ln2_hi, float ln2_lo) {
    V sc, ef, rj, thi, tlo;
    log_lanes(x.hi, s_t, sc, ef, rj, thi, tlo);
    // scale by 2^-e (exact for both parts)
    const V mh = v_mul(x.hi, sc), ml = v_mul(x.lo, sc);
    // t = m r_j in df; r = t - 1 (t.hi - 1 is exact: t.hi lies within 2^-7 of 1)
    DF<V> t = df_two_prod(mh, rj);
    t.lo = v_fma(ml, rj, t.lo);
    const DF<V> r = df_two_sum(v_sub(t.hi, vc<V>(1.0)), t.lo);
    // log1p(r) = r - r^2/2 + r^3 (1/3 - r/4 + r^2/5 - r^3/6), the tail in FP32
    DF<V> r2 = df_two_prod(r.hi, r.hi);
    r2.lo = v_fma(v_add(r.hi, r.hi), r.lo, r2.lo);
    const V h2hi = v_mul(r2.hi, vc<V>(0.5)), h2lo = v_mul(r2.lo, vc<V>(0.5));
    const V rh = r.hi;
    V q = v_fma(rh, vc<V>(-1.0 / 6.0), vc<V>(0.2));
    q = v_fma(rh, q, vc<V>(-0.25));
    q = v_fma(rh, q, vc<V>(1.0 / 3.0));
    const V tail = v_mul(q, v_mul(v_mul(rh, rh), rh));
    // |r| > |r^2/2| > |tail|: the ordered (quick) sums are exact here
    DF<V> l1p = df_quick(rh, v_neg(h2hi));
    l1p = df_quick(l1p.hi, v_add(l1p.lo, v_sub(r.lo, h2lo)));
    l1p = df_quick(l1p.hi, v_add(l1p.lo, tail));
    // e ln 2 + T_j: |e ln 2| >= ln 2 > |T_j| unless e = 0, when the quick sum is exact too
    const DF<V> eln2 = df_mul_f(df_splat(df{ln2_hi, ln2_lo}, ef), ef);
    DF<V> et = df_quick(eln2.hi, thi);
    et = df_quick(et.hi, v_add(et.lo, v_add(eln2.lo, tlo)));
    return df_add(et, l1p);
}

}  // namespace lbvdw
