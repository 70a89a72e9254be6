// lb_lane.cuh -- lane arithmetic of the per-node device code.
//
// The per-node arithmetic (stencils, chemical potential, collision) is written once over
// a lane type V:
//   double   the FP64 path, one component at a time;
//   float    the FP32 paths, one component at a time;
//   float2   the FP32 paths, two components at once in one register pair, on the packed
//            FP32x2 add / multiply / fused multiply-add of sm_100 and later: one issued
//            instruction for both components.
// Every operation states its rounding (nothing is left to the compiler's contraction), so
// a component's value is bitwise the same whether it is computed alone (float) or packed
// with another (float2), and every kernel that runs the same step agrees to the bit.
#pragma once
#include <cuda_runtime.h>

namespace lbvdw {

// ---------------------------------------------------------------- operations
__device__ __forceinline__ double v_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double v_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double v_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double v_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ double v_neg(double a) { return -a; }

__device__ __forceinline__ float v_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float v_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float v_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float v_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float v_neg(float a) { return -a; }

// packed pairs; a negated operand costs no instruction (an operand modifier)
__device__ __forceinline__ float2 v_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 v_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 v_sub(float2 a, float2 b) { return __fadd2_rn(a, v_neg(b)); }
__device__ __forceinline__ float2 v_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 v_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// a constant in every lane (rounded to the element type)
template <class V> __device__ __forceinline__ V vc(double c);
template <> __device__ __forceinline__ double vc<double>(double c) { return c; }
template <> __device__ __forceinline__ float vc<float>(double c) { return (float)c; }
template <> __device__ __forceinline__ float2 vc<float2>(double c) { return make_float2((float)c, (float)c); }

// a scalar of the element type in every lane
__device__ __forceinline__ double vs(double x, double) { return x; }
__device__ __forceinline__ float vs(float x, float) { return x; }
__device__ __forceinline__ float2 vs(float x, float2) { return make_float2(x, x); }

// reciprocal: exact division in FP64, the MUFU approximation in FP32 (per lane)
__device__ __forceinline__ double v_rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float v_rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ float2 v_rcp(float2 x) { return make_float2(__fdividef(1.0f, x.x), __fdividef(1.0f, x.y)); }

// ---------------------------------------------------------------- double-float lanes
// A value hi + lo of two FP32 numbers per lane (T. J. Dekker, "A floating-point technique
// for extending the available precision", Numer. Math. 18, 1971; error-free sums after
// Knuth, products through the fused multiply-add).
template <class V>
struct DF {
    V hi, lo;
};

template <class V>
__device__ __forceinline__ DF<V> df_quick(V a, V b) {  // |a| >= |b|
    V s = v_add(a, b);
    return {s, v_sub(b, v_sub(s, a))};
}

template <class V>
__device__ __forceinline__ DF<V> df_two_sum(V a, V b) {
    V s = v_add(a, b);
    V bb = v_sub(s, a);
    V e = v_add(v_sub(a, v_sub(s, bb)), v_sub(b, bb));
    return {s, e};
}

template <class V>
__device__ __forceinline__ DF<V> df_two_prod(V a, V b) {
    V p = v_mul(a, b);
    return {p, v_fma(a, b, v_neg(p))};
}

template <class V>
__device__ __forceinline__ DF<V> df_add(DF<V> a, DF<V> b) {
    DF<V> s = df_two_sum(a.hi, b.hi);
    V lo = v_add(s.lo, v_add(a.lo, b.lo));
    return df_quick(s.hi, lo);
}

template <class V>
__device__ __forceinline__ DF<V> df_neg(DF<V> a) {
    return {v_neg(a.hi), v_neg(a.lo)};
}

template <class V>
__device__ __forceinline__ DF<V> df_mul(DF<V> a, DF<V> b) {
    DF<V> p = df_two_prod(a.hi, b.hi);
    V lo = v_fma(a.hi, b.lo, v_fma(a.lo, b.hi, p.lo));
    return df_quick(p.hi, lo);
}

// unnormalised products (|lo| up to about an ulp of hi), for values that only feed
// further df arithmetic
template <class V>
__device__ __forceinline__ DF<V> df_mul_u(DF<V> a, DF<V> b) {
    DF<V> p = df_two_prod(a.hi, b.hi);
    return {p.hi, v_fma(a.hi, b.lo, v_fma(a.lo, b.hi, p.lo))};
}

template <class V>
__device__ __forceinline__ DF<V> df_mul_fu(DF<V> a, V b) {
    DF<V> p = df_two_prod(a.hi, b);
    return {p.hi, v_fma(a.lo, b, p.lo)};
}

// a + b for a df a and a working-precision b
template <class V>
__device__ __forceinline__ DF<V> df_add_f(DF<V> a, V b) {
    DF<V> s = df_two_sum(a.hi, b);
    return df_quick(s.hi, v_add(s.lo, a.lo));
}

template <class V>
__device__ __forceinline__ DF<V> df_mul_f(DF<V> a, V b) {
    DF<V> p = df_two_prod(a.hi, b);
    V lo = v_fma(a.lo, b, p.lo);
    return df_quick(p.hi, lo);
}

// a scalar double-float in every lane
__device__ __forceinline__ DF<float> df_splat(DF<float> a, float) { return a; }
__device__ __forceinline__ DF<float2> df_splat(DF<float> a, float2) {
    return {make_float2(a.hi, a.hi), make_float2(a.lo, a.lo)};
}

// ---------------------------------------------------------------- stencils
// The 3 x 3 neighbourhood of a node: c centre, e/w/n/s axis and ne/nw/sw/se diagonal
// neighbours.  D2Q9 (w = 4/9, 1/9, 1/36, theta = 1/3):
//   D phi   = (1/theta) sum_i w_i v_i phi_i = (e - w)/3 + ((ne + se) - (nw + sw))/12 in x
//   Lap phi = (2/theta) sum_i w_i (phi_i - phi_0) = 2/3 axis + 1/6 diag - 10/3 c
// D1Q3: D phi = (e - w)/2, Lap phi = e + w - 2 c (Sec. V).
template <class V>
struct Nbr9 {
    V c, e, w, n, s, ne, nw, sw, se;
};

template <class V>
__device__ __forceinline__ V lap_d2q9(const Nbr9<V> &p) {
    V axis = v_add(v_add(p.e, p.w), v_add(p.n, p.s));
    V diag = v_add(v_add(p.ne, p.nw), v_add(p.se, p.sw));
    return v_fma(axis, vc<V>(2.0 / 3.0), v_fma(diag, vc<V>(1.0 / 6.0), v_mul(p.c, vc<V>(-10.0 / 3.0))));
}

template <class V>
__device__ __forceinline__ void grad_d2q9(const Nbr9<V> &p, V &gx, V &gy) {
    gx = v_fma(v_sub(p.e, p.w), vc<V>(1.0 / 3.0), v_mul(v_sub(v_add(p.ne, p.se), v_add(p.nw, p.sw)), vc<V>(1.0 / 12.0)));
    gy = v_fma(v_sub(p.n, p.s), vc<V>(1.0 / 3.0), v_mul(v_sub(v_add(p.ne, p.nw), v_add(p.se, p.sw)), vc<V>(1.0 / 12.0)));
}

template <class V>
__device__ __forceinline__ V lap_d1q3(V c, V e, V w) {
    return v_fma(c, vc<V>(-2.0), v_add(e, w));
}

template <class V>
__device__ __forceinline__ V grad_d1q3(V e, V w) {
    return v_mul(v_sub(e, w), vc<V>(0.5));
}

// s D phi from the differences of phi across the node (already rounded to the lane type):
// ew = e - w, ns = n - s, d1 = ne - sw, d2 = se - nw; c3 = s/3, c12 = s/12.
template <class V>
__device__ __forceinline__ void grad_d2q9_diff(V ew, V ns, V d1, V d2, V c3, V c12, V &gx, V &gy) {
    gx = v_fma(ew, c3, v_mul(v_add(d1, d2), c12));
    gy = v_fma(ns, c3, v_mul(v_sub(d1, d2), c12));
}

}  // namespace lbvdw
