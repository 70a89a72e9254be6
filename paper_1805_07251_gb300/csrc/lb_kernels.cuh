// lb_kernels.cuh -- device code of the fused multicomponent van der Waals
// lattice Boltzmann timestep (Ridl & Wagner, arXiv:1805.07251, Sec. III and V).
//
// One CTA owns a TX x TY tile of nodes.  A timestep is one launch:
//   phase 1  densities rho^c on the tile plus a 2-node ring        (Sec. III moments)
//   phase 2  mu^c on the tile plus a 1-node ring                   (Eq. discreteChemicalPotential)
//   phase 3  per node: force (Eq. forceMuLog / forceMuId), friction (Eq. forceFriction),
//            Psi (Eq. forceCorrectionsPsi), BGK + forcing (Eqs. feq, BGKcollisionOperator),
//            push-streaming to the other buffer (Eq. LBequation).
// rho and mu live only in shared memory; HBM sees one read and one write of
// every population per step (plus halo re-reads that the L2 serves).
//
// Storage type S holds the deviation g_i^c = f_i^c - w_i rho_ref^c (rho_ref = 0 in the
// FP64 path, so g = f there).  Compute type R is double in the FP64 path and float in
// the mixed paths, where eta, 1/eta, the logarithms and the differences of mu are
// carried in FP64 (MU_TBL) or in double-float arithmetic (MU_DF), see lb_mu.cuh.
// The per-node arithmetic is written over lane types (lb_lane.cuh): an even number of
// FP32 components runs as float2 pairs on the packed FP32x2 instructions
// (step_tile_pair), bitwise equal to one component at a time.
#pragma once
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "lb_mu.cuh"

namespace lbvdw {

constexpr unsigned ERR_DOMAIN = 1u;   // rho^c <= 0, eta <= 0 or non-finite value
constexpr unsigned ERR_TIMEOUT = 2u;  // a bounded wait for bulk copies ran out (lb_strip.cuh)
constexpr unsigned ERR_STALL = 4u;    // a bounded wait for a neighbouring tile's flag ran out (lb_chain.cuh)

struct DevParams {
    int nx, ny;
    double omega;      // 1 / tau
    double psi_g;      // (tau - 1/4) / tau : coefficient of G G / rho in -Psi
    double psi_l;      // 1 / (12 tau)      : coefficient of Lap rho in -Psi
    double kT, gamma;
    double a[16], kappa[16], lam[16];  // stride 4
    double b[4];
    double rho_ref[4];  // FP32-mixed: reference densities (rounded to float values)
    unsigned *err;      // error word (device)
    const LogTables *tbl;  // log tables (device)
    double gkT;         // gamma_mu * kT
    float b_hi[4], b_lo[4];  // double-float copies of b
    // FP32-class mu paths store phi / (gamma kT) = mu / kT (- ln rho / (3 gamma kT) for
    // "nid"); gamma kT then enters with the gradient weights
    float ikT_f;                  // 1 / kT
    float gkt3_f, gkt12_f, gkt2_f;  // gamma kT / 3, gamma kT / 12, gamma kT / 2
    float cnid_hi, cnid_lo;       // 1 / (3 gamma kT) as a double-float
    // FP32 copies for the FP32 paths (no double->float conversion in the kernels)
    float a2_f[16], kappa_f[16], lam_f[16];  // 2 a, kappa, lambda
    float rho_ref_f[4], omega_f, psi_g_f, psi_l_f;
    // 1 - omega, and lambda^12 / (1 + lambda^12 / 2) of the two-component friction
    double omc, lam_fr;
    float omc_f, lam_fr_f;
    float ln2_hi_f, ln2_lo_f;  // ln 2 as a double-float (the df logarithm)
    // moment-space collision (D2Q9, FORCE bit 1): relaxation rates of the shear and ghost
    // moments (the bulk moment keeps omega), and the Psi coefficient of the traceless part
    // of G G / rho, (tau_s - 1/4) / tau_s (psi_g stays that of the trace part)
    double omega_s, omega_g, psi_s;
    float omega_s_f, omega_g_f, psi_s_f;
};

// The FORCE template flag: bit 0 selects the "nid" force (Eq. forceMuId; clear: the
// "log" force, Eq. forceMuLog), bit 1 the moment-space collision with distinct
// relaxation times (D2Q9; clear: BGK).
template <int FORCE> struct Flags {
    static constexpr bool nid = (FORCE & 1) != 0;
    static constexpr bool mrt = (FORCE & 2) != 0;
};

// a parameter in the compute type R: the double value or its precomputed float copy
template <class R>
__device__ __forceinline__ R pv(double d, float f);
template <>
__device__ __forceinline__ double pv<double>(double d, float) { return d; }
template <>
__device__ __forceinline__ float pv<float>(double, float f) { return f; }

// periodic wrap of g in [-n, 2n)
__device__ __forceinline__ int wrap1(int g, int n) { return g < 0 ? g + n : (g >= n ? g - n : g); }

// ---------------------------------------------------------------------------
// lattices.  D1Q3: v = 0, +1, -1 (Sec. V), w = 2/3, 1/6, 1/6 (the weights of the
// explicit D1Q3 update at theta = 1/3).  D2Q9: rest, E, N, W, S, NE, NW, SW, SE.
// ---------------------------------------------------------------------------
template <int LAT> struct Lat;
template <> struct Lat<1> {
    static constexpr int Q = 3, D = 1, HY = 0;
    __host__ __device__ static constexpr int vx(int i) { return i == 1 ? 1 : (i == 2 ? -1 : 0); }
    __host__ __device__ static constexpr int vy(int) { return 0; }
    __host__ __device__ static constexpr double w(int i) { return i == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
};
template <> struct Lat<2> {
    static constexpr int Q = 9, D = 2, HY = 1;
    __host__ __device__ static constexpr int vx(int i) {
        return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
    }
    __host__ __device__ static constexpr int vy(int i) {
        return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
};

__device__ __forceinline__ int wrap(int g, int n) {
    g %= n;
    return g < 0 ? g + n : g;
}

__device__ __forceinline__ size_t pop_index(int c, int i, int Q, int y, int x, int nx, int ny) {
    return ((size_t)(c * Q + i) * (size_t)ny + (size_t)y) * (size_t)nx + (size_t)x;
}

// Stencils on a shared-memory array with row length EXW (the formulas are in lb_lane.cuh).
template <class T>
__device__ __forceinline__ Nbr9<T> nbr9(const T *p, int W) {
    return {p[0], p[1], p[-1], p[W], p[-W], p[W + 1], p[W - 1], p[-W - 1], p[-W + 1]};
}

template <int LAT, class T>
__device__ __forceinline__ void grad_at(const T *s, int ex, int ey, int EXW, T &gx, T &gy) {
    const T *p = s + ey * EXW + ex;
    if constexpr (LAT == 1) {
        gx = grad_d1q3(p[1], p[-1]);
        gy = vc<T>(0.0);
    } else {
        grad_d2q9(nbr9(p, EXW), gx, gy);
    }
}

template <int LAT, class T>
__device__ __forceinline__ T lap_at(const T *s, int ex, int ey, int EXW) {
    const T *p = s + ey * EXW + ex;
    if constexpr (LAT == 1) return lap_d1q3(p[0], p[1], p[-1]);
    else return lap_d2q9(nbr9(p, EXW));
}

// ---------------------------------------------------------------------------
// the fused step
//
// MU selects the chemical-potential arithmetic:
//   MU_F64   FP64 path: everything in double, CUDA's log and division;
//   MU_TBL   mixed path: FP64 eta, 1/eta and table-driven FP64 logs (lb_mu.cuh),
//            FP32 for the linear part of mu, the stencils and everything after;
//   MU_DF    mixed path with the FP64 work replaced by double-float arithmetic;
//   MU_F32   everything in FP32 (CUDA's logf), the reference point for what the
//            FP64-class mu of MU_TBL / MU_DF buys.
// The differences of mu across a node (the only place where mu's extra precision
// matters) are taken in the mu arithmetic, then rounded to R.
// ---------------------------------------------------------------------------
enum { MU_F64 = 0, MU_TBL = 1, MU_DF = 2, MU_F32 = 3 };

template <int MU> struct MuStore;
template <> struct MuStore<MU_F64> { using T = double; };
template <> struct MuStore<MU_TBL> { using T = double; };
template <> struct MuStore<MU_DF> { using T = df; };
template <> struct MuStore<MU_F32> { using T = float; };

// phi difference a - b in the mu arithmetic, rounded to R.  For df values the high
// parts are subtracted first: exact when they are within a factor 2 (Sterbenz), else
// rounded once at the precision of the result, which is rounded to FP32 anyway.
template <class R>
__device__ __forceinline__ R phi_diff(double a, double b) { return (R)(a - b); }
template <class R>
__device__ __forceinline__ R phi_diff(float a, float b) { return (R)__fsub_rn(a, b); }
template <class R>
__device__ __forceinline__ R phi_diff(df a, df b) { return v_add(v_sub(a.hi, b.hi), v_sub(a.lo, b.lo)); }
__device__ __forceinline__ float2 phi_diff2(float2 a, float2 b) { return v_sub(a, b); }
__device__ __forceinline__ float2 phi_diff2(DF<float2> a, DF<float2> b) {
    return v_add(v_sub(a.hi, b.hi), v_sub(a.lo, b.lo));
}

// The weights of D phi: 1/3, 1/12 (D2Q9) and 1/2 (D1Q3) times the scale of the stored phi
// (gamma kT for the FP32-class mu paths, which store phi / (gamma kT); 1 otherwise).
template <class T> struct PhiScaled { static constexpr bool value = false; };
template <> struct PhiScaled<df> { static constexpr bool value = true; };
template <> struct PhiScaled<float> { static constexpr bool value = true; };

template <class R, class T>
__device__ __forceinline__ void phi_weights(const DevParams &P, R &c3, R &c12, R &c2) {
    if constexpr (PhiScaled<T>::value) {
        c3 = P.gkt3_f, c12 = P.gkt12_f, c2 = P.gkt2_f;
    } else {
        c3 = vc<R>(1.0 / 3.0), c12 = vc<R>(1.0 / 12.0), c2 = vc<R>(0.5);
    }
}

// D (gamma mu) at (mx, my) of an MX-wide shared array of phi, differences in the mu arithmetic
template <int LAT, class R, class T>
__device__ __forceinline__ void grad_phi(const T *s, int mx, int my, int MXW, const DevParams &P, R &gx, R &gy) {
    const T *p = s + my * MXW + mx;
    R c3, c12, c2;
    phi_weights<R, T>(P, c3, c12, c2);
    if constexpr (LAT == 1) {
        gx = v_mul(phi_diff<R>(p[1], p[-1]), c2);
        gy = vc<R>(0.0);
    } else {
        grad_d2q9_diff(phi_diff<R>(p[1], p[-1]), phi_diff<R>(p[MXW], p[-MXW]),
                       phi_diff<R>(p[MXW + 1], p[-MXW - 1]),  // NE - SW
                       phi_diff<R>(p[-MXW + 1], p[MXW - 1]),  // SE - NW
                       c3, c12, gx, gy);
    }
}

// shared-memory log tables of the MU variant (TBL_WORDS floats)
template <int MU>
struct TblWords {
    static constexpr int value = MU == MU_TBL ? 3 * LOG_TBL * 2 : (MU == MU_DF ? 4 * LOG_TBL : 4);
};

template <int MU>
__device__ __forceinline__ void load_tables(float *s_tbl, const LogTables *tbl, int tid, int nt) {
    if constexpr (MU == MU_TBL) {
        double *t = reinterpret_cast<double *>(s_tbl);
        for (int k = tid; k < LOG_TBL; k += nt) {
            t[k] = tbl->r64[k];
            t[LOG_TBL + k] = tbl->t64_hi[k];
            t[2 * LOG_TBL + k] = tbl->t64_lo[k];
        }
    } else if constexpr (MU == MU_DF) {
        float4 *t = reinterpret_cast<float4 *>(s_tbl);
        for (int k = tid; k < LOG_TBL; k += nt) t[k] = tbl->t32[k];
    }
}

template <int MU>
__device__ __forceinline__ void load_tables(float *s_tbl, const DevParams &P, int tid, int nt) {
    load_tables<MU>(s_tbl, P.tbl, tid, nt);
}

// Moments of one node's populations (deviations): sum_i g_i and the bare momentum
// sum_i g_i v_i, summed in direction order.
template <int LAT, class V>
__device__ __forceinline__ void moments_lane(const V (&g)[Lat<LAT>::Q], V &acc, V &ax, V &ay) {
    using L = Lat<LAT>;
    acc = g[0];
    bool fx = true, fy = true;
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
        acc = v_add(acc, g[i]);
        if (L::vx(i) != 0) {
            const V t = L::vx(i) == 1 ? g[i] : v_neg(g[i]);
            ax = fx ? t : v_add(ax, t);
            fx = false;
        }
        if (L::vy(i) != 0) {
            const V t = L::vy(i) == 1 ? g[i] : v_neg(g[i]);
            ay = fy ? t : v_add(ay, t);
            fy = false;
        }
    }
    if (fy) ay = vc<V>(0.0);
}

// The linear part of mu^c: lin^c = sum_c' (kappa^{cc'} Lap rho^c' + 2 a^{cc'} rho^c'),
// c' ascending (Eq. discreteChemicalPotential).
template <int N, class R>
__device__ __forceinline__ void lin_node(const R (&r)[N], const R (&lp)[N], const DevParams &P, R (&lin)[N]) {
#pragma unroll
    for (int c = 0; c < N; ++c) {
        R t = v_mul(pv<R>(P.kappa[c * 4], P.kappa_f[c * 4]), lp[0]);
        t = v_fma(pv<R>(2.0 * P.a[c * 4], P.a2_f[c * 4]), r[0], t);
#pragma unroll
        for (int cc = 1; cc < N; ++cc) {
            t = v_fma(pv<R>(P.kappa[c * 4 + cc], P.kappa_f[c * 4 + cc]), lp[cc], t);
            t = v_fma(pv<R>(2.0 * P.a[c * 4 + cc], P.a2_f[c * 4 + cc]), r[cc], t);
        }
        lin[c] = t;
    }
}
// component c of NP lane pairs (pair c / 2, half c % 2)
template <int NP>
__device__ __forceinline__ float comp(const float2 (&v)[NP], int c) {
    return (c & 1) ? v[c >> 1].y : v[c >> 1].x;
}

// the same for NP component pairs, components 2q and 2q+1 in lane pair q
template <int NP>
__device__ __forceinline__ void lin_pairs(const float2 (&r)[NP], const float2 (&lp)[NP], const DevParams &P,
                                          float2 (&lin)[NP]) {
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const int c0 = 8 * q, c1 = 8 * q + 4;  // rows 2q and 2q+1 of the stride-4 matrices
        float2 t = v_mul(make_float2(P.kappa_f[c0], P.kappa_f[c1]), vs(lp[0].x, r[0]));
        t = v_fma(make_float2(P.a2_f[c0], P.a2_f[c1]), vs(r[0].x, r[0]), t);
#pragma unroll
        for (int cc = 1; cc < 2 * NP; ++cc) {
            t = v_fma(make_float2(P.kappa_f[c0 + cc], P.kappa_f[c1 + cc]), vs(comp(lp, cc), r[0]), t);
            t = v_fma(make_float2(P.a2_f[c0 + cc], P.a2_f[c1 + cc]), vs(comp(r, cc), r[0]), t);
        }
        lin[q] = t;
    }
}

// ---------------------------------------------------------------------------
// chemical potential in FP32 storage: phi^c = gamma mu^c (minus theta ln rho^c for "nid")
// with mu^c = kT [ln(rho^c / eta) + b^c rho / eta] - lin^c (Eq. discreteChemicalPotential).
// eta and rho / eta are one value per node; the rest runs per component lane.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float v_log(float x) { return logf(x); }
__device__ __forceinline__ float2 v_log(float2 x) { return make_float2(logf(x.x), logf(x.y)); }

// phi^c / (gamma kT) = ln(rho^c / eta) + b^c rho / eta - lin^c / kT (minus ln rho^c / (3 gamma kT)
// for "nid") of one component lane, from the node's 1/eta and rho/eta
template <class V, int FORCE>
__device__ __forceinline__ DF<V> mu_df_lanes(V r, V lin, DF<V> b, df ieta, df rte, bool ok, const DevParams &P,
                                             const float4 *s_t) {
    const V zero = vc<V>(0.0);
    DF<V> lg = df_log(df_mul_fu(df_splat(ieta, r), r), s_t, P.ln2_hi_f, P.ln2_lo_f);
    if (!ok) lg = DF<V>{zero, zero};
    const DF<V> m = df_add(lg, df_mul_u(df_splat(rte, r), b));
    DF<V> ph = df_add_f(m, v_mul(lin, vs(-P.ikT_f, r)));
    if constexpr (Flags<FORCE>::nid) {
        DF<V> lr = df_log(DF<V>{r, zero}, s_t, P.ln2_hi_f, P.ln2_lo_f);
        if (!ok) lr = DF<V>{zero, zero};
        ph = df_add(ph, df_neg(df_mul_u(lr, df_splat(df{P.cnid_hi, P.cnid_lo}, r))));
    }
    return ph;
}

template <class V, int FORCE>
__device__ __forceinline__ V mu_f32_lanes(V r, V lin, V b, float ieta, float rte, const DevParams &P) {
    const V lg = v_log(v_mul(r, vs(ieta, r)));
    V ph = v_fma(lin, vs(-P.ikT_f, r), v_fma(b, vs(rte, r), lg));
    if constexpr (Flags<FORCE>::nid) ph = v_fma(v_log(r), vs(-P.cnid_hi, r), ph);
    return ph;
}

// eta = 1 - S from S = sum_c b^c rho^c (an unnormalised df): the quick sum is exact while
// S.hi < 1, i.e. wherever eta > 0
__device__ __forceinline__ df eta_of(df S) {
    const df q = df_quick(1.0f, -S.hi);
    return df{q.hi, __fsub_rn(q.lo, S.lo)};
}

// NP component pairs, double-float mu: phi of every lane; false outside the domain.
// S = sum_c b^c rho^c and rho = sum_c rho^c accumulate in component order.
template <int NP, int FORCE>
__device__ __forceinline__ bool mu_pairs_df(const float2 (&r)[NP], const float2 (&lin)[NP], const DevParams &P,
                                            const float4 *s_t, DF<float2> (&phi)[NP]) {
    DF<float2> b[NP], br[NP];
    bool ok = true;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        b[q] = {make_float2(P.b_hi[2 * q], P.b_hi[2 * q + 1]), make_float2(P.b_lo[2 * q], P.b_lo[2 * q + 1])};
        br[q] = df_mul_fu(b[q], r[q]);
        ok = ok && r[q].x > 0.0f && r[q].y > 0.0f;
    }
    df S = {br[0].hi.x, br[0].lo.x};
#pragma unroll
    for (int c = 1; c < 2 * NP; ++c) {
        const float ph = (c & 1) ? br[c >> 1].hi.y : br[c >> 1].hi.x;
        const float pl = (c & 1) ? br[c >> 1].lo.y : br[c >> 1].lo.x;
        const df t = df_two_sum(S.hi, ph);
        S = df{t.hi, __fadd_rn(t.lo, __fadd_rn(S.lo, pl))};
    }
    const df eta = eta_of(S);
    // total density: the sum of the first two FP32 densities is exact as a pair
    df rt = df_two_sum(r[0].x, r[0].y);
#pragma unroll
    for (int c = 2; c < 2 * NP; ++c) rt = df_add(rt, df{comp(r, c), 0.0f});
    ok = ok && eta.hi > 0.0f;
    const df ieta = df_recip(eta);
    const df rte = df_mul_u(rt, ieta);
#pragma unroll
    for (int q = 0; q < NP; ++q) phi[q] = mu_df_lanes<float2, FORCE>(r[q], lin[q], b[q], ieta, rte, ok, P, s_t);
    return ok;
}

template <int NP, int FORCE>
__device__ __forceinline__ bool mu_pairs_f32(const float2 (&r)[NP], const float2 (&lin)[NP], const DevParams &P,
                                             float2 (&phi)[NP]) {
    float eta = 1.0f, rt = r[0].x;
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 2 * NP; ++c) {
        eta = __fmaf_rn(-P.b_hi[c], comp(r, c), eta);
        ok = ok && comp(r, c) > 0.0f;
    }
#pragma unroll
    for (int c = 1; c < 2 * NP; ++c) rt = __fadd_rn(rt, comp(r, c));
    ok = ok && eta > 0.0f;
    const float ieta = __frcp_rn(eta);
    const float rte = __fmul_rn(rt, ieta);
#pragma unroll
    for (int q = 0; q < NP; ++q)
        phi[q] = mu_f32_lanes<float2, FORCE>(r[q], lin[q], make_float2(P.b_hi[2 * q], P.b_hi[2 * q + 1]), ieta,
                                             rte, P);
    return ok;
}

// One node of phase 2: phi^c = gamma mu^c (minus theta ln rho^c for "nid") from the
// densities r and the linear part lin = sum_c' (2 a rho' + kappa Lap rho').
// Returns false when rho^c <= 0 or eta <= 0 (phi is then meaningless).
template <int N, class R, int FORCE, int MU>
__device__ __forceinline__ bool mu_node(const R (&r)[N], const R (&lin)[N], const DevParams &P,
                                        const float *s_tbl, typename MuStore<MU>::T (&phi)[N]) {
    bool ok = true;
#pragma unroll
    for (int c = 0; c < N; ++c) ok = ok && (r[c] > (R)0);
    if constexpr (MU == MU_F64) {
        double eta = 1.0, rt = 0.0;
#pragma unroll
        for (int c = 0; c < N; ++c) {
            eta -= P.b[c] * r[c];
            rt += r[c];
        }
        ok = ok && eta > 0.0;
        const double ieta = 1.0 / eta;
#pragma unroll
        for (int c = 0; c < N; ++c) {
            double m = P.kT * (log(r[c] * ieta) + P.b[c] * rt * ieta) - lin[c];
            double ph = P.gamma * m;
            if constexpr (Flags<FORCE>::nid) ph -= (1.0 / 3.0) * log(r[c]);
            phi[c] = ph;
        }
    } else if constexpr (MU == MU_TBL) {
        const double *t = reinterpret_cast<const double *>(s_tbl);
        double eta = 1.0, rt = 0.0;
#pragma unroll
        for (int c = 0; c < N; ++c) {
            eta = fma(-P.b[c], (double)r[c], eta);
            rt += (double)r[c];
        }
        ok = ok && eta > 0.0;
        double y = (double)__frcp_rn((float)eta);  // Newton: y <- y + y (1 - eta y), twice
        y = fma(y, fma(-eta, y, 1.0), y);
        y = fma(y, fma(-eta, y, 1.0), y);
        const double rte = rt * y;
#pragma unroll
        for (int c = 0; c < N; ++c) {
            double lg = ok ? log64_tbl((double)r[c] * y, t, t + LOG_TBL, t + 2 * LOG_TBL, P.tbl->ln2_hi_d,
                                       P.tbl->ln2_lo_d)
                           : 0.0;
            double ph = fma(P.gkT, fma(P.b[c], rte, lg), -P.gamma * (double)lin[c]);
            if constexpr (Flags<FORCE>::nid)
                ph -= (1.0 / 3.0) * (ok ? log64_tbl((double)r[c], t, t + LOG_TBL, t + 2 * LOG_TBL, P.tbl->ln2_hi_d,
                                                     P.tbl->ln2_lo_d)
                                        : 0.0);
            phi[c] = ph;
        }
    } else if constexpr (N % 2 == 0) {  // MU_DF / MU_F32: components in lane pairs
        constexpr int NP = N / 2;
        float2 r2[NP], l2[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            r2[q] = make_float2(r[2 * q], r[2 * q + 1]);
            l2[q] = make_float2(lin[2 * q], lin[2 * q + 1]);
        }
        if constexpr (MU == MU_DF) {
            DF<float2> ph[NP];
            ok = mu_pairs_df<NP, FORCE>(r2, l2, P, reinterpret_cast<const float4 *>(s_tbl), ph);
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                phi[2 * q] = df{ph[q].hi.x, ph[q].lo.x};
                phi[2 * q + 1] = df{ph[q].hi.y, ph[q].lo.y};
            }
        } else {
            float2 ph[NP];
            ok = mu_pairs_f32<NP, FORCE>(r2, l2, P, ph);
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                phi[2 * q] = ph[q].x;
                phi[2 * q + 1] = ph[q].y;
            }
        }
    } else if constexpr (MU == MU_F32) {
        float eta = 1.0f, rt = r[0];
#pragma unroll
        for (int c = 0; c < N; ++c) eta = __fmaf_rn(-P.b_hi[c], r[c], eta);
#pragma unroll
        for (int c = 1; c < N; ++c) rt = __fadd_rn(rt, r[c]);
        ok = ok && eta > 0.0f;
        const float ieta = __frcp_rn(eta);
        const float rte = __fmul_rn(rt, ieta);
#pragma unroll
        for (int c = 0; c < N; ++c) phi[c] = mu_f32_lanes<float, FORCE>(r[c], lin[c], P.b_hi[c], ieta, rte, P);
    } else {  // MU_DF, one component lane at a time
        df S = df_mul_fu(df{P.b_hi[0], P.b_lo[0]}, r[0]);
#pragma unroll
        for (int c = 1; c < N; ++c) {
            const df p = df_mul_fu(df{P.b_hi[c], P.b_lo[c]}, r[c]);
            const df t = df_two_sum(S.hi, p.hi);
            S = df{t.hi, __fadd_rn(t.lo, __fadd_rn(S.lo, p.lo))};
        }
        const df eta = eta_of(S);
        // total density: the sum of the first two FP32 densities is exact as a pair
        df rt = N == 1 ? df{r[0], 0.0f} : df_two_sum(r[0], r[N > 1 ? 1 : 0]);
#pragma unroll
        for (int c = 2; c < N; ++c) rt = df_add(rt, df{r[c], 0.0f});
        ok = ok && eta.hi > 0.0f;
        const df ieta = df_recip(eta);
        const df rte = df_mul_u(rt, ieta);
#pragma unroll
        for (int c = 0; c < N; ++c)
            phi[c] = mu_df_lanes<float, FORCE>(r[c], lin[c], df{P.b_hi[c], P.b_lo[c]}, ieta, rte, ok, P,
                                               reinterpret_cast<const float4 *>(s_tbl));
    }
    return ok;
}

// ---------------------------------------------------------------------------
// collision (Sec. III): per component lane, then the friction across components
// ---------------------------------------------------------------------------
// G^mu (Eq. forceMuLog: -rho D phi + theta D rho; Eq. forceMuId: -rho D phi), 1/rho, u = j/rho
template <int FORCE, class V>
__device__ __forceinline__ void gain_lane(V rho, V gpx, V gpy, V grx, V gry, V jx, V jy, V &Gx, V &Gy, V &ir, V &ux,
                                          V &uy) {
    if constexpr (!Flags<FORCE>::nid) {
        Gx = v_fma(v_neg(rho), gpx, v_mul(grx, vc<V>(1.0 / 3.0)));
        Gy = v_fma(v_neg(rho), gpy, v_mul(gry, vc<V>(1.0 / 3.0)));
    } else {
        Gx = v_mul(v_neg(rho), gpx);
        Gy = v_mul(v_neg(rho), gpy);
    }
    ir = v_rcp(rho);
    ux = v_mul(jx, ir);
    uy = v_mul(jy, ir);
}

// cx a + cy b for a lattice direction (cx, cy in {-1, 0, 1}), exact
template <int CX, int CY, class V>
__device__ __forceinline__ V dir_dot(V a, V b) {
    if constexpr (CY == 0) return CX == 1 ? a : v_neg(a);
    else if constexpr (CX == 0) return CY == 1 ? b : v_neg(b);
    else if constexpr (CX == CY) return CX == 1 ? v_add(a, b) : v_neg(v_add(a, b));
    else return CX == 1 ? v_sub(a, b) : v_sub(b, a);
}

// One opposite pair (i, ip = -i) of the BGK collision with forcing.  With
// A = w (drho + rho (4.5 (v.u)^2 - 1.5 u^2)), B = 3 w rho v.u, C = 4.5 w S:(vv - theta I),
// D = 3 w v.G:  f^eq - w rho_ref = A +- B and F = C +- D (Eqs. feq, forcing terms);
// post = (1 - omega) g + omega (f^eq - w rho_ref) + F = (1 - omega) g + (omega A + C) +- (omega B + D).
template <int LAT, int I, class V>
__device__ __forceinline__ void bgk_pair(V r, V drho, V u, V v, V gx, V gy, V m15, V Sxx, V Syy, V Sxy, V omega,
                                         V omc, V gi, V gip, V &pi, V &pip) {
    using L = Lat<LAT>;
    constexpr int CX = L::vx(I), CY = L::vy(I);
    constexpr double W = L::w(I);
    const V vu = dir_dot<CX, CY>(u, v);
    const V vG = dir_dot<CX, CY>(gx, gy);
    const V t = v_fma(vu, v_mul(vu, vc<V>(4.5)), m15);
    const V A = v_fma(v_mul(r, vc<V>(W)), t, v_mul(drho, vc<V>(W)));
    const V B = v_mul(vu, v_mul(r, vc<V>(3.0 * W)));
    V C = v_mul(Sxx, vc<V>(4.5 * W * (CX * CX - 1.0 / 3.0)));
    if constexpr (LAT == 2) {
        C = v_fma(Syy, vc<V>(4.5 * W * (CY * CY - 1.0 / 3.0)), C);
        if constexpr (CX * CY != 0) C = v_fma(Sxy, vc<V>(9.0 * W * CX * CY), C);
    }
    const V D = v_mul(vG, vc<V>(3.0 * W));
    const V even = v_fma(omega, A, C), odd = v_fma(omega, B, D);
    pi = v_fma(omc, gi, v_add(even, odd));
    pip = v_fma(omc, gip, v_sub(even, odd));
}

// BGK collision with forcing of one component lane.  The second forcing moment is
// S = G u + u G - Psi, -Psi = cg G G / rho + cl Lap rho I (Eq. forceCorrectionsPsi, sigma = -1).
// The moving populations come first; the rest population takes what is left of the
// node's pre-collision mass (sum f^eq = rho and sum F = 0 make this the same value in
// exact arithmetic), so mass is conserved up to the rounding of two sums.
template <int LAT, class V>
__device__ __forceinline__ void bgk_lane(V r, V u, V v, V gx, V gy, V lapc, V ir, V rref, V omega, V omc, V cg,
                                         V cl, const V (&g)[Lat<LAT>::Q], V (&post)[Lat<LAT>::Q]) {
    constexpr int Q = Lat<LAT>::Q;
    const V cgi = v_mul(cg, ir);
    const V cll = v_mul(cl, lapc);
    const V Sxx = v_fma(gx, v_fma(gx, cgi, v_add(u, u)), cll);
    V Syy = Sxx, Sxy = Sxx, usq;
    if constexpr (LAT == 2) {
        Syy = v_fma(gy, v_fma(gy, cgi, v_add(v, v)), cll);
        Sxy = v_fma(gx, v_fma(gy, cgi, v), v_mul(u, gy));
        usq = v_fma(u, u, v_mul(v, v));
    } else {
        usq = v_mul(u, u);
    }
    const V m15 = v_mul(usq, vc<V>(-1.5));
    const V drho = v_sub(r, rref);
    V moved;
    if constexpr (LAT == 1) {
        bgk_pair<1, 1>(r, drho, u, v, gx, gy, m15, Sxx, Syy, Sxy, omega, omc, g[1], g[2], post[1], post[2]);
        moved = v_add(post[1], post[2]);
    } else {
        // pairs E/W, N/S, NE/SW, NW/SE
        bgk_pair<2, 1>(r, drho, u, v, gx, gy, m15, Sxx, Syy, Sxy, omega, omc, g[1], g[3], post[1], post[3]);
        bgk_pair<2, 2>(r, drho, u, v, gx, gy, m15, Sxx, Syy, Sxy, omega, omc, g[2], g[4], post[2], post[4]);
        bgk_pair<2, 5>(r, drho, u, v, gx, gy, m15, Sxx, Syy, Sxy, omega, omc, g[5], g[7], post[5], post[7]);
        bgk_pair<2, 6>(r, drho, u, v, gx, gy, m15, Sxx, Syy, Sxy, omega, omc, g[6], g[8], post[6], post[8]);
        moved = v_add(post[1], post[3]);
        moved = v_add(moved, v_add(post[2], post[4]));
        moved = v_add(moved, v_add(post[5], post[7]));
        moved = v_add(moved, v_add(post[6], post[8]));
    }
    V before = g[0];
#pragma unroll
    for (int i = 1; i < Q; ++i) before = v_add(before, g[i]);
    post[0] = v_sub(before, moved);
}

// One opposite pair (i, ip = -i) of the moment-space collision with forcing (D2Q9).  The
// relaxation Omega_i = w_i [Axx H_xx + Ayy H_yy + Axy H_xy + Bxxy H_xxy + Bxyy H_xyy +
// Bq H_xxyy](v_i) (amplitudes already divided by the norms of the Hermite polynomials) has
// a part even in v (orders 2 and 4) and an odd part (order 3); the forcing F = C +- D is
// that of bgk_pair.  post = g + Omega + F.
template <int I, class V>
__device__ __forceinline__ void mrt_pair(V Sxx, V Syy, V Sxy, V gx, V gy, V Axx, V Ayy, V Axy, V Bxxy, V Bxyy,
                                         V Bq, V gi, V gip, V &pi, V &pip) {
    using L = Lat<2>;
    constexpr int CX = L::vx(I), CY = L::vy(I);
    constexpr double W = L::w(I), TH = 1.0 / 3.0;
    constexpr double hxx = CX * CX - TH, hyy = CY * CY - TH, hxy = CX * CY;
    constexpr double hxxy = hxx * CY, hxyy = CX * hyy, hq = hxx * hyy;
    V even = v_mul(v_fma(Sxx, vc<V>(4.5), Axx), vc<V>(W * hxx));
    even = v_fma(v_fma(Syy, vc<V>(4.5), Ayy), vc<V>(W * hyy), even);
    if constexpr (CX * CY != 0) even = v_fma(v_fma(Sxy, vc<V>(9.0), Axy), vc<V>(W * hxy), even);
    even = v_fma(Bq, vc<V>(W * hq), even);
    V odd = v_mul(dir_dot<CX, CY>(gx, gy), vc<V>(3.0 * W));
    if constexpr (CY != 0) odd = v_fma(Bxxy, vc<V>(W * hxxy), odd);
    if constexpr (CX != 0) odd = v_fma(Bxyy, vc<V>(W * hxyy), odd);
    pi = v_add(gi, v_add(even, odd));
    pip = v_add(gip, v_sub(even, odd));
}

// Moment-space collision with forcing of one D2Q9 component lane (Eq. BGKcollisionOperator
// with the collision matrix diagonal in the Hermite basis H_a = P_ax(v_x) P_ay(v_y),
// P in {1, v, v^2 - theta}, norms N = 1, theta, 2 theta^2 per factor): the bulk moment
// H_xx + H_yy relaxes with omega (ob), the shear moments H_xx - H_yy and H_xy with
// omega_s (os), the ghost moments H_xxy, H_xyy, H_xxyy with omega_g (og); conserved
// moments are untouched.  -Psi per eigenspace: the trace of G G / rho with cgb =
// (tau - 1/4)/tau and the Laplacian term, its traceless part with cgs = (tau_s - 1/4)/tau_s.
// The rest population takes what is left of the node's mass, as in bgk_lane.
template <class V>
__device__ __forceinline__ void mrt_lane(V r, V u, V v, V gx, V gy, V lapc, V ir, V ob, V os, V og, V cgb, V cgs,
                                         V cl, const V (&g)[9], V (&post)[9]) {
    const V cp = v_mul(v_add(cgb, cgs), vc<V>(0.5)), cm = v_mul(v_sub(cgb, cgs), vc<V>(0.5));
    const V gxx = v_mul(v_mul(gx, gx), ir), gyy = v_mul(v_mul(gy, gy), ir);
    const V cll = v_mul(cl, lapc);
    const V Sxx = v_fma(gx, v_add(u, u), v_fma(cp, gxx, v_fma(cm, gyy, cll)));
    const V Syy = v_fma(gy, v_add(v, v), v_fma(cm, gxx, v_fma(cp, gyy, cll)));
    const V Sxy = v_fma(gx, v, v_fma(u, gy, v_mul(v_mul(cgs, ir), v_mul(gx, gy))));
    // Hermite moments of the stored populations (the rest equilibrium w rho_ref has none
    // beyond order zero, so deviations give those of f)
    const V ax = v_add(g[1], g[3]), ay = v_add(g[2], g[4]);
    const V dsum = v_add(v_add(g[5], g[6]), v_add(g[7], g[8]));
    const V s0 = v_add(g[0], v_add(v_add(ax, ay), dsum));
    const V Pxx = v_fma(s0, vc<V>(-1.0 / 3.0), v_add(ax, dsum));
    const V Pyy = v_fma(s0, vc<V>(-1.0 / 3.0), v_add(ay, dsum));
    const V Pxy = v_sub(v_add(g[5], g[7]), v_add(g[6], g[8]));
    const V Qxxy = v_fma(v_sub(v_add(g[5], g[6]), v_add(g[7], g[8])), vc<V>(2.0 / 3.0),
                         v_mul(v_sub(g[2], g[4]), vc<V>(-1.0 / 3.0)));
    const V Qxyy = v_fma(v_sub(v_add(g[5], g[8]), v_add(g[6], g[7])), vc<V>(2.0 / 3.0),
                         v_mul(v_sub(g[1], g[3]), vc<V>(-1.0 / 3.0)));
    const V Rq = v_fma(dsum, vc<V>(4.0 / 9.0), v_fma(v_add(ax, ay), vc<V>(-2.0 / 9.0), v_mul(g[0], vc<V>(1.0 / 9.0))));
    // m^eq - m: the equilibrium's second moments are rho u u, its ghost moments zero
    const V ru = v_mul(r, u), rv = v_mul(r, v);
    const V dxx = v_fma(ru, u, v_neg(Pxx)), dyy = v_fma(rv, v, v_neg(Pyy)), dxy = v_fma(ru, v, v_neg(Pxy));
    const V bulk = v_mul(v_add(dxx, dyy), v_mul(ob, vc<V>(2.25)));   // omega (dxx + dyy) / 2 / (2 theta^2)
    const V shear = v_mul(v_sub(dxx, dyy), v_mul(os, vc<V>(2.25)));
    const V Axx = v_add(bulk, shear), Ayy = v_sub(bulk, shear);
    const V Axy = v_mul(dxy, v_mul(os, vc<V>(9.0)));                 // / theta^2
    const V Bxxy = v_mul(Qxxy, v_mul(og, vc<V>(-13.5)));             // / (2 theta^3)
    const V Bxyy = v_mul(Qxyy, v_mul(og, vc<V>(-13.5)));
    const V Bq = v_mul(Rq, v_mul(og, vc<V>(-20.25)));                // / (4 theta^4)
    mrt_pair<1>(Sxx, Syy, Sxy, gx, gy, Axx, Ayy, Axy, Bxxy, Bxyy, Bq, g[1], g[3], post[1], post[3]);
    mrt_pair<2>(Sxx, Syy, Sxy, gx, gy, Axx, Ayy, Axy, Bxxy, Bxyy, Bq, g[2], g[4], post[2], post[4]);
    mrt_pair<5>(Sxx, Syy, Sxy, gx, gy, Axx, Ayy, Axy, Bxxy, Bxyy, Bq, g[5], g[7], post[5], post[7]);
    mrt_pair<6>(Sxx, Syy, Sxy, gx, gy, Axx, Ayy, Axy, Bxxy, Bxyy, Bq, g[6], g[8], post[6], post[8]);
    V moved = v_add(post[1], post[3]);
    moved = v_add(moved, v_add(post[2], post[4]));
    moved = v_add(moved, v_add(post[5], post[7]));
    moved = v_add(moved, v_add(post[6], post[8]));
    post[0] = v_sub(s0, moved);
}

// Friction of two components with the implicit u-hat: (D + L/2) h = -L u0, G^f = D h per
// direction (Eq. forceFriction).  L is rank one and the friction conserves momentum
// (rho^1 h^1 = -rho^2 h^2), which leaves one unknown:
//   G^{f,1} = -k (u0^1 - u0^2) = -G^{f,2},  k = [lambda / (1 + lambda/2)] rho^1 rho^2 / (rho^1 + rho^2),
// u0^c = u^c + G^c / (2 rho^c) -- the system's exact solution.
template <class T>
__device__ __forceinline__ T friction_k(T r0, T r1, T lam_fr) {
    return v_mul(v_mul(v_mul(lam_fr, r0), r1), v_rcp(v_add(r0, r1)));
}

// both components in one lane pair (x: component 1, y: component 2)
__device__ __forceinline__ float2 friction_pair(float k, float2 G, float2 u, float2 ir) {
    const float2 t = v_fma(G, v_mul(ir, vc<float2>(0.5)), u);
    const float d = __fsub_rn(t.x, t.y);
    return v_add(G, make_float2(__fmul_rn(-k, d), __fmul_rn(k, d)));
}

// one component per lane
template <class T>
__device__ __forceinline__ void friction_two(T k, T (&G)[2], const T (&u)[2], const T (&ir)[2]) {
    const T t0 = v_fma(G[0], v_mul(ir[0], vc<T>(0.5)), u[0]);
    const T t1 = v_fma(G[1], v_mul(ir[1], vc<T>(0.5)), u[1]);
    const T d = v_sub(t0, t1);
    G[0] = v_add(G[0], v_mul(-k, d));
    G[1] = v_add(G[1], v_mul(k, d));
}

// Friction of N > 2 components, one component per lane: (D + L/2) h = -L u0, G^f = D h per
// direction (Eq. forceFriction), with W^{cc'} = lambda^{cc'} rho^c rho^c' / (rho^c + rho^c'),
// L the weighted Laplacian of W and u0 = u + G / (2 rho).  D + L/2 is symmetric positive
// definite: elimination without pivoting.
template <int N, int DIM, class T>
__device__ __forceinline__ void friction_n(const T (&rho)[N], const T (&ir)[N], const T (&ux)[N], const T (&uy)[N],
                                           const DevParams &P, T (&Gx)[N], T (&Gy)[N]) {
    T W[N][N];
#pragma unroll
    for (int c = 0; c < N; ++c) {
        W[c][c] = vc<T>(0.0);
#pragma unroll
        for (int cc = c + 1; cc < N; ++cc) {
            const T lam = pv<T>(P.lam[c * 4 + cc], P.lam_f[c * 4 + cc]);
            W[c][cc] = v_mul(v_mul(v_mul(lam, rho[c]), rho[cc]), v_rcp(v_add(rho[c], rho[cc])));
            W[cc][c] = W[c][cc];
        }
    }
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        T u0[N], M[N][N], h[N];
#pragma unroll
        for (int c = 0; c < N; ++c) {
            const T gg = d == 0 ? Gx[c] : Gy[c];
            u0[c] = v_fma(v_mul(gg, vc<T>(0.5)), ir[c], d == 0 ? ux[c] : uy[c]);
        }
#pragma unroll
        for (int c = 0; c < N; ++c) {
            T diag = rho[c], rhs = vc<T>(0.0);
#pragma unroll
            for (int cc = 0; cc < N; ++cc) {
                if (cc == c) continue;
                M[c][cc] = v_mul(W[c][cc], vc<T>(-0.5));
                diag = v_fma(W[c][cc], vc<T>(0.5), diag);
                rhs = v_fma(v_neg(W[c][cc]), v_sub(u0[c], u0[cc]), rhs);
            }
            M[c][c] = diag;
            h[c] = rhs;
        }
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const T inv = v_rcp(M[k][k]);
#pragma unroll
            for (int r2 = k + 1; r2 < N; ++r2) {
                const T m = v_mul(M[r2][k], inv);
#pragma unroll
                for (int c2 = k + 1; c2 < N; ++c2) M[r2][c2] = v_fma(v_neg(m), M[k][c2], M[r2][c2]);
                h[r2] = v_fma(v_neg(m), h[k], h[r2]);
            }
        }
#pragma unroll
        for (int k = N - 1; k >= 0; --k) {
            T sacc = h[k];
#pragma unroll
            for (int c2 = k + 1; c2 < N; ++c2) sacc = v_fma(v_neg(M[k][c2]), h[c2], sacc);
            h[k] = v_mul(sacc, v_rcp(M[k][k]));
        }
#pragma unroll
        for (int c = 0; c < N; ++c) {
            if (d == 0) Gx[c] = v_fma(rho[c], h[c], Gx[c]);
            else Gy[c] = v_fma(rho[c], h[c], Gy[c]);
        }
    }
}

// One node of phase 3 for NP component pairs (components 2q, 2q+1 in lane pair q): from rho,
// Lap rho, D phi, D rho ("log" force) and the bare momenta, the total gain G (mean field +
// implicit friction), then Psi, the forcing populations and the BGK collision.  g holds
// the node's stored populations (deviations); post receives the post-collision deviations.
template <int LAT, int NP, int FORCE>
__device__ __forceinline__ void collide_pairs(const float2 (&rho)[NP], const float2 (&lap)[NP],
                                              const float2 (&gpx)[NP], const float2 (&gpy)[NP],
                                              const float2 (&grx)[NP], const float2 (&gry)[NP],
                                              const float2 (&jx)[NP], const float2 (&jy)[NP], const DevParams &P,
                                              const float2 (&g)[NP][Lat<LAT>::Q], float2 (&post)[NP][Lat<LAT>::Q]) {
    float2 Gx[NP], Gy[NP], ir[NP], ux[NP], uy[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q)
        gain_lane<FORCE>(rho[q], gpx[q], gpy[q], grx[q], gry[q], jx[q], jy[q], Gx[q], Gy[q], ir[q], ux[q], uy[q]);
    if constexpr (NP == 1) {
        const float k = friction_k(rho[0].x, rho[0].y, P.lam_fr_f);
        Gx[0] = friction_pair(k, Gx[0], ux[0], ir[0]);
        if constexpr (LAT == 2) Gy[0] = friction_pair(k, Gy[0], uy[0], ir[0]);
    } else {
        constexpr int N = 2 * NP;
        float r1[N], i1[N], ux1[N], uy1[N], gx1[N], gy1[N];
#pragma unroll
        for (int c = 0; c < N; ++c) {
            r1[c] = comp(rho, c), i1[c] = comp(ir, c), ux1[c] = comp(ux, c), uy1[c] = comp(uy, c);
            gx1[c] = comp(Gx, c), gy1[c] = comp(Gy, c);
        }
        friction_n<N, Lat<LAT>::D, float>(r1, i1, ux1, uy1, P, gx1, gy1);
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            Gx[q] = make_float2(gx1[2 * q], gx1[2 * q + 1]);
            Gy[q] = make_float2(gy1[2 * q], gy1[2 * q + 1]);
        }
    }
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        if constexpr (Flags<FORCE>::mrt && LAT == 2)
            mrt_lane<float2>(rho[q], ux[q], uy[q], Gx[q], Gy[q], lap[q], ir[q], make_float2(P.omega_f, P.omega_f),
                             make_float2(P.omega_s_f, P.omega_s_f), make_float2(P.omega_g_f, P.omega_g_f),
                             make_float2(P.psi_g_f, P.psi_g_f), make_float2(P.psi_s_f, P.psi_s_f),
                             make_float2(P.psi_l_f, P.psi_l_f), g[q], post[q]);
        else
            bgk_lane<LAT, float2>(rho[q], ux[q], uy[q], Gx[q], Gy[q], lap[q], ir[q],
                                  make_float2(P.rho_ref_f[2 * q], P.rho_ref_f[2 * q + 1]),
                                  make_float2(P.omega_f, P.omega_f), make_float2(P.omc_f, P.omc_f),
                                  make_float2(P.psi_g_f, P.psi_g_f), make_float2(P.psi_l_f, P.psi_l_f), g[q], post[q]);
    }
}

// One node of phase 3, N components (arrays over c); an even number of FP32 components goes
// through the lane-pair form above, with bitwise the same result as one component at a time.
template <int LAT, int N, class R, int FORCE>
__device__ __forceinline__ void collide_node(const R (&rho)[N], const R (&lap)[N], const R (&gpx)[N],
                                             const R (&gpy)[N], const R (&grx)[N], const R (&gry)[N],
                                             const R (&jx)[N], const R (&jy)[N], const DevParams &P,
                                             const R (&g)[N][Lat<LAT>::Q], R (&post)[N][Lat<LAT>::Q]) {
    using L = Lat<LAT>;
    constexpr int Q = L::Q;
    if constexpr (N % 2 == 0 && sizeof(R) == 4) {
        constexpr int NP = N / 2;
        float2 r2[NP], l2[NP], px[NP], py[NP], qx[NP], qy[NP], ax[NP], ay[NP], g2[NP][Q], p2[NP][Q];
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const int c = 2 * q;
            r2[q] = make_float2(rho[c], rho[c + 1]), l2[q] = make_float2(lap[c], lap[c + 1]);
            px[q] = make_float2(gpx[c], gpx[c + 1]), py[q] = make_float2(gpy[c], gpy[c + 1]);
            qx[q] = make_float2(grx[c], grx[c + 1]), qy[q] = make_float2(gry[c], gry[c + 1]);
            ax[q] = make_float2(jx[c], jx[c + 1]), ay[q] = make_float2(jy[c], jy[c + 1]);
#pragma unroll
            for (int i = 0; i < Q; ++i) g2[q][i] = make_float2(g[c][i], g[c + 1][i]);
        }
        collide_pairs<LAT, NP, FORCE>(r2, l2, px, py, qx, qy, ax, ay, P, g2, p2);
#pragma unroll
        for (int q = 0; q < NP; ++q)
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                post[2 * q][i] = p2[q][i].x;
                post[2 * q + 1][i] = p2[q][i].y;
            }
    } else {
        R ux[N], uy[N], Gx[N], Gy[N], ir[N];
#pragma unroll
        for (int c = 0; c < N; ++c) gain_lane<FORCE>(rho[c], gpx[c], gpy[c], grx[c], gry[c], jx[c], jy[c], Gx[c],
                                                     Gy[c], ir[c], ux[c], uy[c]);
        if constexpr (N == 2) {
            const R k = friction_k(rho[0], rho[1], pv<R>(P.lam_fr, P.lam_fr_f));
            friction_two(k, Gx, ux, ir);
            if constexpr (L::D == 2) friction_two(k, Gy, uy, ir);
        } else if constexpr (N > 2) {
            friction_n<N, L::D, R>(rho, ir, ux, uy, P, Gx, Gy);
        }
        const R omega = pv<R>(P.omega, P.omega_f), omc = pv<R>(P.omc, P.omc_f);
        const R cg = pv<R>(P.psi_g, P.psi_g_f), cl = pv<R>(P.psi_l, P.psi_l_f);
#pragma unroll
        for (int c = 0; c < N; ++c) {
            if constexpr (Flags<FORCE>::mrt && LAT == 2)
                mrt_lane<R>(rho[c], ux[c], uy[c], Gx[c], Gy[c], lap[c], ir[c], omega, pv<R>(P.omega_s, P.omega_s_f),
                            pv<R>(P.omega_g, P.omega_g_f), cg, pv<R>(P.psi_s, P.psi_s_f), cl, g[c], post[c]);
            else
                bgk_lane<LAT, R>(rho[c], ux[c], uy[c], Gx[c], Gy[c], lap[c], ir[c],
                                 pv<R>(P.rho_ref[c], P.rho_ref_f[c]), omega, omc, cg, cl, g[c], post[c]);
        }
    }
}

// Tile geometry of the fused step: densities on the tile plus a 2-node ring, mu on the
// tile plus a 1-node ring; the ring of the density array in one flat index k.
template <int LAT, int TX, int TY>
struct TileGeom {
    static constexpr int HY = Lat<LAT>::HY;
    static constexpr int EX = TX + 4, EY = TY + 4 * HY;  // densities: tile + 2 ring
    static constexpr int MX = TX + 2, MY = TY + 2 * HY;  // mu: tile + 1 ring
    static constexpr int NT = TX * TY;
    static constexpr int RING = EX * EY - TX * TY;
    __device__ static __forceinline__ void ring_node(int k, int &ex, int &ey) {
        if constexpr (LAT == 1) {
            ey = 0;
            ex = k < 2 ? k : EX - 4 + k;
        } else {
            if (k < 2 * EX) {
                ey = k / EX;
                ex = k - ey * EX;
            } else if (k < 4 * EX) {
                int kk = k - 2 * EX;
                ey = EY - 2 + kk / EX;
                ex = kk % EX;
            } else {
                int kk = k - 4 * EX;
                ey = 2 + (kk >> 2);
                int col = kk & 3;
                ex = col < 2 ? col : EX - 4 + col;
            }
        }
    }
};

// Whether a step runs in lane pairs: an even number of FP32 components, FP32-class mu.
template <int N, class S, class R, int MU>
struct PairPath {
    static constexpr bool value = N % 2 == 0 && sizeof(S) == 4 && sizeof(R) == 4 && (MU == MU_DF || MU == MU_F32);
};

// A load of a stored population: plain (LD = 0; the read-only path where the compiler can
// prove it) or cached in L2 only (LD = 1), for the chained steps of lb_chain.cuh, whose
// input may still be written by the previous step's grid while this one runs.
template <int LD>
__device__ __forceinline__ float ld_pop(const float *p) {
    if constexpr (LD == 1) return __ldcg(p);
    else return *p;
}

// An L2 cache policy that marks the lines it touches first for eviction (PTX createpolicy)
__device__ __forceinline__ unsigned long long l2_evict_first_policy() {
    unsigned long long q;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(q));
    return q;
}

// The L2-only load of a chained step with an L2 cache policy.  A step reads its input once
// (and its ring again within the step) and never after, so where one population buffer
// fits in the L2 with room to spare, marking the input evict-first keeps the output just
// written resident for the next step's reads.
__device__ __forceinline__ float ld_pop_policy(const float *p, unsigned long long pol) {
    float v;
    asm volatile("ld.global.cg.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}

// What a tile step needs before it reads its parameter block (its densities phase): the
// lattice size, the log tables and the components' reference densities.  The single-run
// kernels take them from the parameter block itself (a kernel parameter); the batched tile
// kernel from its tile entry, so that its populations are requested while the run's
// parameter block is still on its way into shared memory.
struct TileGeo {
    int nx, ny;
    const LogTables *tbl;
    float rho_ref[4];
    unsigned long long l2_pol = 0;  // L2 policy of the population loads (EF steps)
};

// The default hook of step_tile_pair: nothing before the first barrier.
struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

// The fused step, FP32 components in lane pairs (NP pairs: components 2q and 2q+1 in pair q):
// every per-node quantity of a pair lives in one register pair (densities, momenta, mu,
// forces, populations) and is computed by the packed FP32x2 instructions; shared memory
// holds the pairs interleaved, so one 8-byte (16-byte for double-float mu) access moves
// both components.  Same arithmetic as the general step_tile below, bitwise.
// The densities phase reads only `geo`; `hook` runs on every thread at its end, before the
// first barrier, after which P is read (the batched kernel completes its parameter block
// in shared memory there).  EF (one pair, L2-only loads): the population loads carry the
// evict-first policy geo.l2_pol.
template <int LAT, int NP, int TX, int TY, int FORCE, int MU, int LD = 0, class Hook = NoHook, bool EF = false>
__device__ __forceinline__ void step_tile_pair(const float *__restrict__ fin, float *__restrict__ fout,
                                               const DevParams &P, int x0, int y0, const TileGeo geo,
                                               const Hook &hook) {
    using L = Lat<LAT>;
    using G = TileGeom<LAT, TX, TY>;
    constexpr int Q = L::Q, HY = G::HY, EX = G::EX, MX = G::MX, MY = G::MY, NT = G::NT;
    static_assert(MU == MU_DF || MU == MU_F32, "lane pairs need an FP32-class mu");
    using PT = typename std::conditional<MU == MU_DF, float4, float2>::type;  // phi pair: (hi, hi, lo, lo) / (x, y)

    // the node's own populations wait in shared memory between phases 1 and 3 (one pair,
    // tiles of up to 256 threads), or are read again from global memory (the L2) in phase 3
    // (two pairs: holding them would cost 36 registers and half the resident CTAs), else
    // they wait in registers
    constexpr bool STAGE = NP == 1 && NT <= 256;
    constexpr bool RELOAD = NP > 1;
    __shared__ float2 s_g[STAGE ? Q : 1][STAGE ? NT : 1];
    float2 gk[STAGE || RELOAD ? 1 : NP][STAGE || RELOAD ? 1 : Q];
    __shared__ float2 s_rho[NP][G::EY * EX];
    __shared__ PT s_phi[NP][MY * MX];
    __shared__ __align__(16) float s_tbl[TblWords<MU>::value];

    const int nx = geo.nx, ny = geo.ny;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = tx + TX * ty;
    const int x = x0 + tx, y = y0 + ty;
    const bool inside = x < nx && y < ny;
    load_tables<MU>(s_tbl, geo.tbl, tid, NT);
    const size_t plane = (size_t)nx * (size_t)ny;
    const size_t cq = (size_t)Q * plane;  // component stride
    const bool small = nx <= TX + 1 || (LAT == 2 && ny <= TY + 1);
    auto rref = [&](int q) { return make_float2(geo.rho_ref[2 * q], geo.rho_ref[2 * q + 1]); };

    // One pair: 32-bit element offsets within a component's Q planes (Q nx ny < 2^32 for
    // FP32 storage, checked when the context is created) from per-component base pointers,
    // which saves address arithmetic; two pairs keep 64-bit addressing (the extra base
    // pointers would spill at their 64 registers).
    const unsigned pl = (unsigned)plane;
    // element e of plane i of component c, from the node offset o of plane 0
    static_assert(!EF || (NP == 1 && LD == 1), "evict-first loads: one pair, L2-only loads");
    auto ld = [&](int c, int i, unsigned o) -> float {
        if constexpr (EF) return ld_pop_policy(&(fin + c * cq)[i * pl + o], geo.l2_pol);
        else if constexpr (NP == 1) return ld_pop<LD>(&(fin + c * cq)[i * pl + o]);
        else return ld_pop<LD>(&fin[(size_t)c * cq + (size_t)i * plane + o]);
    };
    // ---- phase 1a: own node -> shared (populations, densities) ------------------
    float2 jx[NP], jy[NP];
    {
        const int gx = small ? wrap(x, nx) : wrap1(x, nx);
        const int gy = LAT == 1 ? 0 : (small ? wrap(y, ny) : wrap1(y, ny));
        const unsigned off = (unsigned)gy * (unsigned)nx + (unsigned)gx;
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            float2 gv[Q], acc;
#pragma unroll
            for (int i = 0; i < Q; ++i) gv[i] = make_float2(ld(2 * q, i, off), ld(2 * q + 1, i, off));
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if constexpr (STAGE) s_g[i][tid] = gv[i];
                else if constexpr (!RELOAD) gk[q][i] = gv[i];
            }
            moments_lane<LAT>(gv, acc, jx[q], jy[q]);
            s_rho[q][(ty + 2 * HY) * EX + tx + 2] = v_add(rref(q), acc);
        }
    }
    // ---- phase 1b: densities on the 2-node ring ---------------------------------
    for (int k = tid; k < G::RING; k += NT) {
        int ex, ey;
        G::ring_node(k, ex, ey);
        const int gx = small ? wrap(x0 + ex - 2, nx) : wrap1(x0 + ex - 2, nx);
        const int gy = (LAT == 1) ? 0 : (small ? wrap(y0 + ey - 2, ny) : wrap1(y0 + ey - 2, ny));
        const unsigned off = (unsigned)gy * (unsigned)nx + (unsigned)gx;
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            float2 acc = make_float2(ld(2 * q, 0, off), ld(2 * q + 1, 0, off));
#pragma unroll
            for (int i = 1; i < Q; ++i) acc = v_add(acc, make_float2(ld(2 * q, i, off), ld(2 * q + 1, i, off)));
            s_rho[q][ey * EX + ex] = v_add(rref(q), acc);
        }
    }
    hook();
    __syncthreads();

    // ---- phase 2: phi on tile + 1 ring --------------------------------------------
    unsigned bad = 0;
    // phi at mu node k (into s_phi when store); false outside the domain
    auto mu_at = [&](int k, bool store) {
        const int mx = k % MX, my = k / MX;
        const int e = (my + HY) * EX + mx + 1;
        float2 r[NP], lp[NP], lin[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            r[q] = s_rho[q][e];
            if constexpr (LAT == 1) lp[q] = lap_d1q3(r[q], s_rho[q][e + 1], s_rho[q][e - 1]);
            else lp[q] = lap_d2q9(nbr9(s_rho[q] + e, EX));
        }
        lin_pairs<NP>(r, lp, P, lin);
        bool ok;
        if constexpr (MU == MU_DF) {
            DF<float2> ph[NP];
            ok = mu_pairs_df<NP, FORCE>(r, lin, P, reinterpret_cast<const float4 *>(s_tbl), ph);
#pragma unroll
            for (int q = 0; q < NP; ++q)
                if (store) s_phi[q][k] = make_float4(ph[q].hi.x, ph[q].hi.y, ph[q].lo.x, ph[q].lo.y);
        } else {
            float2 ph[NP];
            ok = mu_pairs_f32<NP, FORCE>(r, lin, P, ph);
#pragma unroll
            for (int q = 0; q < NP; ++q)
                if (store) s_phi[q][k] = ph[q];
        }
        return ok || !store;
    };
    if constexpr (MX * MY > NT && MX * MY <= 2 * NT) {
        // warps with second-round mu nodes evaluate both of a thread's nodes in one
        // straight-line stream, two independent dependency chains (the second round otherwise
        // runs alone on a third of the warps); a lane without a second node repeats its first
        // without storing it
        if ((tid & ~31) + NT < MX * MY) {
            const bool has2 = tid + NT < MX * MY;
            const bool ok1 = mu_at(tid, true);
            const bool ok2 = mu_at(has2 ? tid + NT : tid, has2);
            if (!(ok1 && ok2)) bad = 1;
        } else if (!mu_at(tid, true)) {
            bad = 1;
        }
    } else {
        for (int k = tid; k < MX * MY; k += NT)
            if (!mu_at(k, true)) bad = 1;
    }
    __syncthreads();
    if (bad) atomicOr(P.err, ERR_DOMAIN);
    if (!inside) return;

    // ---- phase 3: forces, collision, streaming ----------------------------------
    const int e = (ty + 2 * HY) * EX + tx + 2;
    const int m = (ty + HY) * MX + tx + 1;
    float2 rho[NP], lap[NP], grx[NP], gry[NP], gpx[NP], gpy[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const float2 *sr = s_rho[q];
        const PT *sp = s_phi[q];
        auto phi_at = [&](int k) {
            if constexpr (MU == MU_DF) {
                const float4 t = sp[k];
                return DF<float2>{make_float2(t.x, t.y), make_float2(t.z, t.w)};
            } else {
                return sp[k];
            }
        };
        rho[q] = sr[e];
        if constexpr (LAT == 1) {
            lap[q] = lap_d1q3(rho[q], sr[e + 1], sr[e - 1]);
            grx[q] = !Flags<FORCE>::nid ? grad_d1q3(sr[e + 1], sr[e - 1]) : vc<float2>(0.0);
            gry[q] = vc<float2>(0.0);
            gpx[q] = v_mul(phi_diff2(phi_at(m + 1), phi_at(m - 1)), vs(P.gkt2_f, rho[q]));
            gpy[q] = vc<float2>(0.0);
        } else {
            const Nbr9<float2> nb = nbr9(sr + e, EX);
            lap[q] = lap_d2q9(nb);
            if constexpr (!Flags<FORCE>::nid) grad_d2q9(nb, grx[q], gry[q]);
            else grx[q] = gry[q] = vc<float2>(0.0);
            grad_d2q9_diff(phi_diff2(phi_at(m + 1), phi_at(m - 1)), phi_diff2(phi_at(m + MX), phi_at(m - MX)),
                           phi_diff2(phi_at(m + MX + 1), phi_at(m - MX - 1)),  // NE - SW
                           phi_diff2(phi_at(m - MX + 1), phi_at(m + MX - 1)),  // SE - NW
                           vs(P.gkt3_f, rho[q]), vs(P.gkt12_f, rho[q]), gpx[q], gpy[q]);
        }
    }
    float2 gr[NP][Q], post[NP][Q];
#pragma unroll
    for (int q = 0; q < NP; ++q)
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if constexpr (STAGE) gr[q][i] = s_g[i][tid];
            else if constexpr (RELOAD) {
                const float *sq = fin + (size_t)y * nx + x + 2 * q * cq;
                gr[q][i] = make_float2(ld_pop<LD>(&sq[(size_t)i * plane]), ld_pop<LD>(&sq[cq + (size_t)i * plane]));
            } else gr[q][i] = gk[q][i];
        }
    collide_pairs<LAT, NP, FORCE>(rho, lap, gpx, gpy, grx, gry, jx, jy, P, gr, post);

    // push streaming to the periodic neighbours
    const int xe = small ? wrap(x + 1, nx) : (x + 1 == nx ? 0 : x + 1);
    const int xw = small ? wrap(x - 1, nx) : (x == 0 ? nx - 1 : x - 1);
    const int yn = LAT == 1 ? 0 : (small ? wrap(y + 1, ny) : (y + 1 == ny ? 0 : y + 1));
    const int ys = LAT == 1 ? 0 : (small ? wrap(y - 1, ny) : (y == 0 ? ny - 1 : y - 1));
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = L::vx(i), cy = L::vy(i);
        const int dx = cx == 1 ? xe : (cx == -1 ? xw : x);
        const int dy = cy == 1 ? yn : (cy == -1 ? ys : y);
        if constexpr (NP == 1) {
            const unsigned o = i * pl + (unsigned)dy * (unsigned)nx + (unsigned)dx;
            fout[o] = post[0][i].x;
            (fout + cq)[o] = post[0][i].y;
        } else {
            float *dst = fout + (size_t)i * plane + (size_t)dy * nx + dx;
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                dst[2 * q * cq] = post[q][i].x;
                dst[(2 * q + 1) * cq] = post[q][i].y;
            }
        }
    }
}

// The lane-pair step with its geometry from the parameter block.
template <int LAT, int NP, int TX, int TY, int FORCE, int MU, int LD = 0, bool EF = false>
__device__ __forceinline__ void step_tile_pair(const float *__restrict__ fin, float *__restrict__ fout,
                                               const DevParams &P, int x0, int y0) {
    step_tile_pair<LAT, NP, TX, TY, FORCE, MU, LD, NoHook, EF>(
        fin, fout, P, x0, y0,
        TileGeo{P.nx, P.ny, P.tbl, {P.rho_ref_f[0], P.rho_ref_f[1], P.rho_ref_f[2], P.rho_ref_f[3]},
                EF ? l2_evict_first_policy() : 0ull},
        NoHook());
}

// The fused step on one TX x TY tile with origin (x0, y0) of the lattice described by P.
template <int LAT, int N, int TX, int TY, class S, class R, int FORCE, int MU>
__device__ __forceinline__ void step_tile(const S *__restrict__ fin, S *__restrict__ fout, const DevParams &P,
                                          int x0, int y0) {
    if constexpr (PairPath<N, S, R, MU>::value) {
        step_tile_pair<LAT, N / 2, TX, TY, FORCE, MU>(fin, fout, P, x0, y0);
    } else {
    using L = Lat<LAT>;
    using G = TileGeom<LAT, TX, TY>;
    using MT = typename MuStore<MU>::T;
    constexpr int Q = L::Q;
    constexpr int HY = L::HY;
    constexpr int EX = G::EX, EY = G::EY, MX = G::MX, MY = G::MY, NT = G::NT;
    // Between phase 1 and phase 3 the node's own populations wait in shared memory (FP32
    // storage, up to two components, 256-thread tiles: this frees registers for the mu
    // phase), else in registers when they fit comfortably, else they are loaded again in
    // phase 3.
    constexpr bool STAGE = sizeof(S) == 4 && N <= 2 && NT <= 256;
    constexpr bool KEEP = !STAGE && sizeof(S) * N * Q <= 144;
    __shared__ S s_g[STAGE ? N * Q : 1][STAGE ? NT : 1];
    static_assert(MU == MU_F64 ? sizeof(R) == 8 : sizeof(R) == 4, "MU and R mismatch");

    __shared__ R s_rho[N][EY * EX];
    // gamma mu (log) or gamma mu - theta ln rho (nid); divided by gamma kT for FP32-class mu
    __shared__ MT s_phi[N][MY * MX];
    __shared__ __align__(16) float s_tbl[TblWords<MU>::value];

    const int nx = P.nx, ny = P.ny;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = tx + TX * ty;
    const int x = x0 + tx, y = y0 + ty;
    const bool inside = x < nx && y < ny;
    load_tables<MU>(s_tbl, P, tid, NT);

    // ---- phase 1a: own node -> registers, rho^c -> shared -------------------
    const size_t plane = (size_t)nx * (size_t)ny;
    // lattices at least a tile plus its ring wide wrap with one conditional add
    const bool small = nx <= TX + 1 || (LAT == 2 && ny <= TY + 1);
    S g[KEEP ? N : 1][KEEP ? Q : 1];
    R jx[N], jy[N];
    {
        const int gx = small ? wrap(x, nx) : wrap1(x, nx);
        const int gy = LAT == 1 ? 0 : (small ? wrap(y, ny) : wrap1(y, ny));
        const S *src = fin + (size_t)gy * nx + gx;
        const int ex = tx + 2, ey = ty + 2 * HY;
#pragma unroll
        for (int c = 0; c < N; ++c) {
            R gv[Q], acc;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                S v = src[(size_t)(c * Q + i) * plane];
                if constexpr (KEEP) g[c][i] = v;
                if constexpr (STAGE) s_g[c * Q + i][tid] = v;
                gv[i] = (R)v;
            }
            moments_lane<LAT>(gv, acc, jx[c], jy[c]);
            s_rho[c][ey * EX + ex] = v_add(pv<R>(P.rho_ref[c], P.rho_ref_f[c]), acc);
        }
    }
    // ---- phase 1b: rho^c on the 2-node ring -----------------------------------
    for (int k = tid; k < G::RING; k += NT) {
        int ex, ey;
        G::ring_node(k, ex, ey);
        const int gx = small ? wrap(x0 + ex - 2, nx) : wrap1(x0 + ex - 2, nx);
        const int gy = (LAT == 1) ? 0 : (small ? wrap(y0 + ey - 2, ny) : wrap1(y0 + ey - 2, ny));
        const S *src = fin + (size_t)gy * nx + gx;
#pragma unroll
        for (int c = 0; c < N; ++c) {
            R acc = (R)src[(size_t)(c * Q) * plane];
#pragma unroll
            for (int i = 1; i < Q; ++i) acc = v_add(acc, (R)src[(size_t)(c * Q + i) * plane]);
            s_rho[c][ey * EX + ex] = v_add(pv<R>(P.rho_ref[c], P.rho_ref_f[c]), acc);
        }
    }
    __syncthreads();

    // ---- phase 2: phi^c on tile + 1 ring --------------------------------------
    unsigned bad = 0;
    for (int k = tid; k < MX * MY; k += NT) {
        const int mx = k % MX, my = k / MX;
        const int ex = mx + 1, ey = my + HY;
        R r[N], lp[N], lin[N];
#pragma unroll
        for (int c = 0; c < N; ++c) {
            r[c] = s_rho[c][ey * EX + ex];
            lp[c] = lap_at<LAT, R>(s_rho[c], ex, ey, EX);
        }
        lin_node<N, R>(r, lp, P, lin);
        MT phi[N];
        if (!mu_node<N, R, FORCE, MU>(r, lin, P, s_tbl, phi)) bad = 1;
#pragma unroll
        for (int c = 0; c < N; ++c) s_phi[c][k] = phi[c];
    }
    __syncthreads();
    if (bad) atomicOr(P.err, ERR_DOMAIN);
    if (!inside) return;

    // ---- phase 3: forces, collision, streaming --------------------------------
    const int ex = tx + 2, ey = ty + 2 * HY;
    const int mx = tx + 1, my = ty + HY;
    R rho[N], lap[N], gpx[N], gpy[N], grx[N], gry[N];
#pragma unroll
    for (int c = 0; c < N; ++c) {
        rho[c] = s_rho[c][ey * EX + ex];
        lap[c] = lap_at<LAT, R>(s_rho[c], ex, ey, EX);
        grad_phi<LAT, R, MT>(s_phi[c], mx, my, MX, P, gpx[c], gpy[c]);
        if constexpr (!Flags<FORCE>::nid) grad_at<LAT, R>(s_rho[c], ex, ey, EX, grx[c], gry[c]);
        else grx[c] = gry[c] = (R)0;
    }
    R gr[N][Q], post[N][Q];
#pragma unroll
    for (int c = 0; c < N; ++c)
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if constexpr (KEEP) gr[c][i] = (R)g[c][i];
            else if constexpr (STAGE) gr[c][i] = (R)s_g[c * Q + i][tid];
            else gr[c][i] = (R)fin[(size_t)(c * Q + i) * plane + (size_t)y * nx + x];
        }
    collide_node<LAT, N, R, FORCE>(rho, lap, gpx, gpy, grx, gry, jx, jy, P, gr, post);

    // push streaming to the periodic neighbours
    const int xe = small ? wrap(x + 1, nx) : (x + 1 == nx ? 0 : x + 1);
    const int xw = small ? wrap(x - 1, nx) : (x == 0 ? nx - 1 : x - 1);
    const int yn = LAT == 1 ? 0 : (small ? wrap(y + 1, ny) : (y + 1 == ny ? 0 : y + 1));
    const int ys = LAT == 1 ? 0 : (small ? wrap(y - 1, ny) : (y == 0 ? ny - 1 : y - 1));
#pragma unroll
    for (int c = 0; c < N; ++c)
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int cx = L::vx(i), cy = L::vy(i);
            const int dx = cx == 1 ? xe : (cx == -1 ? xw : x);
            const int dy = cy == 1 ? yn : (cy == -1 ? ys : y);
            fout[(size_t)(c * Q + i) * plane + (size_t)dy * nx + dx] = (S)post[c][i];
        }
    }
}

// FP32 storage, 256-thread tiles: ask for five resident CTAs per SM with up to two
// components (48 registers); four for four components in lane pairs (64 registers: their
// populations are read again in phase 3 rather than held); two otherwise (128 registers).
// More resident warps hide the barrier waits between the phases.
template <class S, int N, int NT, bool PAIR>
struct MinBlocks {
    static constexpr int value = (sizeof(S) == 4 && NT == 256) ? (N <= 2 ? 5 : (PAIR && N == 4 ? 4 : 2)) : 1;
};

template <int LAT, int N, int TX, int TY, class S, class R, int FORCE, int MU>
__global__ void __launch_bounds__(TX *TY, MinBlocks<S, N, TX * TY, PairPath<N, S, R, MU>::value>::value)
    lb_step_kernel(const S *__restrict__ fin, S *__restrict__ fout, DevParams P) {
    step_tile<LAT, N, TX, TY, S, R, FORCE, MU>(fin, fout, P, blockIdx.x * TX, blockIdx.y * TY);
}

// ---------------------------------------------------------------------------
// equilibrium initialisation (Eq. feq at theta = 1/3), stored as deviations
// ---------------------------------------------------------------------------
template <int LAT, int N, class S>
__global__ void lb_init_kernel(S *__restrict__ f, const double *__restrict__ rho,
                               const double *__restrict__ mom, DevParams P) {
    using L = Lat<LAT>;
    constexpr int Q = L::Q, D = L::D;
    const size_t n = (size_t)P.nx * P.ny;
    for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < n; s += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(s % P.nx), y = (int)(s / P.nx);
        double eta = 1.0;
        bool ok = true;
#pragma unroll
        for (int c = 0; c < N; ++c) {
            double r = rho[c * n + s];
            eta -= P.b[c] * r;
            ok = ok && (r > 0.0) && isfinite(r);
        }
        if (!(ok && eta > 0.0)) atomicOr(P.err, ERR_DOMAIN);
#pragma unroll
        for (int c = 0; c < N; ++c) {
            double r = rho[c * n + s];
            double u = 0.0, v = 0.0;
            if (mom) {
                u = mom[(c * D + 0) * n + s] / r;
                if (D == 2) v = mom[(c * D + 1) * n + s] / r;
            }
            double usq = u * u + v * v;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                double vu = L::vx(i) * u + L::vy(i) * v;
                double wi = L::w(i);
                double dev = wi * (r - P.rho_ref[c]) + wi * r * (3.0 * vu + 4.5 * vu * vu - 1.5 * usq);
                f[pop_index(c, i, Q, y, x, P.nx, P.ny)] = (S)dev;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// moments rho^c, j^c (FP64 out) of the stored state
// ---------------------------------------------------------------------------
template <int LAT, int N, class S>
__global__ void lb_moments_kernel(const S *__restrict__ f, double *__restrict__ rho,
                                  double *__restrict__ mom, DevParams P) {
    using L = Lat<LAT>;
    constexpr int Q = L::Q, D = L::D;
    const size_t n = (size_t)P.nx * P.ny;
    for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < n; s += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(s % P.nx), y = (int)(s / P.nx);
#pragma unroll
        for (int c = 0; c < N; ++c) {
            double r = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                double g = (double)f[pop_index(c, i, Q, y, x, P.nx, P.ny)];
                r += g;
                jx += L::vx(i) * g;
                jy += L::vy(i) * g;
            }
            rho[c * n + s] = P.rho_ref[c] + r;
            if (mom) {
                mom[(c * D + 0) * n + s] = jx;
                if (D == 2) mom[(c * D + 1) * n + s] = jy;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// diagnostics: per-CTA partials of [mass_0..mass_{N-1}, F, jx, jy] in FP64
// (fixed per-thread order, fixed shuffle tree), then one CTA sums the partials
// in index order.  Also flags rho <= 0, eta <= 0 and non-finite values.
// ---------------------------------------------------------------------------
constexpr int DIAG_THREADS = 256;

template <int V>
__device__ __forceinline__ void block_sum(double (&v)[V], double *out) {
    __shared__ double s_part[DIAG_THREADS / 32][V];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < V; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < V; ++k) s_part[wid][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < V; ++k) {
            double acc = 0.0;
            for (int w = 0; w < DIAG_THREADS / 32; ++w) acc += s_part[w][k];
            out[k] = acc;
        }
    }
}

template <int LAT, int N>
__global__ void __launch_bounds__(DIAG_THREADS)
    lb_diag_partial_kernel(const double *__restrict__ rho, const double *__restrict__ mom,
                           double *__restrict__ partial, DevParams P) {
    using L = Lat<LAT>;
    constexpr int D = L::D;
    constexpr int V = N + 3;
    const size_t n = (size_t)P.nx * P.ny;
    double acc[V];
#pragma unroll
    for (int k = 0; k < V; ++k) acc[k] = 0.0;
    for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < n; s += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(s % P.nx), y = (int)(s / P.nx);
        double r[N], lp[N], eta = 1.0;
        bool ok = true;
#pragma unroll
        for (int c = 0; c < N; ++c) {
            const double *rc = rho + c * n;
            r[c] = rc[s];
            double e = rc[(size_t)y * P.nx + wrap(x + 1, P.nx)], wv = rc[(size_t)y * P.nx + wrap(x - 1, P.nx)];
            if constexpr (LAT == 1) {
                lp[c] = (e + wv) - 2.0 * r[c];
            } else {
                int yn = wrap(y + 1, P.ny), ys = wrap(y - 1, P.ny);
                int xe = wrap(x + 1, P.nx), xw = wrap(x - 1, P.nx);
                double nn = rc[(size_t)yn * P.nx + x], ss = rc[(size_t)ys * P.nx + x];
                double ne = rc[(size_t)yn * P.nx + xe], nw = rc[(size_t)yn * P.nx + xw];
                double se = rc[(size_t)ys * P.nx + xe], sw = rc[(size_t)ys * P.nx + xw];
                lp[c] = ((e + wv) + (nn + ss)) * (2.0 / 3.0) + ((ne + nw) + (se + sw)) * (1.0 / 6.0) -
                        r[c] * (10.0 / 3.0);
            }
            eta -= P.b[c] * r[c];
            ok = ok && (r[c] > 0.0) && isfinite(r[c]);
        }
        ok = ok && eta > 0.0;
        if (!ok) atomicOr(P.err, ERR_DOMAIN);
        double F = 0.0;
#pragma unroll
        for (int c = 0; c < N; ++c) {
            acc[c] += r[c];
            F += P.kT * r[c] * log(r[c] / eta);
#pragma unroll
            for (int cc = 0; cc < N; ++cc) F -= P.a[c * 4 + cc] * r[c] * r[cc] + 0.5 * P.kappa[c * 4 + cc] * r[c] * lp[cc];
            acc[N + 1] += mom[(c * D + 0) * n + s];
            if (D == 2) acc[N + 2] += mom[(c * D + 1) * n + s];
        }
        acc[N] += F;
    }
    block_sum<V>(acc, partial + (size_t)blockIdx.x * V);
}

template <int V>
__global__ void __launch_bounds__(DIAG_THREADS)
    lb_diag_final_kernel(const double *__restrict__ partial, int nparts, double *__restrict__ out) {
    double acc[V];
#pragma unroll
    for (int k = 0; k < V; ++k) acc[k] = 0.0;
    for (int p = threadIdx.x; p < nparts; p += DIAG_THREADS)
#pragma unroll
        for (int k = 0; k < V; ++k) acc[k] += partial[(size_t)p * V + k];
    block_sum<V>(acc, out);
}

}  // namespace lbvdw
