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
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "lb_mu.cuh"

namespace lbvdw {

constexpr unsigned ERR_DOMAIN = 1u;   // rho^c <= 0, eta <= 0 or non-finite value
constexpr unsigned ERR_TIMEOUT = 2u;  // a bounded wait for bulk copies ran out (lb_strip.cuh)

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
    float b_hi[4], b_lo[4];  // double-float copies of b, gamma kT and gamma
    float gkT_hi, gkT_lo, gamma_hi, gamma_lo;
    // FP32 copies for the FP32 paths (no double->float conversion in the kernels)
    float a2_f[16], kappa_f[16], lam_f[16];  // 2 a, kappa, lambda
    float rho_ref_f[4], omega_f, psi_g_f, psi_l_f;
};

// a parameter in the compute type R: the double value or its precomputed float copy
template <class R>
__device__ __forceinline__ R pv(double d, float f);
template <>
__device__ __forceinline__ double pv<double>(double d, float) { return d; }
template <>
__device__ __forceinline__ float pv<float>(double, float f) { return f; }

// 1/x in the compute type: exact division in FP64, MUFU reciprocal in FP32
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }

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

// Stencils on a shared-memory array with row length EXW.
// D1Q3: central difference (phi+ - phi-)/2 and Lap = phi+ + phi- - 2 phi (Sec. V).
// D2Q9: D = (1/theta) sum w_i v_i phi_i, Lap = (2/theta) sum w_i (phi_i - phi_0).
template <int LAT, class T>
__device__ __forceinline__ void grad_at(const T *s, int ex, int ey, int EXW, T &gx, T &gy) {
    const T *p = s + ey * EXW + ex;
    if constexpr (LAT == 1) {
        gx = (T)0.5 * (p[1] - p[-1]);
        gy = (T)0;
    } else {
        T e = p[1], wv = p[-1], n = p[EXW], sv = p[-EXW];
        T ne = p[EXW + 1], nw = p[EXW - 1], sw = p[-EXW - 1], se = p[-EXW + 1];
        gx = (e - wv) * (T)(1.0 / 3.0) + ((ne + se) - (nw + sw)) * (T)(1.0 / 12.0);
        gy = (n - sv) * (T)(1.0 / 3.0) + ((ne + nw) - (se + sw)) * (T)(1.0 / 12.0);
    }
}

template <int LAT, class T>
__device__ __forceinline__ T lap_at(const T *s, int ex, int ey, int EXW) {
    const T *p = s + ey * EXW + ex;
    if constexpr (LAT == 1) {
        return (p[1] + p[-1]) - (T)2 * p[0];
    } else {
        T axis = (p[1] + p[-1]) + (p[EXW] + p[-EXW]);
        T diag = (p[EXW + 1] + p[EXW - 1]) + (p[-EXW + 1] + p[-EXW - 1]);
        return axis * (T)(2.0 / 3.0) + diag * (T)(1.0 / 6.0) - p[0] * (T)(10.0 / 3.0);
    }
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
__device__ __forceinline__ R phi_diff(float a, float b) { return (R)(a - b); }
template <class R>
__device__ __forceinline__ R phi_diff(df a, df b) {
    return (R)__fadd_rn(__fsub_rn(a.hi, b.hi), __fsub_rn(a.lo, b.lo));
}

// D phi at (mx, my) of an MX-wide shared array, differences in the mu arithmetic
template <int LAT, class R, class T>
__device__ __forceinline__ void grad_phi(const T *s, int mx, int my, int MXW, R &gx, R &gy) {
    const T *p = s + my * MXW + mx;
    if constexpr (LAT == 1) {
        gx = (R)0.5 * phi_diff<R>(p[1], p[-1]);
        gy = (R)0;
    } else {
        R ew = phi_diff<R>(p[1], p[-1]);
        R ns = phi_diff<R>(p[MXW], p[-MXW]);
        R d1 = phi_diff<R>(p[MXW + 1], p[-MXW - 1]);  // NE - SW
        R d2 = phi_diff<R>(p[-MXW + 1], p[MXW - 1]);  // SE - NW
        gx = ew * (R)(1.0 / 3.0) + (d1 + d2) * (R)(1.0 / 12.0);
        gy = ns * (R)(1.0 / 3.0) + (d1 - d2) * (R)(1.0 / 12.0);
    }
}

// shared-memory log tables of the MU variant (TBL_WORDS floats)
template <int MU>
struct TblWords {
    static constexpr int value = MU == MU_TBL ? 3 * LOG_TBL * 2 : (MU == MU_DF ? 3 * LOG_TBL : 1);
};

template <int MU>
__device__ __forceinline__ void load_tables(float *s_tbl, const DevParams &P, int tid, int nt) {
    if constexpr (MU == MU_TBL) {
        double *t = reinterpret_cast<double *>(s_tbl);
        for (int k = tid; k < LOG_TBL; k += nt) {
            t[k] = P.tbl->r64[k];
            t[LOG_TBL + k] = P.tbl->t64_hi[k];
            t[2 * LOG_TBL + k] = P.tbl->t64_lo[k];
        }
    } else if constexpr (MU == MU_DF) {
        for (int k = tid; k < LOG_TBL; k += nt) {
            s_tbl[k] = P.tbl->r32[k];
            s_tbl[LOG_TBL + k] = P.tbl->t32_hi[k];
            s_tbl[2 * LOG_TBL + k] = P.tbl->t32_lo[k];
        }
    }
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
            if constexpr (FORCE == 1) ph -= (1.0 / 3.0) * log(r[c]);
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
            if constexpr (FORCE == 1)
                ph -= (1.0 / 3.0) * (ok ? log64_tbl((double)r[c], t, t + LOG_TBL, t + 2 * LOG_TBL, P.tbl->ln2_hi_d,
                                                     P.tbl->ln2_lo_d)
                                        : 0.0);
            phi[c] = ph;
        }
    } else if constexpr (MU == MU_F32) {
        float eta = 1.0f, rt = 0.0f;
#pragma unroll
        for (int c = 0; c < N; ++c) {
            eta = __fmaf_rn(-P.b_hi[c], (float)r[c], eta);
            rt += (float)r[c];
        }
        ok = ok && eta > 0.0f;
        const float ieta = 1.0f / eta;
#pragma unroll
        for (int c = 0; c < N; ++c) {
            const float m = logf((float)r[c] * ieta) + P.b_hi[c] * rt * ieta;
            float ph = P.gkT_hi * m - P.gamma_hi * (float)lin[c];
            if constexpr (FORCE == 1) ph -= (1.0f / 3.0f) * logf((float)r[c]);
            phi[c] = ph;
        }
    } else {  // MU_DF
        df eta = {1.0f, 0.0f};
#pragma unroll
        for (int c = 0; c < N; ++c) eta = df_add(eta, df_neg(df_mul_f({P.b_hi[c], P.b_lo[c]}, r[c])));
        // total density: the sum of the first two FP32 densities is exact as a pair
        df rt = N == 1 ? df{r[0], 0.0f} : df_two_sum(r[0], r[N > 1 ? 1 : 0]);
#pragma unroll
        for (int c = 2; c < N; ++c) rt = df_add(rt, {r[c], 0.0f});
        ok = ok && eta.hi > 0.0f;
        const df ieta = df_recip(eta);
        const df rte = df_mul(rt, ieta);
#pragma unroll
        for (int c = 0; c < N; ++c) {
            df lg = ok ? df_log(df_mul_f(ieta, r[c]), s_tbl, s_tbl + LOG_TBL, s_tbl + 2 * LOG_TBL, P.tbl->ln2_hi_f,
                                P.tbl->ln2_lo_f)
                       : df{0.0f, 0.0f};
            df m = df_add(lg, df_mul(rte, {P.b_hi[c], P.b_lo[c]}));
            df ph = df_add(df_mul(m, {P.gkT_hi, P.gkT_lo}), df_neg(df_mul_f({P.gamma_hi, P.gamma_lo}, lin[c])));
            if constexpr (FORCE == 1) {
                df lr = ok ? df_log({r[c], 0.0f}, s_tbl, s_tbl + LOG_TBL, s_tbl + 2 * LOG_TBL, P.tbl->ln2_hi_f,
                                    P.tbl->ln2_lo_f)
                           : df{0.0f, 0.0f};
                ph = df_add(ph, df_neg(df_mul_f(lr, 1.0f / 3.0f)));
            }
            phi[c] = ph;
        }
    }
    return ok;
}

// One node of phase 3: from rho, Lap rho, D phi, D rho (log force) and the bare momenta,
// the total gain G (mean field + implicit friction), then Psi, the forcing populations
// and the BGK collision.  g holds the node's stored populations (deviations); post
// receives the post-collision deviations in the same order.
template <int LAT, int N, class R, int FORCE>
__device__ __forceinline__ void collide_node(const R (&rho)[N], const R (&lap)[N], const R (&gpx)[N],
                                             const R (&gpy)[N], const R (&grx)[N], const R (&gry)[N],
                                             const R (&jx)[N], const R (&jy)[N], const DevParams &P,
                                             const R (&g)[N][Lat<LAT>::Q], R (&post)[N][Lat<LAT>::Q]) {
    using L = Lat<LAT>;
    constexpr int Q = L::Q;
    R ux[N], uy[N], Gx[N], Gy[N];
#pragma unroll
    for (int c = 0; c < N; ++c) {
        if constexpr (FORCE == 0) {
            Gx[c] = -rho[c] * gpx[c] + (R)(1.0 / 3.0) * grx[c];
            Gy[c] = -rho[c] * gpy[c] + (R)(1.0 / 3.0) * gry[c];
        } else {
            Gx[c] = -rho[c] * gpx[c];
            Gy[c] = -rho[c] * gpy[c];
        }
        const R ir = rcp(rho[c]);
        ux[c] = jx[c] * ir;
        uy[c] = jy[c] * ir;
    }

    // friction with the implicit u-hat: (D + L/2) h = -L u0, G^f = D h  (per direction).
    // Two components: L is rank one and the friction conserves momentum (rho^1 h^1 =
    // -rho^2 h^2), which leaves one unknown: G^{f,1} = -lambda m (u0^1 - u0^2) / (1 + lambda/2)
    // = -G^{f,2}, m = rho^1 rho^2 / (rho^1 + rho^2) -- the system's exact solution.
    if constexpr (N == 2) {
        const R lam = pv<R>(P.lam[1], P.lam_f[1]);
        const R k = lam * rho[0] * rho[1] * rcp(rho[0] + rho[1]) * rcp((R)1 + (R)0.5 * lam);
        const R h0 = (R)0.5 * rcp(rho[0]), h1 = (R)0.5 * rcp(rho[1]);
        const R fx = -k * ((ux[0] + Gx[0] * h0) - (ux[1] + Gx[1] * h1));
        Gx[0] += fx;
        Gx[1] -= fx;
        if constexpr (L::D == 2) {
            const R fy = -k * ((uy[0] + Gy[0] * h0) - (uy[1] + Gy[1] * h1));
            Gy[0] += fy;
            Gy[1] -= fy;
        }
    } else if constexpr (N > 2) {
        R W[N][N];
#pragma unroll
        for (int c = 0; c < N; ++c)
#pragma unroll
            for (int cc = 0; cc < N; ++cc)
                W[c][cc] = (c == cc) ? (R)0
                                     : pv<R>(P.lam[c * 4 + cc], P.lam_f[c * 4 + cc]) * rho[c] * rho[cc] *
                                           rcp(rho[c] + rho[cc]);
#pragma unroll
        for (int d = 0; d < L::D; ++d) {
            R u0[N], M[N][N], h[N];
#pragma unroll
            for (int c = 0; c < N; ++c) {
                R uu = d == 0 ? ux[c] : uy[c];
                R gg = d == 0 ? Gx[c] : Gy[c];
                u0[c] = uu + (R)0.5 * gg * rcp(rho[c]);
            }
#pragma unroll
            for (int c = 0; c < N; ++c) {
                R diag = rho[c], rhs = (R)0;
#pragma unroll
                for (int cc = 0; cc < N; ++cc) {
                    M[c][cc] = (R)(-0.5) * W[c][cc];
                    diag += (R)0.5 * W[c][cc];
                    rhs -= W[c][cc] * (u0[c] - u0[cc]);
                }
                M[c][c] = diag;
                h[c] = rhs;
            }
            // symmetric positive definite: elimination without pivoting
#pragma unroll
            for (int k = 0; k < N; ++k) {
                R inv = rcp(M[k][k]);
#pragma unroll
                for (int r2 = k + 1; r2 < N; ++r2) {
                    R m = M[r2][k] * inv;
#pragma unroll
                    for (int c2 = k + 1; c2 < N; ++c2) M[r2][c2] -= m * M[k][c2];
                    h[r2] -= m * h[k];
                }
            }
#pragma unroll
            for (int k = N - 1; k >= 0; --k) {
                R sacc = h[k];
#pragma unroll
                for (int c2 = k + 1; c2 < N; ++c2) sacc -= M[k][c2] * h[c2];
                h[k] = sacc * rcp(M[k][k]);
            }
#pragma unroll
            for (int c = 0; c < N; ++c) {
                if (d == 0) Gx[c] += rho[c] * h[c];
                else Gy[c] += rho[c] * h[c];
            }
        }
    }

    const R omega = pv<R>(P.omega, P.omega_f), cg = pv<R>(P.psi_g, P.psi_g_f), cl = pv<R>(P.psi_l, P.psi_l_f);
#pragma unroll
    for (int c = 0; c < N; ++c) {
        const R r = rho[c], u = ux[c], v = uy[c], gx = Gx[c], gy = Gy[c];
        const R ir = rcp(r);
        // second forcing moment S = G u + u G - Psi, -Psi = cg G G / rho + cl Lap rho I
        const R Sxx = (R)2 * gx * u + cg * gx * gx * ir + cl * lap[c];
        const R Syy = (R)2 * gy * v + cg * gy * gy * ir + cl * lap[c];
        const R Sxy = gx * v + u * gy + cg * gx * gy * ir;
        const R usq = u * u + v * v;
        const R drho = r - pv<R>(P.rho_ref[c], P.rho_ref_f[c]);
        // Directions come in opposite pairs (i, i'): v.u, v.G flip sign, S:(vv - theta I)
        // does not.  With A = w (drho + rho (4.5 (v.u)^2 - 1.5 u^2)), B = 3 w rho v.u,
        // C = 4.5 w S:(vv - theta I), D = 3 w v.G:  f^eq - w rho_ref = A +- B, F = C +- D.
        // The moving populations are computed first; the rest population takes what is
        // left of the node's pre-collision mass (sum f^eq = rho, sum F = 0 make this the
        // same value in exact arithmetic), so mass is conserved up to the rounding of
        // two sums instead of drifting by (sum of the rounded weights - 1) every step.
        const R third = (R)(1.0 / 3.0);
        R moved = (R)0;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int cx = L::vx(i), cy = L::vy(i);
            // handle each pair once, from its member with the smaller index
            int ip = 0;
#pragma unroll
            for (int k = 1; k < Q; ++k)
                if (L::vx(k) == -cx && L::vy(k) == -cy) ip = k;
            if (ip < i) continue;
            const R wi = (R)L::w(i);
            const R vu = (R)cx * u + (R)cy * v;
            const R vG = (R)cx * gx + (R)cy * gy;
            R SQ = Sxx * ((R)(cx * cx) - third);
            if constexpr (LAT == 2) SQ += Syy * ((R)(cy * cy) - third) + (R)2 * Sxy * (R)(cx * cy);
            const R A = wi * (drho + r * ((R)4.5 * vu * vu - (R)1.5 * usq));
            const R B = (R)3 * wi * r * vu;
            const R C = (R)4.5 * wi * SQ;
            const R D = (R)3 * wi * vG;
            post[c][i] = g[c][i] + omega * (A + B - g[c][i]) + (C + D);
            post[c][ip] = g[c][ip] + omega * (A - B - g[c][ip]) + (C - D);
            moved += post[c][i] + post[c][ip];
        }
        R before = (R)0;
#pragma unroll
        for (int i = 0; i < Q; ++i) before += g[c][i];
        post[c][0] = before - moved;
    }
}

// The fused step on one TX x TY tile with origin (x0, y0) of the lattice described by P.
template <int LAT, int N, int TX, int TY, class S, class R, int FORCE, int MU>
__device__ __forceinline__ void step_tile(const S *__restrict__ fin, S *__restrict__ fout, const DevParams &P,
                                          int x0, int y0) {
    using L = Lat<LAT>;
    using MT = typename MuStore<MU>::T;
    constexpr int Q = L::Q;
    constexpr int HY = L::HY;
    constexpr int EX = TX + 4, EY = TY + 4 * HY;  // densities: tile + 2 ring
    constexpr int MX = TX + 2, MY = TY + 2 * HY;  // mu: tile + 1 ring
    constexpr int NT = TX * TY;
    constexpr int RING = EX * EY - TX * TY;
    // Between phase 1 and phase 3 the node's own populations wait in shared memory (FP32
    // storage, up to two components, 256-thread tiles: this frees 18 registers for the mu
    // phase and measured 3 % faster than holding them in registers), else in registers when
    // they fit comfortably, else they are loaded again in phase 3.
    constexpr bool STAGE = sizeof(S) == 4 && N <= 2 && NT <= 256;
    constexpr bool KEEP = !STAGE && sizeof(S) * N * Q <= 144;
    __shared__ S s_g[STAGE ? N * Q : 1][STAGE ? NT : 1];
    static_assert(MU == MU_F64 ? sizeof(R) == 8 : sizeof(R) == 4, "MU and R mismatch");

    __shared__ R s_rho[N][EY * EX];
    __shared__ MT s_phi[N][MY * MX];  // gamma mu (log) or gamma mu - theta ln rho (nid)
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
            R acc = (R)0, ax = (R)0, ay = (R)0;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                S v = src[(size_t)(c * Q + i) * plane];
                if constexpr (KEEP) g[c][i] = v;
                if constexpr (STAGE) s_g[c * Q + i][tid] = v;
                R rv = (R)v;
                acc += rv;
                if (L::vx(i) == 1) ax += rv;
                if (L::vx(i) == -1) ax -= rv;
                if (L::vy(i) == 1) ay += rv;
                if (L::vy(i) == -1) ay -= rv;
            }
            s_rho[c][ey * EX + ex] = pv<R>(P.rho_ref[c], P.rho_ref_f[c]) + acc;
            jx[c] = ax;
            jy[c] = ay;
        }
    }
    // ---- phase 1b: rho^c on the 2-node ring -----------------------------------
    for (int k = tid; k < RING; k += NT) {
        int ex, ey;
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
        const int gx = small ? wrap(x0 + ex - 2, nx) : wrap1(x0 + ex - 2, nx);
        const int gy = (LAT == 1) ? 0 : (small ? wrap(y0 + ey - 2, ny) : wrap1(y0 + ey - 2, ny));
        const S *src = fin + (size_t)gy * nx + gx;
#pragma unroll
        for (int c = 0; c < N; ++c) {
            R acc = (R)0;
#pragma unroll
            for (int i = 0; i < Q; ++i) acc += (R)src[(size_t)(c * Q + i) * plane];
            s_rho[c][ey * EX + ex] = pv<R>(P.rho_ref[c], P.rho_ref_f[c]) + acc;
        }
    }
    __syncthreads();

    // ---- phase 2: phi^c on tile + 1 ring --------------------------------------
    unsigned bad = 0;
    for (int k = tid; k < MX * MY; k += NT) {
        const int mx = k % MX, my = k / MX;
        const int ex = mx + 1, ey = my + HY;
        R r[N], lin[N];
#pragma unroll
        for (int c = 0; c < N; ++c) {
            r[c] = s_rho[c][ey * EX + ex];
            lin[c] = (R)0;
        }
#pragma unroll
        for (int cc = 0; cc < N; ++cc) {
            R lp = lap_at<LAT, R>(s_rho[cc], ex, ey, EX);
#pragma unroll
            for (int c = 0; c < N; ++c)
                lin[c] += pv<R>(2.0 * P.a[c * 4 + cc], P.a2_f[c * 4 + cc]) * r[cc] +
                          pv<R>(P.kappa[c * 4 + cc], P.kappa_f[c * 4 + cc]) * lp;
        }
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
        grad_phi<LAT, R, MT>(s_phi[c], mx, my, MX, gpx[c], gpy[c]);
        if constexpr (FORCE == 0) grad_at<LAT, R>(s_rho[c], ex, ey, EX, grx[c], gry[c]);
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

// FP32 storage with up to two components: ask for five resident 256-thread CTAs per SM
// (48 registers); more resident warps hide the barrier waits between the phases.
template <class S, int N, int NT>
struct MinBlocks {
    static constexpr int value = (sizeof(S) == 4 && N <= 2 && NT == 256) ? 5 : 1;
};

template <int LAT, int N, int TX, int TY, class S, class R, int FORCE, int MU>
__global__ void __launch_bounds__(TX *TY, MinBlocks<S, N, TX * TY>::value)
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
