// lb_adjoint.cuh -- hand-written adjoint (vector-Jacobian product) of one timestep of the
// fused step (lb_kernels.cuh), "log" force.
//
// The kernels are templates over T, the type of the adjoint populations and of their
// arithmetic: double for the FP64 rollout, float for the FP32 rollouts.  In both, the
// forward recompute of the chemical potential (phi = gamma mu, its gradient) and the
// transpose of its Jacobian d mu / d rho run in FP64, and the parameter gradients are
// summed in FP64 across CTAs.  The FP32 rollouts take the moments of the stored state as
// the FP32 step forms them (rho = rho_ref + sum_i g_i in FP32, adj_moments32_kernel),
// widened to FP64 for mu, and keep everything outside mu on the FP32 pipe (rho, u and
// D rho in FP32, reciprocals from an FP32 seed refined in FP64, per-CTA partial sums in
// FP32).
//
// Forward step (per node x, component c; D = central difference, Lap = lattice
// Laplacian, theta = 1/3):
//   rho = sum_i f_i,  j = sum_i v_i f_i,  u = j / rho
//   mu^c = kT [ln rho^c - ln eta + b^c rho_t / eta] - sum_d (2 a_cd rho^d + kappa_cd Lap rho^d)
//   phi = gamma mu;   Gmu = -rho D phi + theta D rho
//   friction per direction: u0 = u + Gmu/(2 rho), M h = -L_W u0, G = Gmu + rho h,
//     M = diag(rho) + L_W/2, W_cd = lambda rho_c rho_d / (rho_c + rho_d)
//   S = G u + u G + cg G G / rho + cl Lap rho I
//   post_i = f_i + omega (feq_i(rho, u) - f_i) + F_i(G, S),   f'(x + v_i) = post_i(x)
// The adjoint takes fbar' (d loss / d f at t+1) to fbar (at t) in five node-parallel
// kernels, recomputing the forward quantities from f_t:
//   adj_mu      rho -> Lap rho, phi                          (forward recompute)
//   adj_local   gather postbar_i(x) = fbar'_i(x + v_i); the local transpose of the
//               collision, forcing, Psi and friction -> gbar, rhobar_loc, jbar,
//               Dphibar, Drhobar, Lapbar
//   adj_mubar   mubar = gamma (-div Dphibar); parameter-gradient partials
//   adj_rhobar  rhobar = rhobar_loc + (d mu/d rho)^T mubar - Lap(kappa^T mubar)
//               - div Drhobar + Lap Lapbar;  fbar_i = gbar_i + rhobar + v_i . jbar
// Transposes of the stencils: D^T = -D (antisymmetric weights), Lap^T = Lap.
#pragma once
#include "lb_kernels.cuh"

namespace lbvdw {

constexpr int ADJ_THREADS = 256;

template <class T>
struct AdjArrays {
    const double *rho, *j;       // [N][n], [N][D][n] at step t (FP64 moments of the state)
    T *lap;                      // [N][n]
    double *phi;                 // [N][n], gamma mu in FP64
    T *rhob, *jb, *dphib, *drhob, *lapb, *mub;  // adjoint intermediates
    double *partial;             // [blocks][2 N^2 + N] parameter-gradient partials
    // FP32 adjoint only: rho and u = j / rho of the state in FP32, written by adj_mu_kernel,
    // so that the parts of the local transpose outside mu stay off the FP64 pipe
    float *rho_t, *u_t;          // [N][n], [N][D][n]
};

template <class T> struct IsF32 { static constexpr bool value = false; };
template <> struct IsF32<float> { static constexpr bool value = true; };

// 1 / x in FP64 from an FP32 seed and two Newton steps (y <- y + y (1 - x y)), within an
// ulp or two of the quotient for the positive, normal x of this code (densities, eta)
__device__ __forceinline__ double recip64(double x) {
    double y = (double)__frcp_rn((float)x);
    y = fma(y, fma(-x, y, 1.0), y);
    return fma(y, fma(-x, y, 1.0), y);
}

// Block sum of V per-thread values into one FP64 partial per CTA (fixed order): in FP64
// for the FP64 adjoint, for the FP32 adjoint warp shuffles in FP32 and the warp sums in
// FP64
template <class T, int V>
__device__ __forceinline__ void block_sum_adj(T (&v)[V], double *out) {
    if constexpr (!IsF32<T>::value) {
        block_sum<V>(v, out);
    } else {
        __shared__ double s_part[ADJ_THREADS / 32][V];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < V; ++k)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < V; ++k) s_part[wid][k] = (double)v[k];
        __syncthreads();
        if (threadIdx.x == 0) {
#pragma unroll
            for (int k = 0; k < V; ++k) {
                double acc = 0.0;
                for (int w = 0; w < ADJ_THREADS / 32; ++w) acc += s_part[w][k];
                out[k] = acc;
            }
        }
    }
}

template <int LAT>
struct Nb {
    // neighbour of (x, y) along lattice vector i, periodic
    __device__ static inline size_t at(int x, int y, int i, int nx, int ny) {
        int xx = x + Lat<LAT>::vx(i), yy = y + Lat<LAT>::vy(i);
        xx = xx < 0 ? xx + nx : (xx >= nx ? xx - nx : xx);
        yy = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
        return (size_t)yy * nx + xx;
    }
};

// D_alpha phi = (1/theta) sum_i w_i v_i,alpha phi(x + v_i), in the arithmetic of the array
template <int LAT, class A>
__device__ inline void grad_g(const A *phi, int x, int y, int nx, int ny, A &gx, A &gy) {
    using L = Lat<LAT>;
    A ax = A(0), ay = A(0);
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
        A v = phi[Nb<LAT>::at(x, y, i, nx, ny)];
        ax += A(L::w(i) * L::vx(i)) * v;
        ay += A(L::w(i) * L::vy(i)) * v;
    }
    gx = A(3) * ax;
    gy = A(3) * ay;
}

template <int LAT, class A>
__device__ inline A lap_g(const A *phi, int x, int y, int nx, int ny) {
    using L = Lat<LAT>;
    const A c = phi[(size_t)y * nx + x];
    A acc = A(0);
#pragma unroll
    for (int i = 1; i < L::Q; ++i) acc += A(L::w(i)) * (phi[Nb<LAT>::at(x, y, i, nx, ny)] - c);
    return A(6) * acc;
}

// ---- forward recompute: Lap rho and phi = gamma mu (FP64) -----------------------------
template <int LAT, int N, class T>
__global__ void __launch_bounds__(ADJ_THREADS) adj_mu_kernel(AdjArrays<T> A, DevParams P) {
    const size_t n = (size_t)P.nx * P.ny;
    const size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int x = (int)(s % P.nx), y = (int)(s / P.nx);
    double r[N], lp[N], eta = 1.0, rt = 0.0;
#pragma unroll
    for (int c = 0; c < N; ++c) {
        r[c] = A.rho[c * n + s];
        lp[c] = lap_g<LAT>(A.rho + c * n, x, y, P.nx, P.ny);
        A.lap[c * n + s] = T(lp[c]);
        eta -= P.b[c] * r[c];
        rt += r[c];
    }
    // FP64 throughout; the FP32 adjoint takes the table-driven FP64 logarithm of the
    // forward's FP64-mu path (lb_mu.cuh) and an FP32-seeded reciprocal refined in FP64
    const double ieta = IsF32<T>::value ? recip64(eta) : 1.0 / eta;
#pragma unroll
    for (int c = 0; c < N; ++c) {
        const double lg = IsF32<T>::value ? log64_tbl(r[c] * ieta, P.tbl->r64, P.tbl->t64_hi, P.tbl->t64_lo,
                                                      P.tbl->ln2_hi_d, P.tbl->ln2_lo_d)
                                          : log(r[c] * ieta);
        double m = P.kT * (lg + P.b[c] * rt * ieta);
#pragma unroll
        for (int d = 0; d < N; ++d) m -= 2.0 * P.a[c * 4 + d] * r[d] + P.kappa[c * 4 + d] * lp[d];
        A.phi[c * n + s] = P.gamma * m;
    }
}

// Moments of an FP32-storage state for the FP32 adjoint: rho^c = rho_ref^c + sum_i g_i and
// the bare momenta summed in FP32 in direction order, as the forward step kernel forms them,
// then u = j / rho in FP32; rho and j also in FP64 for the FP64 chemical potential.
template <int LAT, int N>
__global__ void __launch_bounds__(ADJ_THREADS) adj_moments32_kernel(const float *__restrict__ g, AdjArrays<float> A,
                                                                    DevParams P) {
    using L = Lat<LAT>;
    constexpr int Q = L::Q, D = L::D;
    const size_t n = (size_t)P.nx * P.ny;
    const size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    double *rho = const_cast<double *>(A.rho), *j = const_cast<double *>(A.j);
#pragma unroll
    for (int c = 0; c < N; ++c) {
        float v[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) v[i] = g[(size_t)(c * Q + i) * n + s];
        float acc = v[0], jx = 0.0f, jy = 0.0f;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            acc += v[i];
            if (L::vx(i) != 0) jx += L::vx(i) == 1 ? v[i] : -v[i];
            if (L::vy(i) != 0) jy += L::vy(i) == 1 ? v[i] : -v[i];
        }
        const float r = P.rho_ref_f[c] + acc;
        A.rho_t[c * n + s] = r;
        rho[c * n + s] = (double)r;
        A.u_t[(c * D) * n + s] = jx / r;
        j[(c * D) * n + s] = (double)jx;
        if (D == 2) {
            A.u_t[(c * D + 1) * n + s] = jy / r;
            j[(c * D + 1) * n + s] = (double)jy;
        }
    }
}

// ---- local transpose of collision, forcing, Psi, friction, force -------------------------
template <int LAT, int N, class T>
__global__ void __launch_bounds__(ADJ_THREADS)
    adj_local_kernel(const T *__restrict__ fbar_next, T *__restrict__ fbar, AdjArrays<T> A, DevParams P) {
    using L = Lat<LAT>;
    constexpr int Q = L::Q, D = L::D;
    const int nx = P.nx, ny = P.ny;
    const size_t n = (size_t)nx * ny;
    const size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int x = (int)(s % nx), y = (int)(s / nx);
    const T th = T(1.0 / 3.0), omega = T(P.omega), cg = T(P.psi_g), cl = T(P.psi_l);

    // ---------- forward recompute at this node (D phi from the FP64 phi, then rounded to T)
    T rho[N], u[N][2], gmu[N][2], G[N][2], dphi[N][2], drho[N][2], h[2][N], u0[2][N];
    T W[N][N], M[N][N];
#pragma unroll
    for (int c = 0; c < N; ++c) {
        double px, py;
        grad_g<LAT>(A.phi + c * n, x, y, nx, ny, px, py);  // D phi in FP64 (FP64 mu)
        dphi[c][0] = T(px), dphi[c][1] = T(py);
        if constexpr (IsF32<T>::value) {
            rho[c] = A.rho_t[c * n + s];
            grad_g<LAT>(A.rho_t + c * n, x, y, nx, ny, drho[c][0], drho[c][1]);
            for (int a = 0; a < 2; ++a) u[c][a] = (a < D) ? A.u_t[(c * D + a) * n + s] : T(0);
        } else {
            rho[c] = T(A.rho[c * n + s]);
            double qx, qy;
            grad_g<LAT>(A.rho + c * n, x, y, nx, ny, qx, qy);
            drho[c][0] = T(qx), drho[c][1] = T(qy);
            for (int a = 0; a < 2; ++a) u[c][a] = (a < D) ? T(A.j[(c * D + a) * n + s] / A.rho[c * n + s]) : T(0);
        }
        for (int a = 0; a < 2; ++a) {
            gmu[c][a] = (a < D) ? -rho[c] * dphi[c][a] + th * drho[c][a] : T(0);
            G[c][a] = gmu[c][a];
        }
    }
#pragma unroll
    for (int c = 0; c < N; ++c)
#pragma unroll
        for (int d = 0; d < N; ++d)
            W[c][d] = (c == d) ? T(0) : T(P.lam[c * 4 + d]) * rho[c] * rho[d] / (rho[c] + rho[d]);
#pragma unroll
    for (int c = 0; c < N; ++c) {
        T diag = rho[c];
#pragma unroll
        for (int d = 0; d < N; ++d) {
            M[c][d] = T(-0.5) * W[c][d];
            diag += T(0.5) * W[c][d];
        }
        M[c][c] = diag;
    }
    // M^{-1} by Gauss-Jordan (symmetric positive definite, N <= 4)
    T Mi[N][N];
    {
        T Tm[N][2 * N];
#pragma unroll
        for (int c = 0; c < N; ++c)
#pragma unroll
            for (int d = 0; d < 2 * N; ++d) Tm[c][d] = d < N ? M[c][d] : (d - N == c ? T(1) : T(0));
#pragma unroll
        for (int k = 0; k < N; ++k) {
            T inv = T(1) / Tm[k][k];
#pragma unroll
            for (int d = 0; d < 2 * N; ++d) Tm[k][d] *= inv;
#pragma unroll
            for (int r2 = 0; r2 < N; ++r2) {
                if (r2 == k) continue;
                T m = Tm[r2][k];
#pragma unroll
                for (int d = 0; d < 2 * N; ++d) Tm[r2][d] -= m * Tm[k][d];
            }
        }
#pragma unroll
        for (int c = 0; c < N; ++c)
#pragma unroll
            for (int d = 0; d < N; ++d) Mi[c][d] = Tm[c][N + d];
    }
    if constexpr (N > 1) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
            T rhs[N];
#pragma unroll
            for (int c = 0; c < N; ++c) u0[a][c] = u[c][a] + gmu[c][a] / (T(2) * rho[c]);
#pragma unroll
            for (int c = 0; c < N; ++c) {
                rhs[c] = T(0);
#pragma unroll
                for (int d = 0; d < N; ++d) rhs[c] -= W[c][d] * (u0[a][c] - u0[a][d]);
            }
#pragma unroll
            for (int c = 0; c < N; ++c) {
                T acc = T(0);
#pragma unroll
                for (int d = 0; d < N; ++d) acc += Mi[c][d] * rhs[d];
                h[a][c] = acc;
                G[c][a] += rho[c] * acc;
            }
        }
    }

    // ---------- backward
    T rhob[N], ub[N][2], Gb[N][2];
#pragma unroll
    for (int c = 0; c < N; ++c) {
        rhob[c] = T(0);
        ub[c][0] = ub[c][1] = T(0);
        Gb[c][0] = Gb[c][1] = T(0);
        const T r = rho[c], ux = u[c][0], uy = u[c][1], gx = G[c][0], gy = G[c][1];
        const T usq = ux * ux + uy * uy;
        T Sxxb = T(0), Syyb = T(0), Sxyb = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const T cx = T(L::vx(i)), cy = T(L::vy(i)), wi = T(L::w(i));
            // streaming: post_i(x) went to x + v_i
            const T pb = fbar_next[(size_t)(c * Q + i) * n + Nb<LAT>::at(x, y, i, nx, ny)];
            fbar[(size_t)(c * Q + i) * n + s] = (T(1) - omega) * pb;   // d post / d f_i (direct)
            const T eb = omega * pb;                                      // feq bar
            const T vu = cx * ux + cy * uy;
            rhob[c] += eb * wi * (T(1) + T(3) * vu + T(4.5) * vu * vu - T(1.5) * usq);
            ub[c][0] += eb * wi * r * (T(3) * cx + T(9) * vu * cx - T(3) * ux);
            ub[c][1] += eb * wi * r * (T(3) * cy + T(9) * vu * cy - T(3) * uy);
            // F_i = w_i (3 v.G + 4.5 S:(vv - theta I))
            Gb[c][0] += pb * wi * T(3) * cx;
            Gb[c][1] += pb * wi * T(3) * cy;
            Sxxb += pb * wi * T(4.5) * (cx * cx - th);
            if (LAT == 2) {
                Syyb += pb * wi * T(4.5) * (cy * cy - th);
                Sxyb += pb * wi * T(9) * cx * cy;
            }
        }
        // S_xx = 2 G_x u_x + cg G_x^2/rho + cl Lap;  S_yy likewise;  S_xy = G_x u_y + u_x G_y + cg G_x G_y/rho
        const T ir = T(1) / r;
        Gb[c][0] += Sxxb * (T(2) * ux + T(2) * cg * gx * ir) + Sxyb * (uy + cg * gy * ir);
        Gb[c][1] += Syyb * (T(2) * uy + T(2) * cg * gy * ir) + Sxyb * (ux + cg * gx * ir);
        ub[c][0] += Sxxb * T(2) * gx + Sxyb * gy;
        ub[c][1] += Syyb * T(2) * gy + Sxyb * gx;
        rhob[c] += -(Sxxb * cg * gx * gx + Syyb * cg * gy * gy + Sxyb * cg * gx * gy) * ir * ir;
        A.lapb[c * n + s] = (Sxxb + Syyb) * cl;
    }
    // friction: G = Gmu + rho h,  M h = rhs,  rhs = -L_W u0,  u0 = u + Gmu/(2 rho)
    T gmub[N][2], Mb[N][N], Wb[N][N];
#pragma unroll
    for (int c = 0; c < N; ++c) {
        gmub[c][0] = Gb[c][0];
        gmub[c][1] = Gb[c][1];
#pragma unroll
        for (int d = 0; d < N; ++d) Mb[c][d] = Wb[c][d] = T(0);
    }
    if constexpr (N > 1) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
            T hb[N], rb[N];
#pragma unroll
            for (int c = 0; c < N; ++c) {
                rhob[c] += h[a][c] * Gb[c][a];
                hb[c] = rho[c] * Gb[c][a];
            }
#pragma unroll
            for (int c = 0; c < N; ++c) {
                T acc = T(0);
#pragma unroll
                for (int d = 0; d < N; ++d) acc += Mi[c][d] * hb[d];  // M symmetric
                rb[c] = acc;
            }
#pragma unroll
            for (int c = 0; c < N; ++c)
#pragma unroll
                for (int d = 0; d < N; ++d) Mb[c][d] -= rb[c] * h[a][d];
#pragma unroll
            for (int c = 0; c < N; ++c) {
                T u0b = T(0);
#pragma unroll
                for (int d = 0; d < N; ++d) {
                    u0b += W[c][d] * (rb[d] - rb[c]);
                    Wb[c][d] += -rb[c] * (u0[a][c] - u0[a][d]);
                }
                ub[c][a] += u0b;
                gmub[c][a] += u0b / (T(2) * rho[c]);
                rhob[c] += -u0b * gmu[c][a] / (T(2) * rho[c] * rho[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < N; ++c) {
            rhob[c] += Mb[c][c];
#pragma unroll
            for (int d = 0; d < N; ++d) {
                if (d == c) continue;
                Wb[c][d] += T(0.5) * Mb[c][c] - T(0.5) * Mb[c][d];
            }
        }
#pragma unroll
        for (int c = 0; c < N; ++c)
#pragma unroll
            for (int d = 0; d < N; ++d) {
                if (d == c) continue;
                const T sum = rho[c] + rho[d];
                const T k = T(P.lam[c * 4 + d]) / (sum * sum);
                rhob[c] += Wb[c][d] * k * rho[d] * rho[d];
                rhob[d] += Wb[c][d] * k * rho[c] * rho[c];
            }
    }
    // u = j / rho;  Gmu = -rho D phi + theta D rho
#pragma unroll
    for (int c = 0; c < N; ++c) {
        const T ir = T(1) / rho[c];
        T acc = T(0);
        for (int a = 0; a < D; ++a) {
            A.jb[(c * D + a) * n + s] = ub[c][a] * ir;
            acc += ub[c][a] * u[c][a];
            A.dphib[(c * D + a) * n + s] = -rho[c] * gmub[c][a];
            A.drhob[(c * D + a) * n + s] = th * gmub[c][a];
            rhob[c] += -gmub[c][a] * dphi[c][a];
        }
        rhob[c] -= acc * ir;
        A.rhob[c * n + s] = rhob[c];
    }
}

// ---- mubar = gamma (-div Dphibar); parameter-gradient partials ---------------------------
template <int LAT, int N, class T>
__global__ void __launch_bounds__(ADJ_THREADS) adj_mubar_kernel(AdjArrays<T> A, DevParams P) {
    using L = Lat<LAT>;
    constexpr int D = L::D;
    constexpr int V = 2 * N * N + N;
    const int nx = P.nx, ny = P.ny;
    const size_t n = (size_t)nx * ny;
    const size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    double acc[IsF32<T>::value ? 1 : V];
    float acc32[IsF32<T>::value ? V : 1];
#pragma unroll
    for (int k = 0; k < (IsF32<T>::value ? 1 : V); ++k) acc[k] = 0.0;
#pragma unroll
    for (int k = 0; k < (IsF32<T>::value ? V : 1); ++k) acc32[k] = 0.0f;
    if (s < n) {
        const int x = (int)(s % nx), y = (int)(s / nx);
        double mb[N], r[N], eta = 1.0, rt = 0.0;
#pragma unroll
        for (int c = 0; c < N; ++c) {
            // div^T: phibar(x) = -sum_a D_a(Dphibar_a)(x)
            T dv = T(0);
            T gx, gy;
            grad_g<LAT>(A.dphib + (c * D + 0) * n, x, y, nx, ny, gx, gy);
            dv += gx;
            if (D == 2) {
                grad_g<LAT>(A.dphib + (c * D + 1) * n, x, y, nx, ny, gx, gy);
                dv += gy;
            }
            const T mbt = T(-P.gamma) * dv;
            A.mub[c * n + s] = mbt;
            mb[c] = (double)mbt;
            r[c] = A.rho[c * n + s];
            eta -= P.b[c] * r[c];
            rt += r[c];
        }
        // d mu^c / d a_cd = -2 rho^d;  d mu^c / d kappa_cd = -Lap rho^d;
        // d mu^c / d b^d = kT [rho^d/eta + delta_cd rho_t/eta + b^c rho_t rho^d / eta^2]
        if constexpr (!IsF32<T>::value) {
#pragma unroll
            for (int c = 0; c < N; ++c)
#pragma unroll
                for (int d = 0; d < N; ++d) {
                    acc[c * N + d] = mb[c] * (-2.0 * r[d]);
                    acc[N * N + c * N + d] = mb[c] * (-(double)A.lap[d * n + s]);
                    acc[2 * N * N + d] += mb[c] * P.kT *
                                          (r[d] / eta + (c == d ? rt / eta : 0.0) + P.b[c] * rt * r[d] / (eta * eta));
                }
        } else {
            // the FP32 adjoint: the a and kappa terms in FP32, the b term (the Jacobian of
            // mu's FP64 part) in FP64 with one reciprocal of eta
            const double ieta = recip64(eta);
#pragma unroll
            for (int c = 0; c < N; ++c)
#pragma unroll
                for (int d = 0; d < N; ++d) {
                    acc32[c * N + d] = (float)mb[c] * (-2.0f * A.rho_t[d * n + s]);
                    acc32[N * N + c * N + d] = (float)mb[c] * (-(float)A.lap[d * n + s]);
                    acc32[2 * N * N + d] += (float)(mb[c] * P.kT *
                                                    (r[d] * ieta + (c == d ? rt * ieta : 0.0) +
                                                     P.b[c] * rt * r[d] * ieta * ieta));
                }
        }
    }
    if constexpr (!IsF32<T>::value) block_sum_adj<double, V>(acc, A.partial + (size_t)blockIdx.x * V);
    else block_sum_adj<float, V>(acc32, A.partial + (size_t)blockIdx.x * V);
}

// ---- rhobar and fbar ---------------------------------------------------------------------
template <int LAT, int N, class T>
__global__ void __launch_bounds__(ADJ_THREADS) adj_rhobar_kernel(T *__restrict__ fbar, AdjArrays<T> A, DevParams P) {
    using L = Lat<LAT>;
    constexpr int Q = L::Q, D = L::D;
    const int nx = P.nx, ny = P.ny;
    const size_t n = (size_t)nx * ny;
    const size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int x = (int)(s % nx), y = (int)(s / nx);
    double r[N], eta = 1.0, rt = 0.0, mb[N];
#pragma unroll
    for (int c = 0; c < N; ++c) {
        r[c] = A.rho[c * n + s];
        mb[c] = (double)A.mub[c * n + s];
        eta -= P.b[c] * r[c];
        rt += r[c];
    }
    // reciprocals: FP64 quotients for the FP64 adjoint; for the FP32 adjoint an FP32 seed
    // refined in FP64 (recip64), which keeps the divisions off the FP64 pipe's slow path
    const double ieta = IsF32<T>::value ? recip64(eta) : 1.0 / eta;
#pragma unroll
    for (int d = 0; d < N; ++d) {
        // local chemical-potential Jacobian (kT part and the -2a term), in FP64
        double jt = 0.0;
#pragma unroll
        for (int c = 0; c < N; ++c) {
            const double ir = c == d ? (IsF32<T>::value ? recip64(r[c]) : 1.0 / r[c]) : 0.0;
            double J = P.kT * (ir + (P.b[c] + P.b[d]) * ieta + P.b[c] * P.b[d] * rt * ieta * ieta) -
                       2.0 * P.a[c * 4 + d];
            jt += mb[c] * J;
        }
        T rb = A.rhob[d * n + s] + T(jt);
        // -kappa Lap rho terms: rhobar^d -= Lap(sum_c kappa_cd mubar^c)
        {
            const T c0 = [&] {
                T t = T(0);
#pragma unroll
                for (int c = 0; c < N; ++c) t += T(P.kappa[c * 4 + d]) * A.mub[c * n + s];
                return t;
            }();
            T accl = T(0);
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const size_t nb = Nb<LAT>::at(x, y, i, nx, ny);
                T t = T(0);
#pragma unroll
                for (int c = 0; c < N; ++c) t += T(P.kappa[c * 4 + d]) * A.mub[c * n + nb];
                accl += T(L::w(i)) * (t - c0);
            }
            rb -= T(6) * accl;
        }
        // D rho^T and Lap^T
        T gx, gy;
        grad_g<LAT>(A.drhob + (d * D + 0) * n, x, y, nx, ny, gx, gy);
        rb -= gx;
        if (D == 2) {
            grad_g<LAT>(A.drhob + (d * D + 1) * n, x, y, nx, ny, gx, gy);
            rb -= gy;
        }
        rb += lap_g<LAT>(A.lapb + d * n, x, y, nx, ny);
        const T jbx = A.jb[(d * D + 0) * n + s];
        const T jby = D == 2 ? A.jb[(d * D + 1) * n + s] : T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i)
            fbar[(size_t)(d * Q + i) * n + s] += rb + T(L::vx(i)) * jbx + T(L::vy(i)) * jby;
    }
}

// ---- small helpers -------------------------------------------------------------------
template <int V>
__global__ void adj_accum_kernel(const double *__restrict__ step, double *__restrict__ accum) {
    if (threadIdx.x == 0)
        for (int k = 0; k < V; ++k) accum[k] += step[k];
}

// fbar_i = rhobar for every i (the loss depends on f only through rho = sum_i f_i)
template <class T>
__global__ void adj_seed_kernel(const double *__restrict__ rb, T *__restrict__ fb, int N, int Q, size_t n) {
    const size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    for (int c = 0; c < N; ++c)
        for (int i = 0; i < Q; ++i) fb[(size_t)(c * Q + i) * n + s] = T(rb[c * n + s]);
}

// f_0 = w_i rho_0 (equilibrium at rest; with FP32 storage g_0 = w_i (rho_0 - rho_ref), the
// same transpose): rhobar_0 = sum_i w_i fbar_0,i, summed in FP64
template <int LAT, class T>
__global__ void adj_init_transpose_kernel(const T *__restrict__ fb, double *__restrict__ rb, int N, size_t n) {
    using L = Lat<LAT>;
    const size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    for (int c = 0; c < N; ++c) {
        double acc = 0.0;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) acc += L::w(i) * (double)fb[(size_t)(c * L::Q + i) * n + s];
        rb[c * n + s] = acc;
    }
}

}  // namespace lbvdw
