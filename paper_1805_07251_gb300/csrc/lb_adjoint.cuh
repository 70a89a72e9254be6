// lb_adjoint.cuh -- hand-written adjoint (vector-Jacobian product) of one FP64 timestep
// of the fused step (lb_kernels.cuh), "log" force.
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

struct AdjArrays {
    const double *rho, *j;       // [N][n], [N][D][n] at step t
    double *lap, *phi;           // [N][n]
    double *rhob, *jb, *dphib, *drhob, *lapb, *mub;  // adjoint intermediates
    double *partial;             // [blocks][2 N^2 + N] parameter-gradient partials
};

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

// D_alpha phi = (1/theta) sum_i w_i v_i,alpha phi(x + v_i)
template <int LAT>
__device__ inline void grad_g(const double *phi, int x, int y, int nx, int ny, double &gx, double &gy) {
    using L = Lat<LAT>;
    double ax = 0.0, ay = 0.0;
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
        double v = phi[Nb<LAT>::at(x, y, i, nx, ny)];
        ax += L::w(i) * L::vx(i) * v;
        ay += L::w(i) * L::vy(i) * v;
    }
    gx = 3.0 * ax;
    gy = 3.0 * ay;
}

template <int LAT>
__device__ inline double lap_g(const double *phi, int x, int y, int nx, int ny) {
    using L = Lat<LAT>;
    const double c = phi[(size_t)y * nx + x];
    double acc = 0.0;
#pragma unroll
    for (int i = 1; i < L::Q; ++i) acc += L::w(i) * (phi[Nb<LAT>::at(x, y, i, nx, ny)] - c);
    return 6.0 * acc;
}

// ---- forward recompute: Lap rho and phi = gamma mu ------------------------------------
template <int LAT, int N>
__global__ void __launch_bounds__(ADJ_THREADS) adj_mu_kernel(AdjArrays A, DevParams P) {
    const size_t n = (size_t)P.nx * P.ny;
    const size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int x = (int)(s % P.nx), y = (int)(s / P.nx);
    double r[N], lp[N], eta = 1.0, rt = 0.0;
#pragma unroll
    for (int c = 0; c < N; ++c) {
        r[c] = A.rho[c * n + s];
        lp[c] = lap_g<LAT>(A.rho + c * n, x, y, P.nx, P.ny);
        A.lap[c * n + s] = lp[c];
        eta -= P.b[c] * r[c];
        rt += r[c];
    }
    const double ieta = 1.0 / eta;
#pragma unroll
    for (int c = 0; c < N; ++c) {
        double m = P.kT * (log(r[c] * ieta) + P.b[c] * rt * ieta);
#pragma unroll
        for (int d = 0; d < N; ++d) m -= 2.0 * P.a[c * 4 + d] * r[d] + P.kappa[c * 4 + d] * lp[d];
        A.phi[c * n + s] = P.gamma * m;
    }
}

// ---- local transpose of collision, forcing, Psi, friction, force -------------------------
template <int LAT, int N>
__global__ void __launch_bounds__(ADJ_THREADS)
    adj_local_kernel(const double *__restrict__ fbar_next, double *__restrict__ fbar, AdjArrays A, DevParams P) {
    using L = Lat<LAT>;
    constexpr int Q = L::Q, D = L::D;
    const int nx = P.nx, ny = P.ny;
    const size_t n = (size_t)nx * ny;
    const size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int x = (int)(s % nx), y = (int)(s / nx);
    const double th = 1.0 / 3.0, omega = P.omega, cg = P.psi_g, cl = P.psi_l;

    // ---------- forward recompute at this node
    double rho[N], u[N][2], gmu[N][2], G[N][2], dphi[N][2], drho[N][2], lap[N], h[2][N], u0[2][N];
    double W[N][N], M[N][N];
#pragma unroll
    for (int c = 0; c < N; ++c) {
        rho[c] = A.rho[c * n + s];
        lap[c] = A.lap[c * n + s];
        grad_g<LAT>(A.phi + c * n, x, y, nx, ny, dphi[c][0], dphi[c][1]);
        grad_g<LAT>(A.rho + c * n, x, y, nx, ny, drho[c][0], drho[c][1]);
        for (int a = 0; a < 2; ++a) {
            u[c][a] = (a < D) ? A.j[(c * D + a) * n + s] / rho[c] : 0.0;
            gmu[c][a] = (a < D) ? -rho[c] * dphi[c][a] + th * drho[c][a] : 0.0;
            G[c][a] = gmu[c][a];
        }
    }
#pragma unroll
    for (int c = 0; c < N; ++c)
#pragma unroll
        for (int d = 0; d < N; ++d) W[c][d] = (c == d) ? 0.0 : P.lam[c * 4 + d] * rho[c] * rho[d] / (rho[c] + rho[d]);
#pragma unroll
    for (int c = 0; c < N; ++c) {
        double diag = rho[c];
#pragma unroll
        for (int d = 0; d < N; ++d) {
            M[c][d] = -0.5 * W[c][d];
            diag += 0.5 * W[c][d];
        }
        M[c][c] = diag;
    }
    // M^{-1} by Gauss-Jordan (symmetric positive definite, N <= 4)
    double Mi[N][N];
    {
        double T[N][2 * N];
#pragma unroll
        for (int c = 0; c < N; ++c)
#pragma unroll
            for (int d = 0; d < 2 * N; ++d) T[c][d] = d < N ? M[c][d] : (d - N == c ? 1.0 : 0.0);
#pragma unroll
        for (int k = 0; k < N; ++k) {
            double inv = 1.0 / T[k][k];
#pragma unroll
            for (int d = 0; d < 2 * N; ++d) T[k][d] *= inv;
#pragma unroll
            for (int r2 = 0; r2 < N; ++r2) {
                if (r2 == k) continue;
                double m = T[r2][k];
#pragma unroll
                for (int d = 0; d < 2 * N; ++d) T[r2][d] -= m * T[k][d];
            }
        }
#pragma unroll
        for (int c = 0; c < N; ++c)
#pragma unroll
            for (int d = 0; d < N; ++d) Mi[c][d] = T[c][N + d];
    }
    if constexpr (N > 1) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
            double rhs[N];
#pragma unroll
            for (int c = 0; c < N; ++c) u0[a][c] = u[c][a] + gmu[c][a] / (2.0 * rho[c]);
#pragma unroll
            for (int c = 0; c < N; ++c) {
                rhs[c] = 0.0;
#pragma unroll
                for (int d = 0; d < N; ++d) rhs[c] -= W[c][d] * (u0[a][c] - u0[a][d]);
            }
#pragma unroll
            for (int c = 0; c < N; ++c) {
                double acc = 0.0;
#pragma unroll
                for (int d = 0; d < N; ++d) acc += Mi[c][d] * rhs[d];
                h[a][c] = acc;
                G[c][a] += rho[c] * acc;
            }
        }
    }

    // ---------- backward
    double rhob[N], ub[N][2], Gb[N][2];
#pragma unroll
    for (int c = 0; c < N; ++c) {
        rhob[c] = 0.0;
        ub[c][0] = ub[c][1] = 0.0;
        Gb[c][0] = Gb[c][1] = 0.0;
        const double r = rho[c], ux = u[c][0], uy = u[c][1], gx = G[c][0], gy = G[c][1];
        const double usq = ux * ux + uy * uy;
        double Sxxb = 0.0, Syyb = 0.0, Sxyb = 0.0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double cx = L::vx(i), cy = L::vy(i), wi = L::w(i);
            // streaming: post_i(x) went to x + v_i
            const double pb = fbar_next[(size_t)(c * Q + i) * n + Nb<LAT>::at(x, y, i, nx, ny)];
            fbar[(size_t)(c * Q + i) * n + s] = (1.0 - omega) * pb;   // d post / d f_i (direct)
            const double eb = omega * pb;                                 // feq bar
            const double vu = cx * ux + cy * uy;
            rhob[c] += eb * wi * (1.0 + 3.0 * vu + 4.5 * vu * vu - 1.5 * usq);
            ub[c][0] += eb * wi * r * (3.0 * cx + 9.0 * vu * cx - 3.0 * ux);
            ub[c][1] += eb * wi * r * (3.0 * cy + 9.0 * vu * cy - 3.0 * uy);
            // F_i = w_i (3 v.G + 4.5 S:(vv - theta I))
            Gb[c][0] += pb * wi * 3.0 * cx;
            Gb[c][1] += pb * wi * 3.0 * cy;
            Sxxb += pb * wi * 4.5 * (cx * cx - th);
            if (LAT == 2) {
                Syyb += pb * wi * 4.5 * (cy * cy - th);
                Sxyb += pb * wi * 9.0 * cx * cy;
            }
        }
        // S_xx = 2 G_x u_x + cg G_x^2/rho + cl Lap;  S_yy likewise;  S_xy = G_x u_y + u_x G_y + cg G_x G_y/rho
        const double ir = 1.0 / r;
        Gb[c][0] += Sxxb * (2.0 * ux + 2.0 * cg * gx * ir) + Sxyb * (uy + cg * gy * ir);
        Gb[c][1] += Syyb * (2.0 * uy + 2.0 * cg * gy * ir) + Sxyb * (ux + cg * gx * ir);
        ub[c][0] += Sxxb * 2.0 * gx + Sxyb * gy;
        ub[c][1] += Syyb * 2.0 * gy + Sxyb * gx;
        rhob[c] += -(Sxxb * cg * gx * gx + Syyb * cg * gy * gy + Sxyb * cg * gx * gy) * ir * ir;
        A.lapb[c * n + s] = (Sxxb + Syyb) * cl;
    }
    // friction: G = Gmu + rho h,  M h = rhs,  rhs = -L_W u0,  u0 = u + Gmu/(2 rho)
    double gmub[N][2], Mb[N][N], Wb[N][N];
#pragma unroll
    for (int c = 0; c < N; ++c) {
        gmub[c][0] = Gb[c][0];
        gmub[c][1] = Gb[c][1];
#pragma unroll
        for (int d = 0; d < N; ++d) Mb[c][d] = Wb[c][d] = 0.0;
    }
    if constexpr (N > 1) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
            double hb[N], rb[N];
#pragma unroll
            for (int c = 0; c < N; ++c) {
                rhob[c] += h[a][c] * Gb[c][a];
                hb[c] = rho[c] * Gb[c][a];
            }
#pragma unroll
            for (int c = 0; c < N; ++c) {
                double acc = 0.0;
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
                double u0b = 0.0;
#pragma unroll
                for (int d = 0; d < N; ++d) {
                    u0b += W[c][d] * (rb[d] - rb[c]);
                    Wb[c][d] += -rb[c] * (u0[a][c] - u0[a][d]);
                }
                ub[c][a] += u0b;
                gmub[c][a] += u0b / (2.0 * rho[c]);
                rhob[c] += -u0b * gmu[c][a] / (2.0 * rho[c] * rho[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < N; ++c) {
            rhob[c] += Mb[c][c];
#pragma unroll
            for (int d = 0; d < N; ++d) {
                if (d == c) continue;
                Wb[c][d] += 0.5 * Mb[c][c] - 0.5 * Mb[c][d];
            }
        }
#pragma unroll
        for (int c = 0; c < N; ++c)
#pragma unroll
            for (int d = 0; d < N; ++d) {
                if (d == c) continue;
                const double sum = rho[c] + rho[d];
                const double k = P.lam[c * 4 + d] / (sum * sum);
                rhob[c] += Wb[c][d] * k * rho[d] * rho[d];
                rhob[d] += Wb[c][d] * k * rho[c] * rho[c];
            }
    }
    // u = j / rho;  Gmu = -rho D phi + theta D rho
#pragma unroll
    for (int c = 0; c < N; ++c) {
        const double ir = 1.0 / rho[c];
        double acc = 0.0;
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
template <int LAT, int N>
__global__ void __launch_bounds__(ADJ_THREADS) adj_mubar_kernel(AdjArrays A, DevParams P) {
    using L = Lat<LAT>;
    constexpr int D = L::D;
    constexpr int V = 2 * N * N + N;
    const int nx = P.nx, ny = P.ny;
    const size_t n = (size_t)nx * ny;
    const size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    double acc[V];
#pragma unroll
    for (int k = 0; k < V; ++k) acc[k] = 0.0;
    if (s < n) {
        const int x = (int)(s % nx), y = (int)(s / nx);
        double mb[N], r[N], eta = 1.0, rt = 0.0;
#pragma unroll
        for (int c = 0; c < N; ++c) {
            // div^T: phibar(x) = -sum_a D_a(Dphibar_a)(x)
            double dv = 0.0;
            double gx, gy;
            grad_g<LAT>(A.dphib + (c * D + 0) * n, x, y, nx, ny, gx, gy);
            dv += gx;
            if (D == 2) {
                grad_g<LAT>(A.dphib + (c * D + 1) * n, x, y, nx, ny, gx, gy);
                dv += gy;
            }
            mb[c] = -P.gamma * dv;
            A.mub[c * n + s] = mb[c];
            r[c] = A.rho[c * n + s];
            eta -= P.b[c] * r[c];
            rt += r[c];
        }
        // d mu^c / d a_cd = -2 rho^d;  d mu^c / d kappa_cd = -Lap rho^d;
        // d mu^c / d b^d = kT [rho^d/eta + delta_cd rho_t/eta + b^c rho_t rho^d / eta^2]
#pragma unroll
        for (int c = 0; c < N; ++c)
#pragma unroll
            for (int d = 0; d < N; ++d) {
                acc[c * N + d] = mb[c] * (-2.0 * r[d]);
                acc[N * N + c * N + d] = mb[c] * (-A.lap[d * n + s]);
                acc[2 * N * N + d] += mb[c] * P.kT *
                                      (r[d] / eta + (c == d ? rt / eta : 0.0) + P.b[c] * rt * r[d] / (eta * eta));
            }
    }
    block_sum<V>(acc, A.partial + (size_t)blockIdx.x * V);
}

// ---- rhobar and fbar ---------------------------------------------------------------------
template <int LAT, int N>
__global__ void __launch_bounds__(ADJ_THREADS) adj_rhobar_kernel(double *__restrict__ fbar, AdjArrays A, DevParams P) {
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
        mb[c] = A.mub[c * n + s];
        eta -= P.b[c] * r[c];
        rt += r[c];
    }
    const double ieta = 1.0 / eta;
#pragma unroll
    for (int d = 0; d < N; ++d) {
        double rb = A.rhob[d * n + s];
        // local chemical-potential Jacobian (kT part and the -2a term)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            double J = P.kT * ((c == d ? 1.0 / r[c] : 0.0) + (P.b[c] + P.b[d]) * ieta + P.b[c] * P.b[d] * rt * ieta * ieta) -
                       2.0 * P.a[c * 4 + d];
            rb += mb[c] * J;
        }
        // -kappa Lap rho terms: rhobar^d -= Lap(sum_c kappa_cd mubar^c)
        {
            const double c0 = [&] {
                double t = 0.0;
#pragma unroll
                for (int c = 0; c < N; ++c) t += P.kappa[c * 4 + d] * A.mub[c * n + s];
                return t;
            }();
            double accl = 0.0;
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const size_t nb = Nb<LAT>::at(x, y, i, nx, ny);
                double t = 0.0;
#pragma unroll
                for (int c = 0; c < N; ++c) t += P.kappa[c * 4 + d] * A.mub[c * n + nb];
                accl += L::w(i) * (t - c0);
            }
            rb -= 6.0 * accl;
        }
        // D rho^T and Lap^T
        double gx, gy;
        grad_g<LAT>(A.drhob + (d * D + 0) * n, x, y, nx, ny, gx, gy);
        rb -= gx;
        if (D == 2) {
            grad_g<LAT>(A.drhob + (d * D + 1) * n, x, y, nx, ny, gx, gy);
            rb -= gy;
        }
        rb += lap_g<LAT>(A.lapb + d * n, x, y, nx, ny);
        const double jbx = A.jb[(d * D + 0) * n + s];
        const double jby = D == 2 ? A.jb[(d * D + 1) * n + s] : 0.0;
#pragma unroll
        for (int i = 0; i < Q; ++i) fbar[(size_t)(d * Q + i) * n + s] += rb + L::vx(i) * jbx + L::vy(i) * jby;
    }
}

// ---- small helpers -------------------------------------------------------------------
template <int V>
__global__ void adj_accum_kernel(const double *__restrict__ step, double *__restrict__ accum) {
    if (threadIdx.x == 0)
        for (int k = 0; k < V; ++k) accum[k] += step[k];
}

// fbar_i = rhobar for every i (the loss depends on f only through rho = sum_i f_i)
__global__ void adj_seed_kernel(const double *__restrict__ rb, double *__restrict__ fb, int N, int Q, size_t n) {
    const size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    for (int c = 0; c < N; ++c)
        for (int i = 0; i < Q; ++i) fb[(size_t)(c * Q + i) * n + s] = rb[c * n + s];
}

// f_0 = w_i rho_0 (equilibrium at rest): rhobar_0 = sum_i w_i fbar_0,i
template <int LAT>
__global__ void adj_init_transpose_kernel(const double *__restrict__ fb, double *__restrict__ rb, int N, size_t n) {
    using L = Lat<LAT>;
    const size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    for (int c = 0; c < N; ++c) {
        double acc = 0.0;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) acc += L::w(i) * fb[(size_t)(c * L::Q + i) * n + s];
        rb[c * n + s] = acc;
    }
}

}  // namespace lbvdw
