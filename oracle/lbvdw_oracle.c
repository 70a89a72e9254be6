/*
 * lbvdw_oracle.c -- plain FP64 CPU oracle of one lattice Boltzmann timestep for
 * an N-component van der Waals mixture (Ridl & Wagner, arXiv:1805.07251).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this file's library.  It shares no source,
 * header, table or helper with the CUDA library: lattice tables, stencils and
 * every formula below are written out here on their own.
 *
 * One timestep is taken in the paper's order, over the whole lattice for each
 * stage before the next stage starts (no fusion, no blocking):
 *   stage 1  moments rho^c = sum_i f_i^c, rho^c u^c = sum_i f_i^c v_i   (Sec. III)
 *   stage 2  chemical potential mu^c from the interaction function psi^{cc'}
 *            (Eq. discreteChemicalPotential; psi from Eqs. a-psi, kappa-psi,
 *            and for D1Q3 the explicit psi of Sec. V)
 *   stage 3  thermodynamic force, "log" (Eq. forceMuLog) or "nid" (Eq. forceMuId)
 *   stage 4  friction with the implicit u-hat (Eq. forceFriction), solved
 *            as an N x N linear system per node and direction
 *   stage 5  Psi correction (Eq. forceCorrectionsPsi)
 *   stage 6  equilibrium (Eq. feq), forcing populations with the moments of
 *            Sec. III, collision (Eq. BGKcollisionOperator): single tau (BGK), or
 *            on D2Q9 optionally distinct relaxation times per moment eigenspace
 *   stage 7  streaming (Eq. LBequation), periodic in every direction
 *
 * Readings of the paper taken here, where it is silent or its printed signs
 * disagree with one another (the reason follows each):
 *   - the momentum GAINED by component c is G^c = -gamma rho^c D mu^c
 *     + theta D rho^c ("log") -- the sign that makes grad mu = 0 the steady
 *     state (Eq. forceMuNid read as the force on the left of the momentum
 *     equation, Sec. IV);
 *   - friction gain G^{f,c} = -sum_c' lambda m (u^c - u^c') with u-hat;
 *   - the second forcing moment is G u + u G + psi_sign * Psi with
 *     psi_sign = -1 by default, as in the explicit D1Q3 update of Sec. V;
 *   - theta (lattice temperature, 1/3) enters f^eq, the forcing populations
 *     and the ideal part of the force; kT enters only mu, p and F;
 *   - the constant +kT that d(rho ln rho)/d rho would add to mu is omitted,
 *     as printed in Eq. discreteChemicalPotential;
 *   - D2Q9 (not in the paper) uses psi(v_i != 0) = -(kappa/theta) w_i and
 *     psi(0) = -a + (kappa/theta)(1 - w_0), which satisfies Eqs. a-psi and
 *     kappa-psi; the D2Q9 gradient is (1/theta) sum_i w_i v_i phi(x + v_i).
 *
 * Data layout: f[c][i][y][x], rho[c][y][x], mom[c][d][y][x] (d = 0: x, 1: y).
 *
 * Threads: when compiled with OpenMP, the rows of each stage are shared among
 * threads.  Every node is still computed by the same arithmetic in the same
 * order (no reduction crosses nodes, except the free energy, which stays serial),
 * so the results are bitwise the same for any number of threads.
 *
 * Parity status: every function is pinned by the oracle tests (closed forms,
 * invariants, the paper's explicit D1Q3 update, textbook coexistence, the
 * Maxwell-Stefan interdiffusion rate of Sec. IV for the friction lambda).  The
 * "nid" force is pinned by its exact zero for an ideal mixture at gamma kT = theta
 * and by its second-order agreement with the "log" force under refinement; the
 * pivoted N-component friction solve by the closed-form uniform relaxation
 * u_{n+1} = (D + L/2)^-1 (D - L/2) u_n.  Lambda in nonlinear dynamics is pinned
 * by the interdiffusion of an ideal mixture, which the Maxwell-Stefan balance of
 * Sec. IV makes linear diffusion at any composition: a wave from x = 0.1 to 0.9
 * decays at the small-amplitude rate.  No function here is without a pin; what no
 * closed form covers is the transient of coarsening and interface motion, whose
 * end states are pinned (coexistence on the common tangent, the Maxwell
 * construction) but whose rates are not.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_E_INVALID 1
#define ORC_E_NOMEM 2
#define ORC_E_DOMAIN 4

/* lattice temperature: sound speed squared of D1Q3 and D2Q9 (Sec. V, theta = 1/3) */
static const double THETA = 1.0 / 3.0;

typedef struct {
    int lattice;          /* 1 = D1Q3, 2 = D2Q9 */
    int nx, ny, ncomp;    /* ny = 1 for D1Q3 */
    double tau;           /* BGK relaxation time */
    double kT;            /* thermodynamic temperature in mu, p and F */
    double gamma_mu;      /* prefactor of mu in the force, Eq. forceMuNid */
    double a[16], kappa[16], lambda[16], b[4];  /* ncomp x ncomp, row major */
    int force_method;     /* 0 = "log" (Eq. forceMuLog), 1 = "nid" (Eq. forceMuId) */
    double psi_sign;      /* sign of Psi in the second forcing moment (-1 default) */
    /* Collision matrix of Eq. BGKcollisionOperator, diagonal in a moment basis (D2Q9
     * only; D1Q3 has a single non-conserved moment, so its collision is always BGK):
     * mrt = 0: one relaxation time tau for every moment (BGK);
     * mrt = 1: tau for the bulk moment (trace of the second moment), tau_s for the two
     * shear moments (its traceless part), tau_g for the three ghost moments. */
    int mrt;
    double tau_s, tau_g;
} orc_params;

/* ---- lattices --------------------------------------------------------- */

/* D1Q3: v in {0, +1, -1} (Sec. V); weights from the D1Q3 update at theta = 1/3 */
static const int D1Q3_VX[3] = {0, 1, -1};
static const double D1Q3_W[3] = {2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0};

/* D2Q9: rest, 4 axis, 4 diagonal; weights 4/9, 1/9, 1/36 */
static const int D2Q9_VX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int D2Q9_VY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double D2Q9_W[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                                 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

typedef struct {
    int q, d;
    const int *vx, *vy;
    const double *w;
} lattice_t;

static int get_lattice(const orc_params *p, lattice_t *L) {
    static const int zero9[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (p->lattice == 1) {
        L->q = 3; L->d = 1; L->vx = D1Q3_VX; L->vy = zero9; L->w = D1Q3_W;
        return p->ny == 1 ? ORC_OK : ORC_E_INVALID;
    }
    if (p->lattice == 2) {
        L->q = 9; L->d = 2; L->vx = D2Q9_VX; L->vy = D2Q9_VY; L->w = D2Q9_W;
        return ORC_OK;
    }
    return ORC_E_INVALID;
}

static int check_params(const orc_params *p, lattice_t *L) {
    if (get_lattice(p, L) != ORC_OK) return ORC_E_INVALID;
    if (p->nx < 1 || p->ny < 1 || p->ncomp < 1 || p->ncomp > 4) return ORC_E_INVALID;
    if (!(p->tau > 0.5)) return ORC_E_INVALID;
    if (p->mrt && !(p->tau_s > 0.5 && p->tau_g > 0.5)) return ORC_E_INVALID;
    return ORC_OK;
}

/* periodic neighbour index of node (x, y) shifted by (dx, dy) */
static long nb(const orc_params *p, int x, int y, int dx, int dy) {
    int xx = ((x + dx) % p->nx + p->nx) % p->nx;
    int yy = ((y + dy) % p->ny + p->ny) % p->ny;
    return (long)yy * p->nx + xx;
}

/* ---- interaction function psi^{cc'}(dx) -------------------------------- */

/* psi for lattice vector i (i = 0 is the node itself).
 * D1Q3: psi(0) = kappa - a, psi(+-1) = -kappa/2 (Sec. V, from Eqs.
 * kappa-psi-D1Q3 and a-psi-D1Q3).  D2Q9: the weighted extension that keeps
 * -sum psi = a and -sum psi dx_a dx_b = kappa delta_ab (Eqs. a-psi, kappa-psi). */
static double psi(const orc_params *p, const lattice_t *L, int c, int cc, int i) {
    double a = p->a[c * 4 + cc], k = p->kappa[c * 4 + cc];
    if (p->lattice == 1) {
        if (i == 0) return k - a;
        return -0.5 * k;
    }
    if (i == 0) return -a + (k / THETA) * (1.0 - L->w[0]);
    return -(k / THETA) * L->w[i];
}

/* ---- stage 1: moments --------------------------------------------------- */

int orc_moments(const orc_params *p, const double *f, double *rho, double *mom) {
    lattice_t L;
    if (check_params(p, &L) != ORC_OK) return ORC_E_INVALID;
    long n = (long)p->nx * p->ny;
    for (int c = 0; c < p->ncomp; ++c)
#pragma omp parallel for schedule(static)
        for (long s = 0; s < n; ++s) {
            double r = 0.0, jx = 0.0, jy = 0.0;
            for (int i = 0; i < L.q; ++i) {
                double fi = f[((long)c * L.q + i) * n + s];
                r += fi;
                jx += fi * L.vx[i];
                jy += fi * L.vy[i];
            }
            rho[(long)c * n + s] = r;
            if (mom) {
                mom[((long)c * L.d + 0) * n + s] = jx;
                if (L.d == 2) mom[((long)c * L.d + 1) * n + s] = jy;
            }
        }
    return ORC_OK;
}

/* ---- stage 2: chemical potential ---------------------------------------- */

/* mu^c(x) = kT ln(rho^c / eta) + kT b^c rho / eta
 *         + 2 sum_c' sum_dx psi^{cc'}(dx) rho^c'(x + dx),  eta = 1 - sum b rho
 * (Eq. discreteChemicalPotential, with theta there being kT). */
int orc_mu(const orc_params *p, const double *rho, double *mu) {
    lattice_t L;
    if (check_params(p, &L) != ORC_OK) return ORC_E_INVALID;
    long n = (long)p->nx * p->ny;
    int N = p->ncomp;
    int bad = 0;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            long s = (long)y * p->nx + x;
            double eta = 1.0, rtot = 0.0;
            for (int c = 0; c < N; ++c) {
                eta -= p->b[c] * rho[(long)c * n + s];
                rtot += rho[(long)c * n + s];
            }
            if (!(eta > 0.0)) {
#pragma omp atomic write
                bad = 1;
                continue;
            }
            for (int c = 0; c < N; ++c) {
                double rc = rho[(long)c * n + s];
                if (!(rc > 0.0)) {
#pragma omp atomic write
                    bad = 1;
                    continue;
                }
                double m = p->kT * log(rc / eta) + p->kT * p->b[c] * rtot / eta;
                double inter = 0.0;
                for (int cc = 0; cc < N; ++cc)
                    for (int i = 0; i < L.q; ++i)
                        inter += psi(p, &L, c, cc, i) *
                                 rho[(long)cc * n + nb(p, x, y, L.vx[i], L.vy[i])];
                mu[(long)c * n + s] = m + 2.0 * inter;
            }
        }
    return bad ? ORC_E_DOMAIN : ORC_OK;
}

/* ---- lattice difference operators --------------------------------------- */

/* central-difference gradient D_a phi.  D1Q3: (phi(x+1) - phi(x-1)) / 2, the
 * central difference of Sec. V.  D2Q9: (1/theta) sum_i w_i v_ia phi(x + v_i). */
static void grad(const orc_params *p, const lattice_t *L, const double *phi, int x, int y,
                 double g[2]) {
    if (p->lattice == 1) {
        g[0] = 0.5 * (phi[nb(p, x, y, 1, 0)] - phi[nb(p, x, y, -1, 0)]);
        g[1] = 0.0;
        return;
    }
    double gx = 0.0, gy = 0.0;
    for (int i = 1; i < L->q; ++i) {
        double v = phi[nb(p, x, y, L->vx[i], L->vy[i])];
        gx += L->w[i] * L->vx[i] * v;
        gy += L->w[i] * L->vy[i] * v;
    }
    g[0] = gx / THETA;
    g[1] = gy / THETA;
}

/* Laplacian.  D1Q3: phi(x+1) - 2 phi(x) + phi(x-1), the stencil that psi of
 * Sec. V implies.  D2Q9: (2/theta) sum_i w_i (phi(x + v_i) - phi(x)). */
static double lap(const orc_params *p, const lattice_t *L, const double *phi, int x, int y) {
    long s = (long)y * p->nx + x;
    if (p->lattice == 1)
        return phi[nb(p, x, y, 1, 0)] - 2.0 * phi[s] + phi[nb(p, x, y, -1, 0)];
    double acc = 0.0;
    for (int i = 1; i < L->q; ++i)
        acc += L->w[i] * (phi[nb(p, x, y, L->vx[i], L->vy[i])] - phi[s]);
    return 2.0 * acc / THETA;
}

/* ---- small dense solve (Gaussian elimination, partial pivoting) --------- */

static int solve(int n, double A[4][4], double bvec[4], double xout[4]) {
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int r = k + 1; r < n; ++r)
            if (fabs(A[r][k]) > fabs(A[piv][k])) piv = r;
        if (A[piv][k] == 0.0) return ORC_E_DOMAIN;
        if (piv != k) {
            for (int cidx = 0; cidx < n; ++cidx) {
                double t = A[k][cidx]; A[k][cidx] = A[piv][cidx]; A[piv][cidx] = t;
            }
            double t = bvec[k]; bvec[k] = bvec[piv]; bvec[piv] = t;
        }
        for (int r = k + 1; r < n; ++r) {
            double m = A[r][k] / A[k][k];
            for (int cidx = k; cidx < n; ++cidx) A[r][cidx] -= m * A[k][cidx];
            bvec[r] -= m * bvec[k];
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        double s = bvec[k];
        for (int cidx = k + 1; cidx < n; ++cidx) s -= A[k][cidx] * xout[cidx];
        xout[k] = s / A[k][k];
    }
    return ORC_OK;
}

/* ---- stages 3 and 4: forces ----------------------------------------------- */

/* Total momentum gain G^c (mean-field force plus friction) and the
 * mean-field part Gmu^c at every node; layout [c][d][y][x].
 *   stage 3 ("log"):  Gmu^c = -gamma rho^c D mu^c + theta D rho^c
 *   stage 3 ("nid"):  Gmu^c = -rho^c D (gamma mu^c - theta ln rho^c)
 *   stage 4: G^{f,c} = -sum_c' lambda^{cc'} m^{cc'} (uh^c - uh^{c'}),
 *            m = rho^c rho^c' / (rho^c + rho^c'), uh^c = u^c + G^c / (2 rho^c),
 *            with G^c = Gmu^c + G^{f,c}: linear in G^f, solved per direction. */
static int forces(const orc_params *p, const lattice_t *L, const double *rho, const double *mom,
                  const double *mu, double *lnrho, double *G, double *Gmu) {
    long n = (long)p->nx * p->ny;
    int N = p->ncomp;
    int bad = 0;
    if (p->force_method == 1)
#pragma omp parallel for schedule(static)
        for (long s = 0; s < (long)N * n; ++s) lnrho[s] = log(rho[s]);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            long s = (long)y * p->nx + x;
            double gm[4][2];
            for (int c = 0; c < N; ++c) {
                double gmu[2], grho[2];
                grad(p, L, mu + (long)c * n, x, y, gmu);
                double rc = rho[(long)c * n + s];
                if (p->force_method == 1) {
                    double gl[2];
                    grad(p, L, lnrho + (long)c * n, x, y, gl);
                    for (int a = 0; a < L->d; ++a)
                        gm[c][a] = -rc * (p->gamma_mu * gmu[a] - THETA * gl[a]);
                } else {
                    grad(p, L, rho + (long)c * n, x, y, grho);
                    for (int a = 0; a < L->d; ++a)
                        gm[c][a] = -p->gamma_mu * rc * gmu[a] + THETA * grho[a];
                }
            }
            for (int a = 0; a < L->d; ++a) {
                /* A Gf = rhs, from Gf^c + sum_c' W_cc' (Gf^c/(2 rho^c) - Gf^c'/(2 rho^c'))
                 *                  = -sum_c' W_cc' (u0^c - u0^c'),  u0 = u + Gmu/(2 rho) */
                double A[4][4], rhs[4], gf[4], u0[4];
                for (int c = 0; c < N; ++c) {
                    double rc = rho[(long)c * n + s];
                    u0[c] = mom[((long)c * L->d + a) * n + s] / rc + gm[c][a] / (2.0 * rc);
                }
                for (int c = 0; c < N; ++c) {
                    double rc = rho[(long)c * n + s];
                    rhs[c] = 0.0;
                    for (int cc = 0; cc < N; ++cc) A[c][cc] = (c == cc) ? 1.0 : 0.0;
                    for (int cc = 0; cc < N; ++cc) {
                        if (cc == c) continue;
                        double rcc = rho[(long)cc * n + s];
                        double W = p->lambda[c * 4 + cc] * rc * rcc / (rc + rcc);
                        A[c][c] += W / (2.0 * rc);
                        A[c][cc] -= W / (2.0 * rcc);
                        rhs[c] -= W * (u0[c] - u0[cc]);
                    }
                }
                if (solve(N, A, rhs, gf) != ORC_OK) {
#pragma omp atomic write
                    bad = 1;
                    continue;
                }
                for (int c = 0; c < N; ++c) {
                    G[((long)c * L->d + a) * n + s] = gm[c][a] + gf[c];
                    if (Gmu) Gmu[((long)c * L->d + a) * n + s] = gm[c][a];
                }
            }
        }
    return bad ? ORC_E_DOMAIN : ORC_OK;
}

/* ---- Hermite basis of D1Q3 (and, as products, of D2Q9) at theta = 1/3 ------- */

/* P_0 = 1, P_1 = v, P_2 = v^2 - theta: orthogonal under the D1Q3 weights */
static double herm(int k, int v) { return k == 0 ? 1.0 : (k == 1 ? (double)v : (double)(v * v) - THETA); }

/* sum_i w_i P_k(v_i)^2 over D1Q3: 1, theta, 2 theta^2 */
static double herm_norm(int k) { return k == 0 ? 1.0 : (k == 1 ? THETA : 2.0 * THETA * THETA); }

/* ---- one timestep ---------------------------------------------------------- */

typedef struct {
    double *rho, *mom, *mu, *lnrho, *G, *fpost;
} work_t;

static int step(const orc_params *p, const lattice_t *L, double *f, work_t *w) {
    long n = (long)p->nx * p->ny;
    int N = p->ncomp, Q = L->q, D = L->d;
    const int mrt = p->mrt && p->lattice == 2;
    int rc = orc_moments(p, f, w->rho, w->mom);                  /* stage 1 */
    if (rc) return rc;
    rc = orc_mu(p, w->rho, w->mu);                               /* stage 2 */
    if (rc) return rc;
    rc = forces(p, L, w->rho, w->mom, w->mu, w->lnrho, w->G, 0); /* stages 3, 4 */
    if (rc) return rc;
    for (int c = 0; c < N; ++c)
#pragma omp parallel for schedule(static)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long s = (long)y * p->nx + x;
                double r = w->rho[(long)c * n + s];
                double u[2] = {0.0, 0.0}, G[2] = {0.0, 0.0};
                for (int a = 0; a < D; ++a) {
                    u[a] = w->mom[((long)c * D + a) * n + s] / r;
                    G[a] = w->G[((long)c * D + a) * n + s];
                }
                /* stage 5: Psi_ab = -(1/tau)[(tau - 1/4) G_a G_b / rho + (1/12) lap rho delta_ab] */
                double lr = lap(p, L, w->rho + (long)c * n, x, y);
                double Psi[2][2];
                for (int a = 0; a < 2; ++a)
                    for (int bb = 0; bb < 2; ++bb)
                        Psi[a][bb] = -(1.0 / p->tau) *
                                     ((p->tau - 0.25) * G[a] * G[bb] / r + (a == bb ? lr / 12.0 : 0.0));
                if (mrt) {
                    /* distinct relaxation times: the same correction taken per eigenspace
                     * of the second moment, the trace part (|G|^2/2 I / rho and the
                     * Laplacian) with the bulk tau, the traceless part of G G / rho with
                     * tau_s; equal to the line above when tau_s = tau */
                    double tr = 0.5 * (G[0] * G[0] + G[1] * G[1]);
                    for (int a = 0; a < 2; ++a)
                        for (int bb = 0; bb < 2; ++bb) {
                            double iso = (a == bb ? tr : 0.0);
                            Psi[a][bb] = -(1.0 / p->tau) * ((p->tau - 0.25) * iso / r + (a == bb ? lr / 12.0 : 0.0))
                                         - (1.0 / p->tau_s) * (p->tau_s - 0.25) * (G[a] * G[bb] - iso) / r;
                        }
                }
                /* second forcing moment S_ab = G_a u_b + u_a G_b + psi_sign Psi_ab */
                double S[2][2];
                for (int a = 0; a < 2; ++a)
                    for (int bb = 0; bb < 2; ++bb)
                        S[a][bb] = G[a] * u[bb] + u[a] * G[bb] + p->psi_sign * Psi[a][bb];
                double usq = u[0] * u[0] + u[1] * u[1];
                /* stage 6: Hermite equilibrium (Eq. feq) and forcing populations
                 * F_i = w_i [ v.G/theta + S:(v v - theta I)/(2 theta^2) ], whose
                 * moments are 0, G and S (Sec. III).  The moving populations
                 * (i = 1 .. Q-1) come from these forms; the rest population (i = 0)
                 * from the zeroth-moment conditions that define f^eq and F in
                 * Sec. III, sum_i f_i^eq = rho and sum_i F_i = 0 (the Hermite forms
                 * satisfy them in exact arithmetic, but the rounded weights w_i do not
                 * sum to one, which would change the mass by a fixed fraction each
                 * step). */
                double feq_moving = 0.0, F_moving = 0.0;
                double feq[9], Fv[9], fv[9], post[9];
                for (int k = 1; k <= Q; ++k) {
                    const int i = k % Q; /* 1, 2, ..., Q-1, then the rest population 0 */
                    double v[2] = {(double)L->vx[i], (double)L->vy[i]};
                    double vu = v[0] * u[0] + v[1] * u[1];
                    feq[i] = r * L->w[i] *
                             (1.0 + vu / THETA + vu * vu / (2.0 * THETA * THETA) - usq / (2.0 * THETA));
                    double vG = v[0] * G[0] + v[1] * G[1];
                    double SQ = 0.0;
                    for (int a = 0; a < D; ++a)
                        for (int bb = 0; bb < D; ++bb)
                            SQ += S[a][bb] * (v[a] * v[bb] - (a == bb ? THETA : 0.0));
                    Fv[i] = L->w[i] * (vG / THETA + SQ / (2.0 * THETA * THETA));
                    if (i == 0) {
                        feq[0] = r - feq_moving;
                        Fv[0] = -F_moving;
                    } else {
                        feq_moving += feq[i];
                        F_moving += Fv[i];
                    }
                    fv[i] = f[((long)c * Q + i) * n + s];
                }
                if (!mrt) {
                    /* BGK (Eq. BGKcollisionOperator, single relaxation time) */
                    for (int i = 0; i < Q; ++i) post[i] = fv[i] + (feq[i] - fv[i]) / p->tau + Fv[i];
                } else {
                    /* Eq. BGKcollisionOperator with the collision matrix diagonal in the
                     * D2Q9 Hermite basis H_a(v) = P_ax(v_x) P_ay(v_y), P in {1, v, v^2 -
                     * theta}, orthogonal under the weights with norms N_a = sum_i w_i H_a^2:
                     *   Omega_i = w_i sum_a (1/tau_a) H_a(v_i) m_a / N_a,
                     *   m_a = sum_j H_a(v_j) (f_j^eq - f_j).
                     * 1/tau_a: conserved moments (1, v_x, v_y; m_a = 0) and the bulk
                     * combination H_xx + H_yy take tau; H_xx - H_yy and H_xy take tau_s;
                     * H_xxy, H_xyy, H_xxyy take tau_g.  The rest population again comes
                     * from the zeroth-moment condition sum_i Omega_i = 0. */
                    double m[3][3];
                    for (int ax = 0; ax < 3; ++ax)
                        for (int ay = 0; ay < 3; ++ay) {
                            double acc = 0.0;
                            for (int i = 0; i < Q; ++i)
                                acc += herm(ax, L->vx[i]) * herm(ay, L->vy[i]) * (feq[i] - fv[i]);
                            m[ax][ay] = acc;
                        }
                    /* bulk / shear split of the H_xx (ax = 2, ay = 0) and H_yy moments */
                    double bulk = 0.5 * (m[2][0] + m[0][2]) / p->tau;
                    double shear = 0.5 * (m[2][0] - m[0][2]) / p->tau_s;
                    double om_moving = 0.0;
                    for (int k = 1; k <= Q; ++k) {
                        const int i = k % Q;
                        double acc = 0.0;
                        for (int ax = 0; ax < 3; ++ax)
                            for (int ay = 0; ay < 3; ++ay) {
                                double Ha = herm(ax, L->vx[i]) * herm(ay, L->vy[i]);
                                double Na = herm_norm(ax) * herm_norm(ay);
                                double rate;
                                if (ax + ay <= 1) rate = 1.0 / p->tau;          /* conserved */
                                else if (ax == 1 && ay == 1) rate = 1.0 / p->tau_s;
                                else if (ax + ay == 2) continue;                /* H_xx, H_yy below */
                                else rate = 1.0 / p->tau_g;                     /* ghosts */
                                acc += rate * Ha * m[ax][ay] / Na;
                            }
                        double hxx = herm(2, L->vx[i]), hyy = herm(2, L->vy[i]);
                        acc += (bulk * (hxx + hyy) + shear * (hxx - hyy)) / herm_norm(2);
                        double om = L->w[i] * acc;
                        if (i == 0) om = -om_moving;
                        else om_moving += om;
                        post[i] = fv[i] + om + Fv[i];
                    }
                }
                /* stage 7: streaming, f_i(x + v_i, t + 1) = post-collision f_i(x, t) */
                for (int i = 0; i < Q; ++i)
                    w->fpost[((long)c * Q + i) * n + nb(p, x, y, L->vx[i], L->vy[i])] = post[i];
            }
    memcpy(f, w->fpost, sizeof(double) * (size_t)N * Q * n);
    return ORC_OK;
}

static void free_work(work_t *w) {
    free(w->rho); free(w->mom); free(w->mu); free(w->lnrho); free(w->G); free(w->fpost);
}

static int alloc_work(const orc_params *p, const lattice_t *L, work_t *w) {
    size_t n = (size_t)p->nx * p->ny, N = (size_t)p->ncomp;
    w->rho = malloc(sizeof(double) * N * n);
    w->mom = malloc(sizeof(double) * N * L->d * n);
    w->mu = malloc(sizeof(double) * N * n);
    w->lnrho = malloc(sizeof(double) * N * n);
    w->G = malloc(sizeof(double) * N * L->d * n);
    w->fpost = malloc(sizeof(double) * N * L->q * n);
    if (!w->rho || !w->mom || !w->mu || !w->lnrho || !w->G || !w->fpost) {
        free_work(w);
        return ORC_E_NOMEM;
    }
    return ORC_OK;
}

/* Advance f (layout [c][i][y][x], pre-collision populations at time t) by
 * nsteps timesteps in place.  Returns ORC_E_DOMAIN as soon as rho^c <= 0 or
 * eta <= 0 is met; f then holds the state at the start of the failing step. */
int orc_run(const orc_params *p, double *f, long nsteps) {
    lattice_t L;
    if (check_params(p, &L) != ORC_OK || nsteps < 0) return ORC_E_INVALID;
    work_t w;
    if (alloc_work(p, &L, &w) != ORC_OK) return ORC_E_NOMEM;
    int rc = ORC_OK;
    for (long t = 0; t < nsteps && rc == ORC_OK; ++t) rc = step(p, &L, f, &w);
    free_work(&w);
    return rc;
}

/* Forces of the current state: total gain G and mean-field part Gmu,
 * layout [c][d][y][x]. */
int orc_forces(const orc_params *p, const double *f, double *G, double *Gmu) {
    lattice_t L;
    if (check_params(p, &L) != ORC_OK) return ORC_E_INVALID;
    work_t w;
    if (alloc_work(p, &L, &w) != ORC_OK) return ORC_E_NOMEM;
    int rc = orc_moments(p, f, w.rho, w.mom);
    if (!rc) rc = orc_mu(p, w.rho, w.mu);
    if (!rc) rc = forces(p, &L, w.rho, w.mom, w.mu, w.lnrho, G, Gmu);
    free_work(&w);
    return rc;
}

/* Populations of the equilibrium (Eq. feq) for densities rho [c][y][x] and
 * momenta mom [c][d][y][x] (NULL: at rest). */
int orc_equilibrium(const orc_params *p, const double *rho, const double *mom, double *f) {
    lattice_t L;
    if (check_params(p, &L) != ORC_OK) return ORC_E_INVALID;
    long n = (long)p->nx * p->ny;
    for (int c = 0; c < p->ncomp; ++c)
#pragma omp parallel for schedule(static)
        for (long s = 0; s < n; ++s) {
            double r = rho[(long)c * n + s];
            double u[2] = {0.0, 0.0};
            if (mom)
                for (int a = 0; a < L.d; ++a) u[a] = mom[((long)c * L.d + a) * n + s] / r;
            double usq = u[0] * u[0] + u[1] * u[1];
            for (int i = 0; i < L.q; ++i) {
                double vu = L.vx[i] * u[0] + L.vy[i] * u[1];
                f[((long)c * L.q + i) * n + s] =
                    r * L.w[i] *
                    (1.0 + vu / THETA + vu * vu / (2.0 * THETA * THETA) - usq / (2.0 * THETA));
            }
        }
    return ORC_OK;
}

/* Lattice free energy of Eq. discreteFreeEnergy for densities rho [c][y][x]:
 * F = sum_x sum_c [ kT rho^c ln(rho^c/eta) + sum_c' sum_dx psi^{cc'}(dx) rho^c(x) rho^c'(x+dx) ].
 * Also returns the per-component mass sum_x rho^c when mass != NULL. */
int orc_free_energy(const orc_params *p, const double *rho, double *F, double *mass) {
    lattice_t L;
    if (check_params(p, &L) != ORC_OK) return ORC_E_INVALID;
    long n = (long)p->nx * p->ny;
    int N = p->ncomp;
    double tot = 0.0;
    for (int c = 0; c < N && mass; ++c) mass[c] = 0.0;
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            long s = (long)y * p->nx + x;
            double eta = 1.0;
            for (int c = 0; c < N; ++c) eta -= p->b[c] * rho[(long)c * n + s];
            if (!(eta > 0.0)) return ORC_E_DOMAIN;
            for (int c = 0; c < N; ++c) {
                double rc = rho[(long)c * n + s];
                if (!(rc > 0.0)) return ORC_E_DOMAIN;
                if (mass) mass[c] += rc;
                double term = p->kT * rc * log(rc / eta);
                for (int cc = 0; cc < N; ++cc)
                    for (int i = 0; i < L.q; ++i)
                        term += psi(p, &L, c, cc, i) * rc *
                                rho[(long)cc * n + nb(p, x, y, L.vx[i], L.vy[i])];
                tot += term;
            }
        }
    *F = tot;
    return ORC_OK;
}

int orc_abi_q(int lattice) { return lattice == 1 ? 3 : (lattice == 2 ? 9 : 0); }

/* Number of threads the stages use (1 without OpenMP); n < 1 leaves it unchanged.
 * Returns the number in effect. */
int orc_set_threads(int n) {
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
