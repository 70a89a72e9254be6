"""Bulk thermodynamics of the van der Waals mixture and coexistence solvers.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Everything here is the
bulk, spatially constant limit of the lattice free energy of Ridl & Wagner,
Sec. II, written out in NumPy in FP64:

* free-energy density  f(rho) = sum_c kT rho^c ln(rho^c/eta) - sum_cc' a^{cc'} rho^c rho^c'
  with eta = 1 - sum_c b^c rho^c  (Eq. continuousFreeEnergy, constant densities);
* chemical potential   mu^c = df/drho^c  (Eq. discreteChemicalPotential in the
  bulk; this module keeps the constant +kT that the paper drops, so
  ``mu_bulk - kT`` equals the lattice mu of a uniform state);
* pressure             p = sum_c rho^c kT/eta - sum_cc' a rho^c rho^c'  (Sec. II);
* critical point of one component, theta_cr = 8a/(27b), rho_cr = 1/(3b),
  p_cr = a/(27 b^2)  (Eqs. tetcr, rhocr, pcr);
* the 2 x 2 (N x N) Hessian of f and its stability test (Sec. VI);
* single-component coexistence by Maxwell's equal-area rule (equal mu and p);
* two-component coexistence by the lower convex hull of f on a fine grid
  (the common-tangent construction), polished by Newton's method on equal
  mu^A, mu^B and p.  This is an independent minimisation of the same bulk
  free energy the paper minimises with its own algorithm (Appendix A).
"""
from __future__ import annotations

import numpy as np

# --------------------------------------------------------------------------
# parameter maps (Sec. II critical relations, Sec. VI component choice)
# --------------------------------------------------------------------------


def critical_point(a, b):
    """(theta_cr, rho_cr, p_cr) of one van der Waals component (Eqs. tetcr, rhocr, pcr)."""
    return 8.0 * a / (27.0 * b), 1.0 / (3.0 * b), a / (27.0 * b * b)


def ab_from_critical(theta_cr, rho_cr):
    """a and b from the critical temperature and density.

    Inverting Eqs. tetcr and rhocr gives b = 1/(3 rho_cr) and
    a = 27 b theta_cr / 8 = 9 theta_cr / (8 rho_cr).  The paper's Sec. VI
    prints theta_cr squared in a; the linear form is the one consistent with
    Eq. tetcr and with the (xi, zeta, Lambda) values printed in its captions.
    """
    b = 1.0 / (3.0 * rho_cr)
    a = 9.0 * theta_cr / (8.0 * rho_cr)
    return a, b


def mixture_from_critical(theta_A, theta_B, rho_B, nu, kappa, rho_A=1.0):
    """Two-component parameters of Sec. VI: geometric mixing a^AB = nu sqrt(a^A a^B),
    kappa^AB = nu kappa (Eq. vdwConstantAB and the text after it)."""
    aA, bA = ab_from_critical(theta_A, rho_A)
    aB, bB = ab_from_critical(theta_B, rho_B)
    aAB = nu * np.sqrt(aA * aB)
    a = np.array([[aA, aAB], [aAB, aB]])
    k = np.array([[kappa, nu * kappa], [nu * kappa, kappa]])
    return a, np.array([bA, bB]), k


def konynenburg_scott(a, b):
    """(xi, zeta, Lambda) of van Konynenburg and Scott, as defined in Sec. VI."""
    aA, aB, aAB = a[0, 0], a[1, 1], a[0, 1]
    bA, bB = b[0], b[1]
    xi = (bB - bA) / (bA + bB)
    pA, pB = aA / bA ** 2, aB / bB ** 2
    zeta = (pB - pA) / (pA + pB)
    lam = (pA - 2.0 * aAB / (bA * bB) + pB) / (pA + pB)
    return xi, zeta, lam


def one_fluid_critical_temperature(a, b, x):
    """van der Waals one-fluid critical temperature 8 (x.a.x) / (27 b.x) at mole fractions x."""
    x = np.asarray(x, dtype=np.float64)
    return 8.0 * float(x @ np.asarray(a) @ x) / (27.0 * float(np.asarray(b) @ x))


# --------------------------------------------------------------------------
# bulk functions; rho has shape (N, ...) and broadcasts over trailing axes
# --------------------------------------------------------------------------


def _eta(b, rho):
    return 1.0 - np.tensordot(np.asarray(b), rho, axes=(0, 0))


def free_energy_density(kT, a, b, rho):
    rho = np.asarray(rho, dtype=np.float64)
    eta = _eta(b, rho)
    ideal = np.sum(kT * rho * np.log(rho / eta), axis=0)
    attr = np.einsum("ij,i...,j...->...", np.asarray(a), rho, rho)
    return ideal - attr


def chemical_potential(kT, a, b, rho):
    """mu^c = df/drho^c = kT ln(rho^c/eta) + kT + kT b^c rho_tot/eta - 2 sum_c' a^{cc'} rho^c'."""
    rho = np.asarray(rho, dtype=np.float64)
    b = np.asarray(b)
    eta = _eta(b, rho)
    rt = np.sum(rho, axis=0)
    out = []
    for c in range(rho.shape[0]):
        out.append(kT * np.log(rho[c] / eta) + kT + kT * b[c] * rt / eta
                   - 2.0 * np.tensordot(np.asarray(a)[c], rho, axes=(0, 0)))
    return np.stack(out)


def pressure(kT, a, b, rho):
    rho = np.asarray(rho, dtype=np.float64)
    eta = _eta(b, rho)
    return kT * np.sum(rho, axis=0) / eta - np.einsum("ij,i...,j...->...", np.asarray(a), rho, rho)


def hessian(kT, a, b, rho):
    """d^2 f / drho^c drho^c' at one state rho (shape (N,)), analytic.

    With eta = 1 - b.rho: d mu^c / d rho^c' = kT delta_cc'/rho^c
    + kT (b^c + b^c')/eta + kT b^c b^c' rho_tot / eta^2 - 2 a^{cc'}."""
    rho = np.asarray(rho, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    eta = 1.0 - b @ rho
    rt = rho.sum()
    H = (kT * np.diag(1.0 / rho) + kT * (b[:, None] + b[None, :]) / eta
         + kT * np.outer(b, b) * rt / eta ** 2 - 2.0 * np.asarray(a))
    return H


def is_unstable(kT, a, b, rho):
    """True when the bulk Hessian has a negative eigenvalue (Sec. VI stability test)."""
    return bool(np.linalg.eigvalsh(hessian(kT, a, b, rho))[0] < 0.0)


# --------------------------------------------------------------------------
# single component: Maxwell construction
# --------------------------------------------------------------------------


def spinodal_1c(kT, a, b):
    """Densities where dp/drho = 0 for one component (None above the critical point).

    dp/drho = kT/(1-b rho)^2 - 2 a rho = 0  <=>  2 a rho (1 - b rho)^2 = kT."""
    coeffs = [2.0 * a * b * b, -4.0 * a * b, 2.0 * a, -kT]
    r = np.roots(coeffs)
    r = np.sort(r[np.isreal(r)].real)
    r = r[(r > 0) & (r < 1.0 / b)]
    if len(r) < 2:
        return None
    return r[0], r[1]


def maxwell_1c(kT, a, b, tol=1e-14, maxit=200):
    """Coexisting gas and liquid densities of one van der Waals component:
    equal chemical potential and equal pressure, by Newton's method."""
    sp = spinodal_1c(kT, a, b)
    if sp is None:
        raise ValueError("above the critical temperature")
    A = np.array([[a]])
    B = np.array([b])

    def mu(r):
        return float(chemical_potential(kT, A, B, np.array([r]))[0])

    def p(r):
        return float(pressure(kT, A, B, np.array([r])))

    def dmu(r):
        return float(hessian(kT, A, B, np.array([r]))[0, 0])

    # start: for a pressure P between the spinodal pressures (and above 0) take the gas
    # and liquid densities with p = P; the coexistence pressure is the root of
    # mu_gas(P) - mu_liquid(P) (equal-area rule), found by bisection, then Newton
    from scipy.optimize import brentq
    p_lo = max(p(sp[1]), 1e-300)
    p_hi = p(sp[0])

    def branch(P):
        rg = brentq(lambda r: p(r) - P, 1e-300, sp[0], xtol=1e-300, rtol=1e-15, maxiter=500)
        rl = brentq(lambda r: p(r) - P, sp[1], (1.0 - 1e-15) / b, xtol=1e-300, rtol=1e-15, maxiter=500)
        return rg, rl

    def dmu_of(P):
        rg, rl = branch(P)
        return mu(rg) - mu(rl)

    P = brentq(dmu_of, p_lo * (1 + 1e-12), p_hi * (1 - 1e-12), rtol=1e-14, maxiter=500)
    x = np.array(branch(P))
    for _ in range(maxit):
        F = np.array([mu(x[0]) - mu(x[1]), p(x[0]) - p(x[1])])
        # dp/drho = rho dmu/drho
        J = np.array([[dmu(x[0]), -dmu(x[1])], [x[0] * dmu(x[0]), -x[1] * dmu(x[1])]])
        dx = np.linalg.solve(J, -F)
        x = x + dx
        if np.max(np.abs(dx)) < tol:
            break
    return float(x[0]), float(x[1])


# --------------------------------------------------------------------------
# two components: lower convex hull (common tangent) + Newton polish
# --------------------------------------------------------------------------


class HullPhaseDiagram:
    """Lower convex hull of f(rho^A, rho^B) sampled on a grid.

    A mean state inside a hull facet whose corners lie far apart (more than
    ``split`` in density) is in a coexistence region; the facet corners are
    the approximate coexisting phases (2 distinct corners: two phases, 3:
    three phases)."""

    def __init__(self, kT, a, b, n=600, margin=1e-6):
        from scipy.spatial import ConvexHull

        self.kT, self.a, self.b = kT, np.asarray(a, float), np.asarray(b, float)
        rmaxA = (1.0 - margin) / self.b[0]
        rmaxB = (1.0 - margin) / self.b[1]
        # grid finer near zero density (gas phases) via a square-root map
        s = np.linspace(0.0, 1.0, n + 1)[1:] ** 2
        gA, gB = np.meshgrid(s * rmaxA, s * rmaxB, indexing="ij")
        keep = self.b[0] * gA + self.b[1] * gB < 1.0 - margin
        pts = np.stack([gA[keep], gB[keep]])
        fv = free_energy_density(kT, self.a, self.b, pts)
        self.pts = pts.T.copy()
        self.f = fv
        hull = ConvexHull(np.column_stack([self.pts, fv]))
        eq = hull.equations
        lower = eq[:, 2] < 0.0
        self.simplices = hull.simplices[lower]
        self.eqs = eq[lower]

    def facet_of(self, rho):
        """Index of the lower-hull facet above which the point rho lies."""
        P = self.pts[self.simplices]  # (m, 3, 2)
        v0 = P[:, 1] - P[:, 0]
        v1 = P[:, 2] - P[:, 0]
        v2 = np.asarray(rho)[None, :] - P[:, 0]
        d00 = np.einsum("ij,ij->i", v0, v0)
        d01 = np.einsum("ij,ij->i", v0, v1)
        d11 = np.einsum("ij,ij->i", v1, v1)
        d20 = np.einsum("ij,ij->i", v2, v0)
        d21 = np.einsum("ij,ij->i", v2, v1)
        den = d00 * d11 - d01 * d01
        with np.errstate(divide="ignore", invalid="ignore"):
            v = (d11 * d20 - d01 * d21) / den
            w = (d00 * d21 - d01 * d20) / den
        u = 1.0 - v - w
        ok = (u >= -1e-12) & (v >= -1e-12) & (w >= -1e-12) & (den > 0)
        idx = np.nonzero(ok)[0]
        if len(idx) == 0:
            return None
        # largest facet containing the point (degenerate ties on shared edges)
        area = np.abs(den[idx])
        return idx[np.argmax(area)]

    def phases(self, rho, split=0.05):
        """Approximate coexisting phases at mean state rho: list of corner points."""
        k = self.facet_of(rho)
        if k is None:
            return [np.asarray(rho, float)]
        P = self.pts[self.simplices[k]]
        groups = []
        for p in P:
            for g in groups:
                if np.max(np.abs(g[0] - p)) < split:
                    g.append(p)
                    break
            else:
                groups.append([p])
        return [np.mean(g, axis=0) for g in groups]


def polish_two_phase(kT, a, b, rho_mean, ph1, ph2, tol=1e-13, maxit=100):
    """Newton polish of a two-phase tie line through rho_mean:
    mu^A, mu^B and p equal in both phases, and the mean on the tie line."""
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    m = np.asarray(rho_mean, float)
    x = np.concatenate([ph1, ph2]).astype(float)

    def resid(x):
        r1, r2 = x[:2], x[2:]
        mu1 = chemical_potential(kT, a, b, r1)
        mu2 = chemical_potential(kT, a, b, r2)
        p1 = pressure(kT, a, b, r1)
        p2 = pressure(kT, a, b, r2)
        d = r2 - r1
        e = m - r1
        return np.array([mu1[0] - mu2[0], mu1[1] - mu2[1], p1 - p2, d[0] * e[1] - d[1] * e[0]])

    for _ in range(maxit):
        F = resid(x)
        J = np.empty((4, 4))
        for k in range(4):
            h = 1e-7 * max(1.0, abs(x[k]))
            xp = x.copy(); xp[k] += h
            xm = x.copy(); xm[k] -= h
            J[:, k] = (resid(xp) - resid(xm)) / (2 * h)
        dx = np.linalg.solve(J, -F)
        # keep inside the domain
        lam = 1.0
        while True:
            xn = x + lam * dx
            ok = np.all(xn > 0) and b @ xn[:2] < 1 and b @ xn[2:] < 1
            if ok or lam < 1e-6:
                break
            lam *= 0.5
        x = xn
        if np.max(np.abs(lam * dx)) < tol:
            break
    return x[:2].copy(), x[2:].copy()


def polish_three_phase(kT, a, b, ph1, ph2, ph3, tol=1e-13, maxit=100):
    """Newton polish of a three-phase triangle: mu^A, mu^B, p equal in all three."""
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    x = np.concatenate([ph1, ph2, ph3]).astype(float)

    def resid(x):
        r = [x[0:2], x[2:4], x[4:6]]
        mu = [chemical_potential(kT, a, b, ri) for ri in r]
        p = [pressure(kT, a, b, ri) for ri in r]
        return np.array([mu[0][0] - mu[1][0], mu[0][1] - mu[1][1], p[0] - p[1],
                         mu[0][0] - mu[2][0], mu[0][1] - mu[2][1], p[0] - p[2]])

    for _ in range(maxit):
        F = resid(x)
        J = np.empty((6, 6))
        for k in range(6):
            h = 1e-7 * max(1.0, abs(x[k]))
            xp = x.copy(); xp[k] += h
            xm = x.copy(); xm[k] -= h
            J[:, k] = (resid(xp) - resid(xm)) / (2 * h)
        dx = np.linalg.solve(J, -F)
        x = x + dx
        if np.max(np.abs(dx)) < tol:
            break
    return x[0:2].copy(), x[2:4].copy(), x[4:6].copy()



def polish_invariant_point(kT, a, b, phases, tol=1e-14, maxit=100):
    """Newton solve for N + 1 coexisting phases of an N-component mixture (Sec. II: equal
    chemical potentials mu^c and equal pressure in every phase; with N + 1 phases at fixed
    kT the Gibbs phase rule leaves no freedom, so the point is isolated).  ``phases`` is a
    list of N + 1 starting density vectors; returns the polished list.  The Jacobian is
    analytic: d mu / d rho is the Hessian H of the free-energy density and
    d p / d rho = rho^T H (from dp = sum_c rho^c d mu^c)."""
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    P = len(phases)
    N = len(b)
    if P != N + 1:
        raise ValueError("an invariant point has N + 1 phases")
    x = np.concatenate([np.asarray(q, float) for q in phases])
    for _ in range(maxit):
        r = [x[q * N:(q + 1) * N] for q in range(P)]
        mu = [chemical_potential(kT, a, b, ri) for ri in r]
        p = [pressure(kT, a, b, ri) for ri in r]
        H = [hessian(kT, a, b, ri) for ri in r]
        F = np.zeros((P - 1) * (N + 1))
        J = np.zeros(((P - 1) * (N + 1), P * N))
        for q in range(1, P):
            row = (q - 1) * (N + 1)
            F[row:row + N] = mu[q] - mu[0]
            F[row + N] = p[q] - p[0]
            J[row:row + N, q * N:(q + 1) * N] = H[q]
            J[row:row + N, 0:N] = -H[0]
            J[row + N, q * N:(q + 1) * N] = r[q] @ H[q]
            J[row + N, 0:N] = -(r[0] @ H[0])
        dx = np.linalg.solve(J, -F)
        lam = 1.0
        while True:
            xn = x + lam * dx
            ok = np.all(xn > 0) and all(b @ xn[q * N:(q + 1) * N] < 1 for q in range(P))
            if ok or lam < 1e-6:
                break
            lam *= 0.5
        x = xn
        if np.max(np.abs(lam * dx) / np.maximum(np.abs(x), 1e-300)) < tol:
            break
    return [x[q * N:(q + 1) * N].copy() for q in range(P)]

def coexistence(kT, a, b, rho_mean, hull=None, n=600):
    """Coexisting phases for a two-component mean state: a list of 1, 2 or 3
    density pairs (one pair: the mean is a single stable phase)."""
    hull = hull or HullPhaseDiagram(kT, a, b, n=n)
    ph = hull.phases(rho_mean)
    if len(ph) == 2:
        return list(polish_two_phase(kT, a, b, rho_mean, ph[0], ph[1]))
    if len(ph) == 3:
        return list(polish_three_phase(kT, a, b, ph[0], ph[1], ph[2]))
    return [np.asarray(rho_mean, float)]
