"""Pins of the oracle's lattice Boltzmann step (Ridl & Wagner, Sec. III and V)
against invariants, closed forms, the paper's explicit D1Q3 update, textbook
coexistence and the spinodal criterion of the free energy.  CPU only."""
import numpy as np
import pytest
from scipy.optimize import root

import oracle
from oracle import thermo as T

THETA = 1.0 / 3.0


def lat(lattice, nx, ny, N, kT=0.6, gamma=0.5, a=None, kappa=0.1, lam=1.0, b=None, tau=1.0, **kw):
    a = np.full((N, N), 0.5) + 0.3 * np.eye(N) if a is None else np.asarray(a, float)
    b = np.full(N, 0.3) if b is None else np.asarray(b, float)
    K = np.full((N, N), kappa) if np.isscalar(kappa) else np.asarray(kappa, float)
    Lm = np.full((N, N), lam) if np.isscalar(lam) else np.asarray(lam, float)
    return oracle.Lattice(lattice, nx, ny, N, tau, kT, gamma, a, K, Lm, b, **kw)


def noisy(L, mean, sigma, seed):
    r = np.random.default_rng(seed)
    mean = np.asarray(mean, float).reshape(-1, 1, 1)
    return mean + r.normal(0, sigma, size=L.rshape())


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("lattice,ny", [("D1Q3", 1), ("D2Q9", 6)])
@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_uniform_rest_state_is_fixed_point(lattice, ny, N):
    L = lat(lattice, 8, ny, N)
    rho = np.broadcast_to(np.linspace(0.2, 0.5, N).reshape(N, 1, 1), L.rshape()).copy()
    f = L.equilibrium(rho)
    f2 = L.run(f, 20)
    assert np.max(np.abs(f2 - f)) < 1e-15


@pytest.mark.parametrize("lattice,nx,ny", [("D1Q3", 64, 1), ("D2Q9", 24, 20)])
@pytest.mark.parametrize("N", [2, 3])
def test_mass_conserved_per_component(lattice, nx, ny, N):
    L = lat(lattice, nx, ny, N)
    rho = noisy(L, np.linspace(0.25, 0.45, N), 0.02, 11)
    f = L.equilibrium(rho)
    m0 = L.free_energy(rho)[1]
    f = L.run(f, 300)
    r, _ = L.moments(f)
    m1 = L.free_energy(r)[1]
    assert np.max(np.abs(m1 - m0) / m0) < 1e-13


@pytest.mark.parametrize("lattice,ny,direction", [("D1Q3", 1, (1, 0)), ("D2Q9", 4, (1, 0)),
                                                  ("D2Q9", 4, (1, 1))])
@pytest.mark.parametrize("lam", [0.0, 0.5, 1.0, 4.0])
def test_friction_relaxation_closed_form(lattice, ny, direction, lam):
    # Uniform densities, opposite uniform velocities: no mean-field force, and the
    # implicit friction of Eq. forceFriction gives du_{n+1} = du_n (1 - lam/2)/(1 + lam/2)
    # while the total momentum stays fixed.
    L = lat(lattice, 6, ny, 2, lam=lam)
    d = L.d
    rho = np.empty(L.rshape()); rho[0] = 0.3; rho[1] = 0.5
    u = np.array([0.01, -0.006])
    mom = np.zeros(L.mshape())
    e = np.array(direction[:d], float)
    for c in range(2):
        for a in range(d):
            mom[c, a] = rho[c] * u[c] * e[a]
    f = L.equilibrium(rho, mom)
    P0 = mom.sum(axis=(0, 2, 3))
    r = (1 - lam / 2) / (1 + lam / 2)
    du0 = u[0] - u[1]
    for n in range(1, 6):
        f = L.run(f, 1)
        rr, j = L.moments(f)
        uu = j / rr[:, None]
        du = uu[0, 0] - uu[1, 0]
        assert np.max(np.abs(du - du0 * e[0] * r ** n)) < 1e-16
        assert np.max(np.abs(j.sum(axis=(0, 2, 3)) - P0)) < 1e-15


# symmetric friction matrix with distinct pair values and unequal densities, so that a
# transposed or shifted index, or a wrong sign, changes the result
LAM4 = np.array([[0.0, 0.5, 2.0, 1.3], [0.5, 0.0, 0.8, 3.0], [2.0, 0.8, 0.0, 0.25], [1.3, 3.0, 0.25, 0.0]])
RHO4 = np.array([0.3, 0.55, 0.42, 0.2])


@pytest.mark.parametrize("lattice,ny", [("D1Q3", 1), ("D2Q9", 4)])
@pytest.mark.parametrize("N", [3, 4])
def test_friction_n_components_uniform_relaxation_closed_form(lattice, ny, N):
    # Eq. forceFriction for N components: on a uniform state the mean-field force
    # vanishes, and the friction gain G = -L u-hat with u-hat = u + D^-1 G / 2 (D = diag
    # rho, L the weighted Laplacian of W^{cc'} = lambda^{cc'} rho^c rho^c' / (rho^c +
    # rho^c')) is the step's whole momentum change, j_{n+1} = j_n + G_n.  Eliminating G:
    #   u_{n+1} = (D + L/2)^-1 (D - L/2) u_n,
    # built here from the equation with numpy, independently of the oracle's pivoted
    # per-node solve.  1^T L = 0 makes the total momentum sum_c rho^c u^c invariant.
    L = lat(lattice, 6, ny, N, lam=LAM4[:N, :N], b=np.full(N, 0.3))
    d = L.d
    u0 = np.random.default_rng(7).normal(0.0, 0.01, (N, d))
    rho = np.empty(L.rshape())
    mom = np.zeros(L.mshape())
    for c in range(N):
        rho[c] = RHO4[c]
        for a in range(d):
            mom[c, a] = RHO4[c] * u0[c, a]
    W = np.zeros((N, N))
    for c in range(N):
        for cc in range(N):
            if c != cc:
                W[c, cc] = LAM4[c, cc] * RHO4[c] * RHO4[cc] / (RHO4[c] + RHO4[cc])
    Lap = np.diag(W.sum(axis=1)) - W
    D = np.diag(RHO4[:N])
    M = np.linalg.solve(D + 0.5 * Lap, D - 0.5 * Lap)
    P0 = (RHO4[:N, None] * u0).sum(axis=0)
    f = L.equilibrium(rho, mom)
    u = u0.copy()
    for n in range(1, 6):
        f = L.run(f, 1)
        u = M @ u
        r, j = L.moments(f)
        ug = (j / r[:, None]).reshape(N, d, -1)
        # u of order 1e-2: 1e-15 absolute is the rounding of the populations' moments
        assert np.max(np.abs(ug - u[:, :, None])) < 1e-15
        assert np.max(np.abs(r - rho)) < 1e-15
        P = j.sum(axis=(0, 2, 3)) / L.nodes
        assert np.max(np.abs(P - P0)) < 1e-16
    # the relaxation is real: the velocities moved by far more than the tolerance
    assert np.max(np.abs(u - u0)) > 1e-3


def test_nid_force_vanishes_for_ideal_mixture_at_matching_temperature():
    # Eq. forceMuId: G^{mu,c} = -rho^c D(gamma mu^c - theta ln rho^c).  With no attraction
    # (a = kappa = 0) and no excluded volume (b = 0), Eq. discreteChemicalPotential gives
    # mu^c = kT ln rho^c, so for gamma kT = theta the bracket vanishes identically and the
    # force is zero to rounding on any profile, while the "log" form (Eq. forceMuLog), a
    # different discretisation, leaves a residual of the order of the gradients.
    for lattice, nx, ny in (("D1Q3", 64, 1), ("D2Q9", 24, 20)):
        for kT in (THETA, 0.7):
            kw = dict(kT=kT, gamma=THETA / kT, a=np.zeros((2, 2)), kappa=0.0, b=[0.0, 0.0], lam=1.0)
            Lnid = lat(lattice, nx, ny, 2, force_method=1, **kw)
            Llog = lat(lattice, nx, ny, 2, force_method=0, **kw)
            rho = noisy(Lnid, [0.4, 0.7], 0.05, 3)
            f = Lnid.equilibrium(rho)
            G, Gmu = Lnid.forces(f)
            assert np.max(np.abs(Gmu)) < 1e-16
            assert np.max(np.abs(G)) < 1e-16       # at rest: no friction either
            _, Gmu_log = Llog.forces(f)
            assert np.max(np.abs(Gmu_log)) > 1e-3


@pytest.mark.parametrize("lattice", ["D1Q3", "D2Q9"])
def test_nid_and_log_forces_converge_at_second_order(lattice):
    # Both forces discretise the same continuum force, -gamma rho grad mu + theta grad rho
    # (rho grad ln rho = grad rho): they differ by theta (rho D ln rho - D rho), which for
    # second-order central differences is O(k^3) on a wave of wavenumber k, against a
    # force of O(k).  Refining the lattice (same profile on 2x the nodes) must divide the
    # difference by 8 and the relative difference by 4.
    a = np.array([[1.0, 0.9], [0.9, 0.6]])
    diffs, forces = [], []
    for n in (32, 64, 128, 256):
        ny = 1 if lattice == "D1Q3" else n
        kw = dict(kT=0.73, gamma=0.35, a=a, b=[0.25, 0.3], kappa=0.1)
        Lnid = lat(lattice, n, ny, 2, force_method=1, **kw)
        Llog = lat(lattice, n, ny, 2, force_method=0, **kw)
        x = np.arange(n)[None, :]
        y = np.arange(ny)[:, None]
        ph = 2 * np.pi * (x + (y if lattice == "D2Q9" else 0)) / n     # diagonal wave in 2-D
        rho = np.stack([0.48 + 0.1 * np.sin(ph), 0.72 + 0.08 * np.cos(ph + 0.3)])
        f = Lnid.equilibrium(rho)
        _, g_nid = Lnid.forces(f)
        _, g_log = Llog.forces(f)
        diffs.append(np.max(np.abs(g_nid - g_log)))
        forces.append(np.max(np.abs(g_log)))
    diffs, forces = np.array(diffs), np.array(forces)
    order_abs = np.log2(diffs[:-1] / diffs[1:])
    order_rel = np.log2((diffs / forces)[:-1] / (diffs / forces)[1:])
    assert np.all(np.abs(order_abs[1:] - 3.0) < 0.05) and abs(order_abs[0] - 3.0) < 0.1
    assert np.all(np.abs(order_rel[1:] - 2.0) < 0.05) and abs(order_rel[0] - 2.0) < 0.1


def test_momentum_bookkeeping():
    # Sec. III: collision and friction conserve the total momentum; the only change is
    # the sum over nodes of the mean-field forces (whose ideal part telescopes).
    L = lat("D2Q9", 20, 16, 2, a=[[1.0, 0.9], [0.9, 0.6]], b=[0.25, 0.3], kT=0.73, gamma=0.35)
    f = L.equilibrium(noisy(L, [0.48, 0.72], 0.01, 3))
    f = L.run(f, 50)
    for _ in range(3):
        _, j0 = L.moments(f)
        G, Gmu = L.forces(f)
        f = L.run(f, 1)
        _, j1 = L.moments(f)
        dP = j1.sum(axis=(0, 2, 3)) - j0.sum(axis=(0, 2, 3))
        assert np.max(np.abs(dP - Gmu.sum(axis=(0, 2, 3)))) < 1e-13
        # friction is an internal force: per node sum_c G^f = 0
        assert np.max(np.abs((G - Gmu).sum(axis=0))) < 1e-15


def test_mirror_symmetric_state_keeps_zero_momentum():
    L = lat("D1Q3", 64, 1, 2)
    rho = noisy(L, [0.3, 0.4], 0.02, 5)
    rho = 0.5 * (rho + rho[..., ::-1])          # mirror about x = 31.5
    f = L.run(L.equilibrium(rho), 200)
    _, j = L.moments(f)
    assert abs(j.sum()) < 1e-13


# ------------------------------------------------------------- D1Q3 update

def test_hermite_forms_equal_paper_explicit_d1q3_update():
    # Sec. V prints the D1Q3 update (collision + forcing) component by component.
    # It is applied here node by node with the oracle's forces G (stages 3-4) and
    # Psi of Eq. forceCorrectionsPsi, then streamed; the oracle's general Hermite
    # equilibrium/forcing must give the same populations.
    for tau in (1.0, 0.8):
        L = lat("D1Q3", 32, 1, 2, tau=tau)
        rho = noisy(L, [0.3, 0.45], 0.02, 9)
        mom = np.random.default_rng(2).normal(0, 0.005, L.mshape())
        f = L.equilibrium(rho, mom) + np.random.default_rng(4).normal(0, 1e-3, L.fshape())
        G, _ = L.forces(f)
        r, j = L.moments(f)
        new = np.empty_like(f)
        nx = L.nx
        for c in range(2):
            for x in range(nx):
                R, u, F = r[c, 0, x], j[c, 0, 0, x] / r[c, 0, x], G[c, 0, 0, x]
                lap = r[c, 0, (x + 1) % nx] - 2 * R + r[c, 0, (x - 1) % nx]
                Psi = -(1 / tau) * ((tau - 0.25) * F * F / R + lap / 12)
                f0, fp, fm = f[c, 0, 0, x], f[c, 1, 0, x], f[c, 2, 0, x]
                n0 = f0 + (1 / tau) * (R - R * THETA - R * u * u - f0) - (2 * F * u - Psi)
                npl = fp + (1 / tau) * (0.5 * (R * u * u + R * u + R * THETA) - fp) - (-F * u - 0.5 * F + 0.5 * Psi)
                nmi = fm + (1 / tau) * (0.5 * (R * u * u - R * u + R * THETA) - fm) - (-F * u + 0.5 * F + 0.5 * Psi)
                new[c, 0, 0, x] = n0
                new[c, 1, 0, (x + 1) % nx] = npl
                new[c, 2, 0, (x - 1) % nx] = nmi
        got = L.run(f, 1)
        assert np.max(np.abs(got - new)) < 1e-15


# ------------------------------------------------------- special cases

def test_identical_components_reduce_to_single_component():
    # Sec. VI: identical species (same a, b, kappa) at uniform composition behave as one
    # component: f^c = x_c f_single for every node, step and population.
    aa, bb = 0.45, 1 / 3
    xs = np.array([0.35, 0.65])
    L1 = lat("D1Q3", 64, 1, 1, kT=THETA, gamma=0.9, a=[[aa]], b=[bb])
    L2 = lat("D1Q3", 64, 1, 2, kT=THETA, gamma=0.9, a=np.full((2, 2), aa), b=[bb, bb], lam=1.0)
    xg = np.arange(64)
    tot = 0.3 + 1.5 * 0.5 * (np.tanh((xg - 16) / 3) - np.tanh((xg - 48) / 3))
    f1 = L1.run(L1.equilibrium(tot.reshape(L1.rshape())), 300)
    f2 = L2.run(L2.equilibrium(np.stack([xs[0] * tot, xs[1] * tot]).reshape(L2.rshape())), 300)
    for c in range(2):
        assert np.max(np.abs(f2[c] - xs[c] * f1[0])) < 1e-13


def test_d2q9_y_uniform_field_projects_onto_d1q3():
    # A D2Q9 field that does not depend on y evolves like the D1Q3 model: the D2Q9
    # weights, stencils and Hermite forms project onto those of Sec. V.
    N = 2
    a = [[1.0, 0.7], [0.7, 1.0]]
    L1 = lat("D1Q3", 48, 1, N, a=a, b=[0.25, 0.25], kT=0.9, gamma=0.1)
    L2 = lat("D2Q9", 48, 5, N, a=a, b=[0.25, 0.25], kT=0.9, gamma=0.1)
    rho1 = noisy(L1, [0.5, 0.5], 0.05, 8)
    rho2 = np.broadcast_to(rho1, L2.rshape()).copy()
    mom1 = np.random.default_rng(1).normal(0, 0.01, L1.mshape())
    mom2 = np.zeros(L2.mshape()); mom2[:, 0] = mom1[:, 0]
    f1 = L1.run(L1.equilibrium(rho1, mom1), 100)
    f2 = L2.run(L2.equilibrium(rho2, mom2), 100)
    r1, j1 = L1.moments(f1)
    r2, j2 = L2.moments(f2)
    assert np.max(np.abs(r2 - r1)) < 1e-12
    assert np.max(np.abs(j2[:, 0] - j1[:, 0])) < 1e-12
    assert np.max(np.abs(j2[:, 1])) < 1e-14


def test_d2q9_rotation_and_reflection_symmetry():
    L = lat("D2Q9", 16, 16, 2, a=[[1.0, 0.9], [0.9, 0.6]], b=[0.25, 0.3], kT=0.73, gamma=0.35)
    rho = noisy(L, [0.48, 0.72], 0.02, 13)
    r_a, _ = L.moments(L.run(L.equilibrium(rho), 60))
    rot = np.ascontiguousarray(np.rot90(rho, 1, axes=(1, 2)))
    r_b, _ = L.moments(L.run(L.equilibrium(rot), 60))
    assert np.max(np.abs(np.rot90(r_a, 1, axes=(1, 2)) - r_b)) < 1e-12
    ref = np.ascontiguousarray(rho[:, :, ::-1])
    r_c, _ = L.moments(L.run(L.equilibrium(ref), 60))
    assert np.max(np.abs(r_a[:, :, ::-1] - r_c)) < 1e-12


# ------------------------------------------------------- chemical potential

@pytest.mark.parametrize("lattice,nx,ny", [("D1Q3", 12, 1), ("D2Q9", 7, 6)])
def test_mu_is_derivative_of_lattice_free_energy(lattice, nx, ny):
    # Eq. discreteChemicalPotential: mu^c(x) = dF/drho^c(x), less the constant kT the
    # paper drops from d(rho ln rho)/d rho.
    N = 2
    L = lat(lattice, nx, ny, N, a=[[1.0, 0.7], [0.7, 0.8]], kappa=[[0.1, 0.05], [0.05, 0.2]], kT=0.7)
    rho = noisy(L, [0.4, 0.5], 0.05, 21)
    mu = L.mu(rho)
    h = 1e-6
    for (c, y, x) in [(0, 0, 3), (1, ny - 1, 0), (0, ny // 2, nx - 1)]:
        rp = rho.copy(); rp[c, y, x] += h
        rm = rho.copy(); rm[c, y, x] -= h
        fd = (L.free_energy(rp)[0] - L.free_energy(rm)[0]) / (2 * h)
        assert abs(fd - L.kT - mu[c, y, x]) < 1e-7


@pytest.mark.parametrize("lattice,ny", [("D1Q3", 1), ("D2Q9", 3)])
def test_uniform_mu_and_free_energy_match_bulk_thermodynamics(lattice, ny):
    N = 3
    a = np.array([[1.0, 0.6, 0.8], [0.6, 0.9, 0.7], [0.8, 0.7, 1.1]])
    b = np.array([0.25, 0.3, 0.2])
    L = lat(lattice, 5, ny, N, a=a, b=b, kT=0.8)
    r0 = np.array([0.2, 0.35, 0.3])
    rho = np.broadcast_to(r0.reshape(N, 1, 1), L.rshape()).copy()
    mu = L.mu(rho)
    want = T.chemical_potential(0.8, a, b, r0) - 0.8
    assert np.max(np.abs(mu - want.reshape(N, 1, 1))) < 1e-13
    F, _ = L.free_energy(rho)
    assert abs(F - L.nodes * T.free_energy_density(0.8, a, b, r0)) < 1e-12 * L.nodes


# ------------------------------------------------------- spinodal criterion

def _symbol_minus_laplacian(lattice, kx, ky=0.0):
    if lattice == "D1Q3":
        return 2.0 * (1.0 - np.cos(kx))
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    vx = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    vy = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
    return (2.0 / THETA) * np.sum(w * (1.0 - np.cos(kx * vx + ky * vy)))


@pytest.mark.parametrize("lattice", ["D1Q3", "D2Q9"])
def test_small_perturbations_grow_iff_free_energy_is_concave(lattice):
    # Sec. VI stability analysis on the lattice: a density wave exp(ikx) along the
    # softest direction grows iff H(rho) + kappa lambda_D(k) has a negative
    # eigenvalue, lambda_D the symbol of -Lap (the interaction psi of Sec. V).
    a = np.array([[1.0, 0.9], [0.9, 0.6]]); b = np.array([0.25, 0.3])
    kT = 0.85 * T.one_fluid_critical_temperature(a, b, [0.4, 0.6])
    kap = 0.1
    mean = 1.2 * np.array([0.4, 0.6])
    H = T.hessian(kT, a, b, mean)
    nx = 40
    ny = 1 if lattice == "D1Q3" else 4
    results = {}
    for m in (4, 10, 17):
        k = 2 * np.pi * m / nx
        K = H + kap * np.ones((2, 2)) * _symbol_minus_laplacian(lattice, k)
        ev, vec = np.linalg.eigh(K)
        L = lat(lattice, nx, ny, 2, a=a, b=b, kT=kT, gamma=0.35, kappa=kap)
        amp = 1e-6
        rho = mean.reshape(2, 1, 1) + amp * vec[:, 0].reshape(2, 1, 1) * np.cos(k * np.arange(nx)).reshape(1, 1, nx)
        rho = np.broadcast_to(rho, L.rshape()).copy()
        f = L.run(L.equilibrium(rho), 150)
        r, _ = L.moments(f)
        proj = np.einsum("c,cyx->yx", vec[:, 0], r - mean.reshape(2, 1, 1))
        a_k = 2 * np.abs(np.mean(proj * np.exp(-1j * k * np.arange(nx))))
        results[m] = (ev[0], a_k / amp)
    for m, (lmin, growth) in results.items():
        if lmin < -0.1:
            assert growth > 10.0, (m, lmin, growth)
        elif lmin > 0.05:
            assert growth < 1.0, (m, lmin, growth)
    assert any(v[0] < -0.1 for v in results.values()) and any(v[0] > 0.05 for v in results.values())


# ------------------------------------------------------- steady state

def _mu_flat_profile(L, guess):
    """Stationary point of the lattice free energy at fixed mass: mu(x) = const."""
    M = guess.sum()

    def resid(z):
        r = z[:-1]
        if np.any(r <= 0) or np.any(L.b[0] * r >= 1):
            return np.full_like(z, 1e3)
        mu = L.mu(r.reshape(L.rshape()))[0, 0]
        return np.concatenate([mu - z[-1], [r.sum() - M]])

    z0 = np.concatenate([guess, [L.mu(guess.reshape(L.rshape()))[0, 0].mean()]])
    z = root(resid, z0, method="hybr", options=dict(xtol=1e-14)).x
    # Newton polish with the exact Jacobian of the single-component D1Q3 mu:
    # d mu(x)/d rho(x) = kT (1/rho + 2b/eta + b^2 rho/eta^2) + 2 psi(0),
    # d mu(x)/d rho(x +- 1) = 2 psi(+-1) = -kappa
    n = len(guess)
    kT, a, b, kap = L.kT, L.a[0, 0], L.b[0], L.kappa[0, 0]
    for _ in range(4):
        r = z[:-1]
        eta = 1 - b * r
        J = np.zeros((n + 1, n + 1))
        J[np.arange(n), np.arange(n)] = kT * (1 / r + 2 * b / eta + b * b * r / eta ** 2) + 2 * (kap - a)
        J[np.arange(n), (np.arange(n) + 1) % n] = -kap
        J[np.arange(n), (np.arange(n) - 1) % n] = -kap
        J[:n, n] = -1.0
        J[n, :n] = 1.0
        z = z - np.linalg.solve(J, resid(z))
    res = resid(z)
    assert np.max(np.abs(res[:-1])) < 1e-14 and abs(res[-1]) < 1e-12
    return z[:-1]


@pytest.mark.parametrize("psi_sign,force,exact", [(-1.0, 0, True), (1.0, 0, False), (-1.0, 1, False)])
def test_mu_flat_profile_is_exact_fixed_point(psi_sign, force, exact):
    # The consistency correction Psi (Eq. forceCorrectionsPsi) with the "log" force
    # (Eq. forceMuLog) makes every profile with D mu = 0 an exact steady state once
    # the bare momentum carries -G/2 (u-hat = 0).  The opposite Psi sign, or the "nid"
    # force, leave a residual flow: this discriminates the readings of the signs.
    aa, bb = T.ab_from_critical(0.4, 1.0)
    rg, rl = T.maxwell_1c(THETA, aa, bb)
    nx = 64
    xg = np.arange(nx)
    # interfaces centred on nodes: the lattice-pinned position that is stable
    guess = rg + (rl - rg) * 0.5 * (np.tanh((xg - 16.0) / 2.5) - np.tanh((xg - 48.0) / 2.5))
    L = lat("D1Q3", nx, 1, 1, kT=THETA, gamma=0.3, a=[[aa]], b=[bb], kappa=0.3,
            psi_sign=psi_sign, force_method=force)
    Lref = lat("D1Q3", nx, 1, 1, kT=THETA, gamma=0.3, a=[[aa]], b=[bb], kappa=0.3)
    prof = _mu_flat_profile(Lref, guess).reshape(L.rshape())
    f = L.equilibrium(prof)
    _, Gmu = L.forces(f)
    f = L.equilibrium(prof, -0.5 * Gmu)
    f = L.run(f, 1)                  # relaxes the (non-conserved) second moment
    r0, j0 = L.moments(f)
    f = L.run(f, 50)
    r1, j1 = L.moments(f)
    change = max(np.max(np.abs(r1 - r0)), np.max(np.abs(j1 - j0)))
    if exact:
        assert change < 1e-13
        assert np.max(np.abs(r1[0, 0] - prof[0, 0])) < 1e-13
    else:
        assert change > 1e-6


@pytest.mark.slow
def test_slab_converges_to_maxwell_and_is_gamma_independent():
    # Sec. VI: equal mu and p in the bulk phases (Maxwell construction for one
    # component), and the equilibrium does not depend on gamma_mu (Eq. forceMuNid).
    aa, bb = T.ab_from_critical(0.4, 1.0)
    rg, rl = T.maxwell_1c(THETA, aa, bb)
    nx = 128
    xg = np.arange(nx)
    prof = rg + (rl - rg) * 0.5 * (np.tanh((xg - 32.0) / 2.5) - np.tanh((xg - 96.0) / 2.5))
    prof = prof + 1e-3 * np.cos(2 * np.pi * xg / nx)      # start away from equilibrium
    final = {}
    for g in (0.3, 0.15):
        L = lat("D1Q3", nx, 1, 1, kT=THETA, gamma=g, a=[[aa]], b=[bb], kappa=0.3)
        f = L.equilibrium(prof.reshape(L.rshape()))
        _, Gmu = L.forces(f)
        f = L.equilibrium(prof.reshape(L.rshape()), -0.5 * Gmu)
        f = L.run(f, 120000 if g == 0.3 else 240000)
        r, _ = L.moments(f)
        mu = L.mu(r)[0, 0]
        # steady state of the discrete scheme: D mu = 0, i.e. mu constant on each
        # sublattice.  The central difference does not see the period-2 mode, which the
        # start-up transient excites; bulk densities are therefore averaged over the two
        # sublattices.
        assert np.ptp(mu[0::2]) < 1e-11 and np.ptp(mu[1::2]) < 1e-11
        gas = 0.5 * (r[0, 0, 0] + r[0, 0, 1])
        liq = 0.5 * (r[0, 0, 64] + r[0, 0, 65])
        final[g] = (gas, liq)
        # kappa = 0.3 keeps the lattice pinning of the interfaces below 1e-6 (Sec. VI: ~1e-6)
        assert abs(gas - rg) < 2e-6 and abs(liq - rl) < 2e-6
    # the period-2 amplitude left by the transient depends on gamma and shifts the
    # sublattice averages at second order (~1e-8 here)
    assert abs(final[0.3][0] - final[0.15][0]) < 1e-7 and abs(final[0.3][1] - final[0.15][1]) < 1e-7


def test_kT_scaling_equivalence():
    # (kT, a, kappa, gamma) and (theta, a theta/kT, kappa theta/kT, gamma kT/theta)
    # give the same dynamics: mu is homogeneous of degree one in (kT, a, kappa) and only
    # gamma mu enters the force.
    kT = 0.9
    a = np.array([[1.0, 0.7], [0.7, 1.0]]); b = np.array([0.25, 0.25])
    s = THETA / kT
    L1 = lat("D2Q9", 12, 10, 2, kT=kT, gamma=0.2, a=a, b=b, kappa=0.1)
    L2 = lat("D2Q9", 12, 10, 2, kT=THETA, gamma=0.2 / s, a=a * s, b=b, kappa=0.1 * s)
    rho = noisy(L1, [0.5, 0.5], 0.03, 17)
    r1, _ = L1.moments(L1.run(L1.equilibrium(rho), 100))
    r2, _ = L2.moments(L2.run(L2.equilibrium(rho), 100))
    assert np.max(np.abs(r1 - r2)) < 1e-13


@pytest.mark.slow
def test_two_component_slab_lies_on_common_tangent():
    # Sec. VI: the bulk phases of a converged two-component slab coexist in the sense of
    # the free-energy minimisation -- equal mu^A, mu^B and p -- i.e. they are the ends of
    # the convex-hull tie line through their midpoint (Newton-polished).
    a = np.array([[1.0, 0.9], [0.9, 0.6]]); b = np.array([0.25, 0.3])
    kT = 0.85 * T.one_fluid_critical_temperature(a, b, [0.4, 0.6])
    hull = T.HullPhaseDiagram(kT, a, b, n=400)
    p1, p2 = sorted(T.coexistence(kT, a, b, 1.2 * np.array([0.4, 0.6]), hull=hull), key=lambda q: q.sum())
    nx, kap = 128, 0.3
    xg = np.arange(nx)
    s = 0.5 * (np.tanh((xg - 32.0) / 2.5) - np.tanh((xg - 96.0) / 2.5))
    rho = np.stack([p1[c] + (p2[c] - p1[c]) * s for c in range(2)]).reshape(2, 1, nx)
    L = lat("D1Q3", nx, 1, 2, kT=kT, gamma=1 / (6 * kap * p2.sum()), a=a, b=b, kappa=kap, lam=1.0)
    f = L.equilibrium(rho)
    _, Gmu = L.forces(f)
    f = L.run(L.equilibrium(rho, -0.5 * Gmu), 160000)
    r, _ = L.moments(f)
    mu = L.mu(r)
    assert np.max(np.ptp(mu[..., 0::2], axis=(1, 2))) < 1e-10
    gas = 0.5 * (r[:, 0, 0] + r[:, 0, 1])
    liq = 0.5 * (r[:, 0, 64] + r[:, 0, 65])
    mid = 0.5 * (gas + liq)
    ph = T.coexistence(kT, a, b, mid, hull=hull)
    assert len(ph) == 2
    q1, q2 = sorted(ph, key=lambda q: q.sum())
    assert np.max(np.abs(q1 - gas)) < 1e-5 and np.max(np.abs(q2 - liq)) < 1e-5


@pytest.mark.parametrize("lam", [0.5, 1.0, 4.0])
def test_interdiffusion_follows_maxwell_stefan_fick_law(lam):
    # Sec. IV: with friction lambda between two components, a composition wave at fixed
    # total density relaxes by Fickian interdiffusion; for two components the
    # Maxwell-Stefan relation gives -gamma D(mu^A - mu^B) = lambda (u^A - u^B), so
    # the mode exp(ikx) decays at rate gamma rho^A rho^B h k^2 / (rho lambda), with
    # h = H_AA - H_AB - H_BA + H_BB the bulk Hessian along the composition direction.
    a = np.array([[1.0, 0.7], [0.7, 1.0]]); b = np.array([0.25, 0.25])
    kT = 1.2 * T.one_fluid_critical_temperature(a, b, [0.5, 0.5])
    nx, gam, rA, rho, eps = 128, 0.5, 0.5, 1.0, 1e-4
    x = np.arange(nx)
    k = 2 * np.pi / nx
    H = T.hessian(kT, a, b, np.array([rA, rho - rA]))
    h = H[0, 0] - H[0, 1] - H[1, 0] + H[1, 1]
    L = lat("D1Q3", nx, 1, 2, kT=kT, gamma=gam, a=a, b=b, kappa=0.1, lam=[[0, lam], [lam, 0]])
    r0 = np.stack([rA + eps * np.cos(k * x), rho - rA - eps * np.cos(k * x)]).reshape(L.rshape())
    f = L.equilibrium(r0)
    ts, amps = [], []
    for t in range(1, 41):
        f = L.run(f, 200)
        r, _ = L.moments(f)
        ts.append(200 * t)
        amps.append(np.abs(np.mean(0.5 * (r[0, 0] - r[1, 0]) * np.exp(-1j * k * x))))
    rate = -np.polyfit(ts[15:], np.log(amps[15:]), 1)[0]
    predicted = gam * rA * (rho - rA) * h * k * k / (rho * lam)
    assert abs(rate / predicted - 1) < 0.01


@pytest.mark.parametrize("force", ["nid", "log"])
@pytest.mark.parametrize("lam", [0.5, 2.0])
def test_ideal_mixture_interdiffusion_is_linear_at_large_amplitude(force, lam):
    # lambda in nonlinear dynamics (Sec. IV, Eq. MaxwellStefan): for an ideal mixture
    # (a = kappa = 0, equal b, so eta depends on the total density only) at uniform total
    # density rho, the Maxwell-Stefan balance lambda rho^A rho^B (u^A - u^B) / rho =
    # -gamma (rho^B rho^A D mu^A - rho^A rho^B D mu^B) / rho gives the flux
    # J^A = -(gamma kT / lambda) D rho^A: linear diffusion whatever the composition.
    # (With the "nid" force at gamma kT = theta the mean-field force vanishes and the
    # lattice's own pressure theta rho^c drives it, so D = theta / lambda.)  A composition
    # wave from x = 0.1 to 0.9 therefore decays at the small-amplitude rate, with no even
    # harmonics (the dynamics are odd under A <-> B); the friction's composition weight
    # rho^A rho^B / (rho^A + rho^B) and the implicit u-hat must cancel the driving force's
    # composition dependence exactly, which a linearised check cannot see.
    nx, rho, kT = 256, 1.6, 0.5
    gam = THETA / kT if force == "nid" else 0.6
    k = 2 * np.pi / nx
    x = np.arange(nx)
    rates, last = {}, {}
    for A in (0.005, 0.4):
        L = lat("D1Q3", nx, 1, 2, kT=kT, gamma=gam, a=np.zeros((2, 2)), kappa=0.0, b=[0.2, 0.2],
                lam=[[0, lam], [lam, 0]], force_method=1 if force == "nid" else 0)
        xa = 0.5 + A * np.cos(k * x)
        f = L.equilibrium(np.stack([rho * xa, rho * (1 - xa)]).reshape(L.rshape()))
        ts, a1, a2, a3 = [], [], [], []
        for t in range(1, 41):
            f = L.run(f, 250)
            r, _ = L.moments(f)
            d = 0.5 * (r[0, 0] - r[1, 0])
            ts.append(250 * t)
            a1.append(abs(np.mean(d * np.exp(-1j * k * x))))
            a2.append(abs(np.mean(d * np.exp(-2j * k * x))))
            a3.append(abs(np.mean(d * np.exp(-3j * k * x))))
        a1 = np.array(a1)
        rates[A] = -np.polyfit(ts[5:], np.log(a1[5:]), 1)[0]
        last[A] = a1[-1] / (rho * A)
        assert max(np.array(a2) / a1) < 1e-9
        # measured up to 1.0e-4 (the lattice's own weak nonlinearity); composition-dependent
        # mistakes in the friction or the force give 1e-3 to 1e-1
        assert max(np.array(a3) / a1) < 5e-4
    predicted = (THETA if force == "nid" else gam * kT) * k * k / lam
    assert abs(rates[0.005] / predicted - 1) < 0.005
    # measured up to 7.1e-6 ("log", lambda = 2); those mistakes move it by 1.7e-4 to 7e-2
    assert abs(rates[0.4] / rates[0.005] - 1) < 5e-5
    assert abs(last[0.4] / last[0.005] - 1) < 1e-4


# ------------------------------------------------------------ MRT collision (D2Q9)

def test_mrt_with_equal_relaxation_times_is_bgk():
    # Eq. BGKcollisionOperator with the collision matrix diagonal in the Hermite moment
    # basis: when every eigenvalue is 1/tau the matrix is (1/tau) I and the step is BGK.
    for tau in (1.0, 0.8):
        kw = dict(tau=tau, a=[[1.0, 0.9], [0.9, 0.6]], b=[0.25, 0.3], kT=0.73, gamma=0.35)
        L0 = lat("D2Q9", 24, 20, 2, **kw)
        L1 = lat("D2Q9", 24, 20, 2, tau_s=tau, tau_g=tau, **kw)
        f = L0.equilibrium(noisy(L0, [0.48, 0.72], 0.01, 3))
        f = L0.run(f, 20) + np.random.default_rng(8).normal(0, 1e-4, L0.fshape())
        # a few ulps of the populations (~0.3); a wrong norm or sign would show at ~1e-5
        assert np.max(np.abs(L1.run(f, 1) - L0.run(f, 1))) < 1e-15


@pytest.mark.parametrize("tau_s", [0.55, 0.7, 0.9])
def test_mrt_shear_wave_decays_at_shear_viscosity(tau_s):
    # A transverse wave u_y = U sin(kx) in an ideal gas (no force) decays at nu k^2 with
    # the kinematic viscosity nu = theta (tau_s - 1/2) of the shear moments: the shear
    # eigenvalue alone sets it, whatever the bulk and ghost relaxation times (the ghosts
    # enter only the O(k^2) lattice correction, ~1e-4 at k = 2 pi / 128).
    nx = 128
    k = 2 * np.pi / nx
    x = np.arange(nx)
    rates = []
    for tau_g in (0.8, 1.2):
        L = lat("D2Q9", nx, 4, 1, tau=1.0, tau_s=tau_s, tau_g=tau_g, a=[[0.0]], kappa=0.0, b=[0.0],
                kT=THETA, gamma=1.0)
        mom = np.zeros(L.mshape())
        mom[0, 1] = 1e-4 * np.sin(k * x)[None, :]
        f = L.equilibrium(np.ones(L.rshape()), mom)
        ts, amps = [], []
        for t in range(1, 21):
            f = L.run(f, 50)
            _, j = L.moments(f)
            ts.append(50 * t)
            amps.append(np.abs(np.mean(j[0, 1].mean(axis=0) * np.exp(-1j * k * x))))
        rates.append(-np.polyfit(ts, np.log(amps), 1)[0])
    nu = THETA * (tau_s - 0.5)
    for r in rates:
        assert abs(r / (nu * k * k) - 1) < 5e-4
    assert abs(rates[0] - rates[1]) < 5e-4 * rates[0]


@pytest.mark.parametrize("tau_s", [0.55, 0.8])
def test_mrt_diagonal_shear_wave_decays_at_shear_viscosity(tau_s):
    # The same for a wave along the lattice diagonal, k = (1, 1) 2 pi / n, with velocity
    # along (1, -1): its shear stress lies in the H_xx - H_yy moment (the transverse wave
    # along x checks H_xy), which must relax with the shear time as well.
    n = 64
    k1 = 2 * np.pi / n
    L = lat("D2Q9", n, n, 1, tau=1.0, tau_s=tau_s, tau_g=1.0, a=[[0.0]], kappa=0.0, b=[0.0], kT=THETA, gamma=1.0)
    X, Y = np.meshgrid(np.arange(n), np.arange(n))
    phase = np.exp(1j * k1 * (X + Y))
    mom = np.zeros(L.mshape())
    mom[0, 0] = 1e-4 * np.sin(k1 * (X + Y))
    mom[0, 1] = -mom[0, 0]
    f = L.equilibrium(np.ones(L.rshape()), mom)
    ts, amps = [], []
    for t in range(1, 21):
        f = L.run(f, 20)
        _, j = L.moments(f)
        ts.append(20 * t)
        amps.append(np.abs(np.mean((j[0, 0] - j[0, 1]) * np.conj(phase))))
    rate = -np.polyfit(ts, np.log(amps), 1)[0]
    assert abs(rate / (THETA * (tau_s - 0.5) * 2 * k1 * k1) - 1) < 2e-3


@pytest.mark.parametrize("tau_g", [0.6, 1.3])
def test_mrt_ghost_relaxation_keeps_mu_flat_fixed_point(tau_g):
    # the ghost moments (third and fourth order) carry no hydrodynamics: relaxing them at
    # their own rate leaves every D mu = 0 profile an exact steady state (planar profile in
    # D2Q9, built as in the D1Q3 fixed-point test)
    aa, bb = T.ab_from_critical(0.4, 1.0)
    rg, rl = T.maxwell_1c(THETA, aa, bb)
    nx = 64
    xg = np.arange(nx)
    guess = rg + (rl - rg) * 0.5 * (np.tanh((xg - 16.0) / 2.5) - np.tanh((xg - 48.0) / 2.5))
    Lref = lat("D1Q3", nx, 1, 1, kT=THETA, gamma=0.3, a=[[aa]], b=[bb], kappa=0.3)
    prof = _mu_flat_profile(Lref, guess)
    L = lat("D2Q9", nx, 2, 1, kT=THETA, gamma=0.3, a=[[aa]], b=[bb], kappa=0.3, tau=1.0, tau_s=1.0, tau_g=tau_g)
    P = np.broadcast_to(prof.reshape(1, 1, nx), (1, 2, nx)).copy()
    f = L.equilibrium(P)
    _, Gmu = L.forces(f)
    f = L.run(L.equilibrium(P, -0.5 * Gmu), 1)
    r0, j0 = L.moments(f)
    f = L.run(f, 50)
    r1, j1 = L.moments(f)
    assert max(np.max(np.abs(r1 - r0)), np.max(np.abs(j1 - j0))) < 1e-13


def test_mrt_momentum_bookkeeping_and_mass():
    # the collision conserves rho^c and rho^c u^c for any relaxation times (Sec. III):
    # total momentum changes by the sum of the mean-field forces only, mass not at all
    L = lat("D2Q9", 20, 16, 2, a=[[1.0, 0.9], [0.9, 0.6]], b=[0.25, 0.3], kT=0.73, gamma=0.35, tau=1.0,
            tau_s=0.65, tau_g=0.8)
    f = L.equilibrium(noisy(L, [0.48, 0.72], 0.01, 3))
    m0 = L.moments(f)[0].sum(axis=(1, 2))
    f = L.run(f, 50)
    for _ in range(3):
        _, j0 = L.moments(f)
        G, Gmu = L.forces(f)
        f = L.run(f, 1)
        r1, j1 = L.moments(f)
        dP = j1.sum(axis=(0, 2, 3)) - j0.sum(axis=(0, 2, 3))
        assert np.max(np.abs(dP - Gmu.sum(axis=(0, 2, 3)))) < 1e-13
    assert np.max(np.abs(r1.sum(axis=(1, 2)) - m0) / m0) < 1e-14


def test_mrt_low_shear_viscosity_stays_stable_where_bgk_does_not():
    # with the Psi correction, BGK at tau = 0.6 amplifies density noise in an ideal gas,
    # while a bulk time tau = 1 with the shear time 0.6 (same viscosity) keeps it bounded;
    # shear times above the bulk time are unstable (the library rejects them)
    def grows(**kw):
        L = lat("D2Q9", 32, 32, 1, a=[[0.0]], kappa=0.0, b=[0.0], kT=THETA, gamma=1.0, **kw)
        f = L.equilibrium(noisy(L, [1.0], 1e-6, 1))
        try:
            r, _ = L.moments(L.run(f, 1500))
        except oracle.OracleDomainError:
            return True
        return np.max(np.abs(r - 1.0)) > 1e-6
    assert grows(tau=0.6)
    assert not grows(tau=1.0, tau_s=0.6, tau_g=1.0)
    assert grows(tau=1.0, tau_s=1.2, tau_g=1.0)


def test_two_step_window_reference_equals_direct_two_steps():
    """The exact two-step reference that the full-size chained GPU test builds from one-step
    9 x 9 windows (tests/oracle_windows.py) equals two oracle steps of the whole periodic
    lattice at every sampled node."""
    import lbinputs
    from oracle_windows import oracle_two_steps_at

    p = lbinputs.base_params("c2")
    kw = lbinputs.lib_kwargs(p)
    n = 24
    rho = lbinputs.fields("c2", n, n)
    lat = oracle.Lattice("D2Q9", n, n, 2, kw["tau"], kw["kT"], kw["gamma_mu"], kw["a"], kw["kappa"], kw["lam"],
                         kw["b"])
    f0 = lat.run(lat.equilibrium(rho), 50)
    r2, j2 = lat.moments(lat.run(f0, 2))
    win9 = oracle.Lattice("D2Q9", 9, 9, 2, kw["tau"], kw["kT"], kw["gamma_mu"], kw["a"], kw["kappa"], kw["lam"],
                          kw["b"])
    for (y, x) in [(0, 0), (5, 17), (23, 23), (11, 3)]:
        ro, jo = oracle_two_steps_at(win9, f0, y, x)
        assert np.array_equal(ro, r2[:, y, x]) and np.array_equal(jo, j2[:, :, y, x])
